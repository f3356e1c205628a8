"""The named ray-casting workloads as seeded inputs.

  tiny_cast     : 10x8x3 m room + 8 boxes (108 tris), one pose, 16 beams over
                  -15..+15 deg x 360 azimuths (5,760 rays), max range 100 m.
  indoor_scan   : 20x15x4 m room with 2,000 icospheres and 834 subdivided boxes
                  (1,000,300 tris), one pose, 32 beams over -16..+15 deg x
                  1,800 azimuths (57,600 rays), max range 120 m.
  batched_walk  : the indoor_scan mesh, 4,096 environments each following a
                  seeded SE(3) random walk (0.1 m / 2 deg per step) over 100
                  steps, 16 x 360 rays per environment (23.6 M rays per step),
                  max range 120 m.
"""

from __future__ import annotations

import dataclasses
from typing import List

import numpy as np

from . import poses as _poses
from . import scenes as _scenes
from . import sensors as _sensors


@dataclasses.dataclass
class Workload:
    name: str
    verts: np.ndarray
    tris: np.ndarray
    sensor: _sensors.SensorTable
    poses: np.ndarray          # [n_env, 3, 4] or [n_steps, n_env, 3, 4]
    max_range: float
    obstacles: object = None

    @property
    def n_rays_per_step(self) -> int:
        n_env = self.poses.shape[-3]
        return n_env * self.sensor.n_rays


def tiny_cast(seed: int = 1) -> Workload:
    v, t, obs = _scenes.tiny_room_scene(seed)
    P = _poses.sample_free_pose(np.random.default_rng(seed + 1000), obs, 1)
    return Workload("tiny_cast", v, t, _sensors.grid_sensor(16, -15.0, 15.0, 360), P, 100.0, obs)


_INDOOR_CACHE: dict = {}


def indoor_mesh(seed: int = 2):
    if seed not in _INDOOR_CACHE:
        _INDOOR_CACHE[seed] = _scenes.indoor_scene(seed)
    return _INDOOR_CACHE[seed]


def indoor_scan(seed: int = 2) -> Workload:
    v, t, obs = indoor_mesh(seed)
    P = _poses.sample_free_pose(np.random.default_rng(seed + 1000), obs, 1)
    return Workload("indoor_scan", v, t, _sensors.grid_sensor(32, -16.0, 15.0, 1800), P, 120.0, obs)


def batched_walk(seed: int = 2, n_env: int = 4096, n_steps: int = 100) -> Workload:
    v, t, obs = indoor_mesh(seed)
    W = _poses.random_walk(np.random.default_rng(seed + 2000), obs, n_env, n_steps)
    return Workload("batched_walk", v, t, _sensors.grid_sensor(16, -15.0, 15.0, 360), W, 120.0, obs)
