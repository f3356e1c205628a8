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
  hetero_batch  : 8 meshes extracted (density, TSDF, marching tetrahedra;
                  the mesher is passed in: the GPU pipeline in the bench, the
                  oracle's in the tests) from 50k-2M seeded Gaussians on
                  open-topped rooms of growing size, voxels 5 cm -> 2 cm
                  (about 90k -> 5M triangles), each on a grid covering its room
                  plus MESH_MARGIN; 256 environments assigned round-robin to the
                  meshes, each with a sensor drawn from 16/32/64/128 beams x
                  360-2048 azimuths or the 20k-ray rosette.
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


# (room extent m, boxes, spheres, Gaussians, voxel m): about 17 * area / voxel^2
# triangles each, from ~50k to ~5M
HETERO_LADDER = [
    ((2.0, 1.5, 1.0), 1, 1, 50_000, 0.05),
    ((2.5, 2.0, 1.2), 2, 1, 85_000, 0.05),
    ((3.0, 2.5, 1.5), 2, 2, 145_000, 0.04),
    ((3.5, 3.0, 1.8), 3, 2, 250_000, 0.035),
    ((4.5, 3.5, 2.0), 3, 3, 420_000, 0.03),
    ((5.0, 4.0, 2.5), 4, 3, 720_000, 0.025),
    ((6.0, 4.5, 2.6), 5, 4, 1_200_000, 0.022),
    ((6.0, 5.0, 3.0), 6, 4, 2_000_000, 0.02),
]


@dataclasses.dataclass
class MeshSpec:
    verts: np.ndarray
    tris: np.ndarray
    obstacles: object
    voxel: float
    n_gauss: int
    stats: dict


# grid margin around each room: 3 sigma of the largest Gaussian (20 cm), the
# 6 cm TSDF band and a few voxels, so the level set never meets the grid's faces
MESH_MARGIN = 0.75

_HETERO_CACHE: dict = {}


def hetero_grid(room, h):
    """(origin, dims) of a ladder set's grid: the room plus MESH_MARGIN."""
    from .gaussians import grid_around
    return grid_around((0.0, 0.0, 0.0), room, h, MESH_MARGIN)


def hetero_meshes(mesher, seed: int = 4, ladder=None) -> List[MeshSpec]:
    """The heterogeneous workload's meshes: each ladder set's Gaussians on its
    hetero_grid, turned into a mesh by mesher(gs, origin, h, dims) ->
    (verts f32 [nv, 3], tris i32 [nt, 3]).  Set k of the ladder uses seed
    seed * 100 + k.  Cached per process, mesher, seed and set, so a prefix of
    the ladder shares its meshes with the whole ladder."""
    from . import gaussians
    ladder = HETERO_LADDER if ladder is None else ladder
    name = getattr(mesher, "__qualname__", repr(mesher))
    out = []
    for k, (room, nb, ns, ng, h) in enumerate(ladder):
        key = (name, seed, k, (tuple(room), nb, ns, ng, h))
        if key not in _HETERO_CACHE:
            gs, obs = gaussians.gaussian_room(seed * 100 + k, room, ng, nb, ns, with_obstacles=True)
            origin, dims = hetero_grid(room, h)
            v, t = mesher(gs, origin, h, dims)
            _HETERO_CACHE[key] = MeshSpec(np.ascontiguousarray(v, np.float32),
                                          np.ascontiguousarray(t, np.int32), obs, h, ng, {"dims": dims})
        out.append(_HETERO_CACHE[key])
    return out


def hetero_sensors(seed: int = 4):
    return _sensors.mixed_sensors(seed)


def hetero_envs(seed: int, meshes: List[MeshSpec], n_env: int = 256):
    """Environments assigned round-robin to the meshes, each with a sensor
    index into hetero_sensors() and a free upright pose (random yaw) in its
    room.  Returns a list of (mesh index, sensor index, pose[3,4])."""
    rng = np.random.default_rng(seed + 7)
    n_sensors = len(_sensors.MIXED_BEAMS) * len(_sensors.MIXED_AZ) + 1
    envs = []
    for e in range(n_env):
        m = e % len(meshes)
        s = int(rng.integers(n_sensors))
        P = _poses.sample_free_pose(rng, meshes[m].obstacles, 1, margin=0.25)
        envs.append((m, s, P[0]))
    return envs


@dataclasses.dataclass
class WalkInstances:
    meshes: list          # [(verts f32 [nv, 3], tris i32 [nt, 3])] in instance frames
    poses: np.ndarray     # [S, n_env, K, 3, 4] instance-to-world per step
    walk: object          # the batched_walk these ride on


def walk_instances(seed: int, n_env: int, n_steps: int, walk=None) -> WalkInstances:
    """Four rigid instances per environment of the batched walk (an
    icosphere of radius 0.3 m, two subdivided boxes and a 1.8 m pillar), each
    0.6-1.2 m from its environment's sensor horizontally (the walk's scene is
    cluttered: half of its returns lie within 0.5 m), turning 0.05 rad and
    drifting 5 mm a step."""
    from .scenes import aabb_box, icosphere_unit
    w = batched_walk(seed, n_env=n_env, n_steps=n_steps) if walk is None else walk
    S = w.poses.shape[0]
    uv, ut = icosphere_unit(3)
    meshes = [((0.3 * uv).astype(np.float32), ut),
              aabb_box((-0.4, -0.3, -0.3), (0.4, 0.3, 0.3), 4),
              aabb_box((-0.25, -0.25, -0.25), (0.25, 0.25, 0.25), 4),
              aabb_box((-0.1, -0.1, -0.9), (0.1, 0.1, 0.9), 3)]
    K = len(meshes)
    rng = np.random.default_rng(77)
    ang = rng.uniform(0, 2 * np.pi, (n_env, K))
    rad = rng.uniform(0.6, 1.2, (n_env, K))
    base = np.stack([rad * np.cos(ang), rad * np.sin(ang), rng.uniform(-0.2, 0.2, (n_env, K))], -1)
    yaw0 = rng.uniform(0, 2 * np.pi, (n_env, K))
    IP = np.zeros((S, n_env, K, 3, 4), np.float32)
    for st in range(S):
        a = yaw0 + 0.05 * st
        c, sn = np.cos(a), np.sin(a)
        IP[st, :, :, 0, 0], IP[st, :, :, 0, 1], IP[st, :, :, 1, 0], IP[st, :, :, 1, 1] = c, -sn, sn, c
        IP[st, :, :, 2, 2] = 1
        IP[st, :, :, :, 3] = w.poses[st][:, None, :, 3] + base + 0.005 * st
    return WalkInstances(meshes, IP, w)

