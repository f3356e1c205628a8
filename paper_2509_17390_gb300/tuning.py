"""Autotuning of BVH width, sensor tile shape and launch options, with a
JSON cache.

Width and tile shape are properties of the scene and sensor objects, so this
layer builds the variants and calls the native coordinate-descent tuner
(fgl_autotune) once per (width, tile) pair.  Results change speed only; every
variant returns bitwise identical ranges and triangle ids.
"""

from __future__ import annotations

import json
import os
import threading
from typing import Dict, Iterable, Optional, Sequence, Tuple

from . import BatchOpts, Scene, Sensor, autotune

DEFAULT_WIDTHS = (8, 4)
DEFAULT_TILES = ((4, 8), (2, 16), (8, 4), (1, 32))
_lock = threading.Lock()


def _gpu_name() -> str:
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def workload_key(n_tris: int, sensor_rows: int, sensor_cols: int, n_env: int) -> str:
    """Cache key: scene size class, sensor grid, environments (power-of-two
    bucket) and GPU."""
    env_bucket = 1 << max(0, (max(1, n_env) - 1).bit_length())
    tri_bucket = 1 << max(0, (max(1, n_tris) - 1).bit_length())
    return f"tris<={tri_bucket}|sensor={sensor_rows}x{sensor_cols}|envs<={env_bucket}|{_gpu_name()}"


def load_cache(path: str) -> Dict[str, dict]:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(path: str, key: str, value: dict) -> None:
    with _lock:
        data = load_cache(path)
        data[key] = value
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def opts_from_dict(d: dict) -> BatchOpts:
    return BatchOpts(**{k: int(v) for k, v in d.items() if k in dict(BatchOpts._fields_)})


def tune_workload(verts, tris, sensor_table, poses, max_range: float,
                  widths: Sequence[int] = DEFAULT_WIDTHS,
                  tiles: Sequence[Tuple[int, int]] = DEFAULT_TILES,
                  cache_path: Optional[str] = None, reps: int = 3, passes: int = 2,
                  use_graph: bool = True, stream=None, scenes: Optional[Dict[int, Scene]] = None):
    """Pick (width, tile, launch options) for casting ``sensor_table`` from
    ``poses`` (a CUDA float32 [n_env,3,4] tensor) against the mesh.

    Returns a dict {"width", "tile", "opts", "ms", "trials", "key", "cached"}.
    ``scenes`` may pass already built scenes by width to avoid rebuilding.
    """
    import torch

    n_env = poses.shape[0]
    key = workload_key(len(tris), sensor_table.rows, sensor_table.cols, n_env)
    if cache_path:
        hit = load_cache(cache_path).get(key)
        if hit:
            return {**hit, "key": key, "cached": True}
    scenes = dict(scenes or {})
    if stream is None and use_graph:
        stream = torch.cuda.Stream(device=poses.device)   # graphs need a capturable stream
    best = None
    trials = 0
    n = n_env * sensor_table.n_rays
    out_r = torch.empty(n, dtype=torch.float32, device=poses.device)
    out_i = torch.empty(n, dtype=torch.int32, device=poses.device)
    for W in widths:
        if W not in scenes:
            scenes[W] = Scene(verts, tris, width=W)
        for tile in tiles:
            sensor = Sensor.from_table(sensor_table, *tile)
            items = [(scenes[W], sensor, poses, max_range, out_r, out_i)]
            opts, res = autotune(items, BatchOpts(use_graph=1 if use_graph else 0), reps=reps,
                                 passes=passes, stream=stream)
            trials += res["trials"]
            if best is None or res["best_ms"] < best["ms"]:
                best = {"width": W, "tile": list(tile), "opts": opts.as_dict(), "ms": res["best_ms"]}
            sensor.close()
    torch.cuda.synchronize(poses.device)
    best["trials"] = trials
    if cache_path:
        store_cache(cache_path, key, best)
    return {**best, "key": key, "cached": False}
