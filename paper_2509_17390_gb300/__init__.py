"""Python binding of libfgl (include/fgl.h): batched LiDAR ray casting on GB300.

Argument marshalling only -- every step of the ray-casting path runs in the
CUDA kernels of libfgl.so.  Device buffers are torch CUDA tensors (their
data_ptr is passed through); streams are torch.cuda.Stream objects or raw
cudaStream_t integers.  There is no CPU fallback: if the native library is
missing and cannot be built, importing the binding's functions raises.
"""

from __future__ import annotations

import ctypes
import os
import threading
from typing import Iterable, Optional, Sequence

import numpy as np

from . import build_native

__all__ = ["Scene", "Sensor", "BatchOpts", "cast", "cast_opts", "cast_batched",
           "cast_batched_host", "cast_batched_static", "autotune", "TuneOpts", "world_rays", "sync", "work_counters", "FglError", "lib",
           "gaussian_density", "Gaussians", "Grid", "Lbvh", "denoise", "tsdf", "marching_tets",
           "mesh_from_surface", "mesh_from_gaussians"]

FGL_OK, FGL_ERR_INVALID, FGL_ERR_OOM, FGL_ERR_CUDA = 0, 1, 2, 3
FGL_ERR_BUDGET, FGL_ERR_TIMEOUT, FGL_ERR_CANCELLED, FGL_ERR_DEVICE = 4, 5, 6, 7
FGL_ERR_CAPACITY = 8
FGL_ERR_INTERNAL = 9
STATUS_NAMES = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "BUDGET", 5: "TIMEOUT",
                6: "CANCELLED", 7: "DEVICE", 8: "CAPACITY"}


class FglError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"fgl {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


P = ctypes.c_void_p
I32, I64, F32, F64, U64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double, ctypes.c_uint64


class BuildOpts(ctypes.Structure):
    _fields_ = [("width", I32), ("sah_bins", I32), ("n_threads", I32), ("upload", I32)]


class SceneStats(ctypes.Structure):
    _fields_ = [("n_tris", I64), ("n_nodes", I64), ("node_bytes", I64), ("tri_bytes", I64),
                ("width", I32), ("node_stride", I32), ("depth", I32), ("resident", I32),
                ("sah_cost", F64), ("build_ms", F64), ("bounds_lo", F32 * 3),
                ("bounds_hi", F32 * 3), ("margin", F32)]


class CastItem(ctypes.Structure):
    _fields_ = [("scene", P), ("sensor", P), ("poses", P), ("n_env", I32), ("max_range", F32),
                ("out_range", P), ("out_tri", P), ("min_range", F32), ("out_points", P),
                ("n_instances", I32), ("instances", P), ("instance_poses", P), ("out_instance", P)]


class BatchOpts(ctypes.Structure):
    """Launch options (fgl_batch_opts); 0 in a field selects its default."""
    _fields_ = [("packet_rays", I32), ("block_threads", I32), ("stack_smem", I32),
                ("blocks_per_sm", I32), ("use_graph", I32), ("refill_min", I32),
                ("postpone_pct", I32), ("count_work", I32), ("tri_mode", I32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def lib():
    """Load (building in-tree first if needed) libfgl.so; with the
    environment variable FGL_CHECKED=1 set before the first call, the checked
    library libfgl_checked.so (bounds-checked traversal, for debugging)."""
    global _lib
    with _lock:
        if _lib is None:
            checked = os.environ.get("FGL_CHECKED") == "1"
            path = build_native.LIB_CHECKED if checked else build_native.LIB
            if not os.path.exists(path):
                build_native.build(checked=checked)
            L = ctypes.CDLL(path)
            sig = {
                "fgl_scene_build": ([P, I64, P, I64, P, P], I32),
                "fgl_scene_destroy": ([P], I32),
                "fgl_scene_get_stats": ([P, P], I32),
                "fgl_scene_export": ([P, P, I64, P, I64], I32),
                "fgl_scene_verify": ([P, P], I32),
                "fgl_scene_upload": ([P], I32),
                "fgl_scene_evict": ([P], I32),
                "fgl_sensor_create": ([P, P, I32, I32, I32, I32, I32, P], I32),
                "fgl_sensor_destroy": ([P], I32),
                "fgl_sensor_n_rays": ([P, P], I32),
                "fgl_sensor_dirs": ([P, P], I32),
                "fgl_cast": ([P, P, P, I32, F32, P, P, P], I32),
                "fgl_cast_opts": ([P, P, P, I32, F32, P, P, P, P], I32),
                "fgl_cast_batched": ([P, I32, P, P], I32),
                "fgl_cast_batched_host": ([P, I32, P, P], I32),
                "fgl_cast_batched_static": ([P, I32, P, P], I32),
                "fgl_autotune": ([P, I32, P, P, P, P], I32),
                "fgl_server_create": ([P, P], I32),
                "fgl_server_add_scene": ([P, P, P], I32),
                "fgl_server_add_sensor": ([P, P, P], I32),
                "fgl_server_submit": ([P, P, P], I32),
                "fgl_server_add_envs": ([P, I32, P, P], I32),
                "fgl_server_read_poses": ([P, I32, I32, P], I32),
                "fgl_server_wait": ([P, I64, I32, P], I32),
                "fgl_server_cancel": ([P, I64], I32),
                "fgl_server_get_stats": ([P, P], I32),
                "fgl_server_reset_stats": ([P], I32),
                "fgl_server_inject_alloc_failures": ([P, I32], I32),
                "fgl_server_inject_worker_faults": ([P, I32], I32),
                "fgl_server_destroy": ([P], I32),
                "fgl_sync": ([P], I32),
                "fgl_work_counters": ([P, P, P], I32),
                "fgl_work_phase_counters": ([P, I32], I32),
                "fgl_world_rays": ([P, P, I32, P, P, P], I32),
                "fgl_probe_l2_read": ([P, I64, I32, P, P], I32),
                "fgl_apply_sensor_effects": ([P, P, P, I32, I32, P], I32),
                "fgl_gaussian_density": ([P, P, F32, P, P, P, P, P], I32),
                "fgl_lbvh_build": ([P, I64, P, I64, P, P], I32),
                "fgl_lbvh_destroy": ([P], I32),
                "fgl_lbvh_get_stats": ([P, P], I32),
                "fgl_lbvh_export": ([P, P, I64, P, I64], I32),
                "fgl_cast_lbvh": ([P, P, P, I32, F32, F32, P, P, P], I32),
                "fgl_denoise": ([P, P, F32, I32, F32, P, P, P, P], I32),
                "fgl_tsdf": ([P, P, F32, P, P, P, P, P], I32),
                "fgl_marching_tets": ([P, P, F32, I32, P, I64, P, I64, P, P, P, P], I32),
                "fgl_last_error": ([], ctypes.c_char_p),
                "fgl_version": ([], I32),
            }
            for name, (args, res) in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(status: int):
    if status != FGL_OK:
        raise FglError(status, lib().fgl_last_error().decode(errors="replace"))


def _np_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _dev_ptr(t, dtype_name: str, numel: int, what: str) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if str(t.dtype) != "torch." + dtype_name:
        raise TypeError(f"{what} must be {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() < numel:
        raise ValueError(f"{what} has {t.numel()} elements, needs {numel}")
    return t.data_ptr()


class Scene:
    """A triangle mesh with its wide BVH (fgl_scene_build)."""

    def __init__(self, verts, tris, width: int = 8, sah_bins: int = 0, n_threads: int = 0,
                 upload: bool = True):
        v = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
        t = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
        o = BuildOpts(width, sah_bins, n_threads, 1 if upload else 0)
        h = P()
        _check(lib().fgl_scene_build(_np_ptr(v), len(v), _np_ptr(t), len(t), ctypes.byref(o),
                                     ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        s = SceneStats()
        _check(lib().fgl_scene_get_stats(self._h, ctypes.byref(s)))
        d = {k: getattr(s, k) for k, _ in SceneStats._fields_}
        for k in ("bounds_lo", "bounds_hi"):
            d[k] = list(d[k])
        return d

    def export(self):
        st = self.stats()
        nodes = np.empty(st["node_bytes"], np.uint8)
        tris = np.empty(st["tri_bytes"] // 4, np.float32)
        _check(lib().fgl_scene_export(self._h, _np_ptr(nodes), nodes.nbytes, _np_ptr(tris),
                                      tris.nbytes))
        return nodes, tris.reshape(-1, 12)

    def verify(self) -> int:
        n = ctypes.c_int64(0)
        _check(lib().fgl_scene_verify(self._h, ctypes.byref(n)))
        return int(n.value)

    def upload(self):
        _check(lib().fgl_scene_upload(self._h))

    def evict(self):
        _check(lib().fgl_scene_evict(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().fgl_scene_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sensor:
    """A scan pattern (fgl_sensor_create) from per-beam elevation/azimuth."""

    def __init__(self, elev, azim, rows: int = 1, cols: Optional[int] = None,
                 tile_rows: int = 0, tile_cols: int = 0):
        el = np.ascontiguousarray(elev, np.float32).reshape(-1)
        az = np.ascontiguousarray(azim, np.float32).reshape(-1)
        if cols is None:
            cols = len(el) // max(rows, 1)
        h = P()
        _check(lib().fgl_sensor_create(_np_ptr(el), _np_ptr(az), len(el), rows, cols, tile_rows,
                                       tile_cols, ctypes.byref(h)))
        self._h = h
        self.n_rays = len(el)
        self.rows, self.cols = rows, cols

    @classmethod
    def from_table(cls, table, tile_rows: int = 0, tile_cols: int = 0):
        return cls(table.elev, table.azim, table.rows, table.cols, tile_rows, tile_cols)

    @property
    def handle(self):
        return self._h

    def dirs(self) -> np.ndarray:
        out = np.empty((self.n_rays, 3), np.float32)
        _check(lib().fgl_sensor_dirs(self._h, _np_ptr(out)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            lib().fgl_sensor_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _outputs(n, device, out_range, out_tri):
    import torch
    if out_range is None:
        out_range = torch.empty(n, dtype=torch.float32, device=device)
    if out_tri is None:
        out_tri = torch.empty(n, dtype=torch.int32, device=device)
    return out_range, out_tri


def cast(scene: Scene, sensor: Sensor, poses, max_range: float, out_range=None, out_tri=None,
         stream=None):
    """Plain form (fgl_cast): one launch, one thread per ray."""
    n_env = poses.shape[0] if poses.dim() == 3 else poses.numel() // 12
    n = n_env * sensor.n_rays
    out_range, out_tri = _outputs(n, poses.device, out_range, out_tri)
    _check(lib().fgl_cast(scene.handle, sensor.handle, _dev_ptr(poses, "float32", n_env * 12, "poses"),
                          n_env, float(max_range), _dev_ptr(out_range, "float32", n, "out_range"),
                          _dev_ptr(out_tri, "int32", n, "out_tri"), _stream_handle(stream)))
    return out_range, out_tri


def cast_opts(scene: Scene, sensor: Sensor, poses, max_range: float, opts: BatchOpts,
              out_range=None, out_tri=None, stream=None):
    """Plain form with explicit launch options (fgl_cast_opts)."""
    n_env = poses.shape[0] if poses.dim() == 3 else poses.numel() // 12
    n = n_env * sensor.n_rays
    out_range, out_tri = _outputs(n, poses.device, out_range, out_tri)
    _check(lib().fgl_cast_opts(scene.handle, sensor.handle,
                               _dev_ptr(poses, "float32", n_env * 12, "poses"), n_env,
                               float(max_range), _dev_ptr(out_range, "float32", n, "out_range"),
                               _dev_ptr(out_tri, "int32", n, "out_tri"), ctypes.byref(opts),
                               _stream_handle(stream)))
    return out_range, out_tri


def make_items(items: Sequence[tuple]):
    """items: (scene, sensor, poses, max_range, out_range, out_tri[, min_range
    [, extras]]) tuples with torch CUDA tensors, extras a dict with any of
    "points" (out [n, 3] float32), "instances" (list of Scene), "instance_poses"
    ([n_env, n_instances, 3, 4] float32) and "out_instance" ([n] int32).
    Returns the ctypes array (it keeps the instance handle arrays alive)."""
    arr = (CastItem * max(1, len(items)))()
    keep = []
    for i, item in enumerate(items):
        sc, se, poses, rmax, orng, otri = item[:6]
        rmin = float(item[6]) if len(item) > 6 and item[6] is not None else 0.0
        ex = item[7] if len(item) > 7 and item[7] else {}
        n_env = poses.shape[0] if poses.dim() == 3 else poses.numel() // 12
        n = n_env * se.n_rays
        c = CastItem(sc.handle, se.handle, _dev_ptr(poses, "float32", n_env * 12, "poses"),
                     n_env, float(rmax), _dev_ptr(orng, "float32", n, "out_range"),
                     _dev_ptr(otri, "int32", n, "out_tri"), rmin)
        if ex.get("points") is not None:
            c.out_points = _dev_ptr(ex["points"], "float32", 3 * n, "points")
        insts = ex.get("instances") or []
        if insts:
            h = (P * len(insts))(*[x.handle for x in insts])
            keep.append(h)
            c.n_instances = len(insts)
            c.instances = ctypes.cast(h, P)
            c.instance_poses = _dev_ptr(ex["instance_poses"], "float32", n_env * len(insts) * 12,
                                        "instance_poses")
        if ex.get("out_instance") is not None:
            c.out_instance = _dev_ptr(ex["out_instance"], "int32", n, "out_instance")
        arr[i] = c
    arr._keep = keep
    return arr


def cast_batched(items: Sequence[tuple], opts: Optional[BatchOpts] = None, stream=None, arr=None):
    """Batched form (fgl_cast_batched) over (scene, sensor, poses, max_range,
    out_range, out_tri) tuples.  Pass a prepared ``arr`` (make_items) to skip
    re-marshalling in a loop."""
    if arr is None:
        arr = make_items(items)
    _check(lib().fgl_cast_batched(arr, len(items), ctypes.byref(opts) if opts else None,
                                  _stream_handle(stream)))


def cast_batched_static(items: Sequence[tuple], opts: Optional[BatchOpts] = None, stream=None,
                        arr=None):
    """fgl_cast_batched_static: the batched form without any allocation (work
    queue in a fixed library array, at most 256 items; calls that overlap on
    the GPU race)."""
    if arr is None:
        arr = make_items(items)
    _check(lib().fgl_cast_batched_static(arr, len(items), ctypes.byref(opts) if opts else None,
                                         _stream_handle(stream)))


class TuneOpts(ctypes.Structure):
    _fields_ = [("reps", I32), ("passes", I32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("best_ms", F64), ("start_ms", F64), ("trials", I32)]


def autotune(items: Sequence[tuple], start: Optional[BatchOpts] = None, reps: int = 3,
             passes: int = 2, stream=None):
    """fgl_autotune: fastest launch options for these items.  Returns
    (BatchOpts, {"best_ms", "start_ms", "trials"})."""
    arr = make_items(items)
    best = BatchOpts() if start is None else BatchOpts(*[getattr(start, k) for k, _ in BatchOpts._fields_])
    res = TuneResult()
    _check(lib().fgl_autotune(arr, len(items), ctypes.byref(TuneOpts(reps, passes)), ctypes.byref(best),
                              ctypes.byref(res), _stream_handle(stream)))
    return best, {"best_ms": res.best_ms, "start_ms": res.start_ms, "trials": res.trials}


def cast_batched_host(items: Sequence[tuple], opts: Optional[BatchOpts] = None, stream=None):
    """End-to-end batched form (fgl_cast_batched_host): poses and outputs are
    host tensors/arrays (page-locked for full speed), item tuples as for
    cast_batched (extras included, all on the host); blocks until done."""
    arr = (CastItem * max(1, len(items)))()
    keep = []
    for i, item in enumerate(items):
        sc, se, poses, rmax, orng, otri = item[:6]
        rmin = float(item[6]) if len(item) > 6 and item[6] is not None else 0.0
        ex = item[7] if len(item) > 7 and item[7] else {}
        n_env = int(np.prod(poses.shape)) // 12
        c = CastItem(sc.handle, se.handle, _host_ptr(poses), n_env, float(rmax),
                     _host_ptr(orng), _host_ptr(otri), rmin)
        if ex.get("points") is not None:
            c.out_points = _host_ptr(ex["points"])
        insts = ex.get("instances") or []
        if insts:
            h = (P * len(insts))(*[x.handle for x in insts])
            keep.append(h)
            c.n_instances = len(insts)
            c.instances = ctypes.cast(h, P)
            c.instance_poses = _host_ptr(ex["instance_poses"])
        if ex.get("out_instance") is not None:
            c.out_instance = _host_ptr(ex["out_instance"])
        arr[i] = c
    _check(lib().fgl_cast_batched_host(arr, len(items), ctypes.byref(opts) if opts else None,
                                       _stream_handle(stream)))


def _host_ptr(x) -> int:
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be contiguous")
        return x.ctypes.data
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or not x.is_contiguous():
            raise ValueError("host tensors must be contiguous CPU tensors")
        return x.data_ptr()
    raise TypeError("expected a numpy array or a CPU tensor")


def world_rays(sensor: Sensor, poses, stream=None):
    """Float32 world rays exactly as the kernels trace them: (o, d) [n, 3]."""
    import torch
    n_env = poses.shape[0] if poses.dim() == 3 else poses.numel() // 12
    n = n_env * sensor.n_rays
    o = torch.empty((n, 3), dtype=torch.float32, device=poses.device)
    d = torch.empty((n, 3), dtype=torch.float32, device=poses.device)
    _check(lib().fgl_world_rays(sensor.handle, _dev_ptr(poses, "float32", n_env * 12, "poses"),
                                n_env, o.data_ptr(), d.data_ptr(), _stream_handle(stream)))
    return o, d


def sync(stream=None):
    """Wait for the stream and surface asynchronous / device-side errors."""
    _check(lib().fgl_sync(_stream_handle(stream)))


class LbvhStats(ctypes.Structure):
    _fields_ = [("n_tris", I64), ("n_nodes", I64), ("depth", I32), ("overflow", I32),
                ("build_ms", F32), ("margin", F32), ("centroid_lo", F32 * 3), ("centroid_hi", F32 * 3)]


class Lbvh:
    """A triangle LBVH built on the GPU from CUDA tensors (fgl_lbvh_build):
    verts float32 [nv, 3], tris int32 [nt, 3].  rebuild() refits it to moved
    vertices (a full rebuild into the same buffers)."""

    def __init__(self, verts, tris, stream=None):
        self._h = P()
        self._nt = 0
        self.rebuild(verts, tris, stream)

    def rebuild(self, verts, tris, stream=None):
        nv = verts.numel() // 3
        nt = tris.numel() // 3
        _check(lib().fgl_lbvh_build(_dev_ptr(verts, "float32", 3 * nv, "verts"), nv,
                                    _dev_ptr(tris, "int32", 3 * nt, "tris"), nt,
                                    _stream_handle(stream), ctypes.byref(self._h)))
        self._nt = nt

    @property
    def handle(self):
        return self._h

    def stats(self) -> dict:
        st = LbvhStats()
        _check(lib().fgl_lbvh_get_stats(self._h, ctypes.byref(st)))
        return {"n_tris": st.n_tris, "n_nodes": st.n_nodes, "depth": st.depth, "overflow": st.overflow,
                "build_ms": st.build_ms, "margin": st.margin,
                "centroid_lo": list(st.centroid_lo), "centroid_hi": list(st.centroid_hi)}

    def export(self):
        """(nodes uint8 [n_nodes*64], tris float32 [nt, 12]) host copies."""
        n_nodes = max(0, self._nt - 1)
        nodes = np.empty(n_nodes * 64, np.uint8)
        tris = np.empty((self._nt, 12), np.float32)
        _check(lib().fgl_lbvh_export(self._h, _np_ptr(nodes), nodes.nbytes, _np_ptr(tris), tris.nbytes))
        return nodes, tris

    def cast(self, sensor: "Sensor", poses, max_range: float, min_range: float = 0.0,
             out_range=None, out_tri=None, stream=None):
        """eq. t_j* over the LBVH, one thread per beam (fgl_cast_lbvh)."""
        n_env = poses.shape[0] if poses.dim() == 3 else poses.numel() // 12
        n = n_env * sensor.n_rays
        out_range, out_tri = _outputs(n, poses.device, out_range, out_tri)
        _check(lib().fgl_cast_lbvh(self._h, sensor.handle, _dev_ptr(poses, "float32", n_env * 12, "poses"),
                                   n_env, float(min_range), float(max_range),
                                   _dev_ptr(out_range, "float32", n, "out_range"),
                                   _dev_ptr(out_tri, "int32", n, "out_tri"), _stream_handle(stream)))
        return out_range, out_tri

    def close(self):
        if getattr(self, "_h", None):
            lib().fgl_lbvh_destroy(self._h)
            self._h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Gaussians(ctypes.Structure):
    _fields_ = [("mu", P), ("scale", P), ("quat", P), ("opacity", P), ("n", I64)]


class Grid(ctypes.Structure):
    _fields_ = [("origin", F32 * 3), ("h", F32), ("dims", I32 * 3), ("tile", I32)]


class DensityStats(ctypes.Structure):
    _fields_ = [("timing", I32), ("n_pairs", I64), ("n_tiles", I64), ("n_voxels", I64),
                ("ms_total", F32), ("ms_density", F32), ("n_launches", I32)]


def gaussian_density(mu, scale, quat, opacity, origin, h: float, dims, theta: float = 0.5,
                     tile: int = 0, out_density=None, out_occ=None, out_surf=None, stream=None,
                     masks: bool = True, timing: bool = False):
    """Gaussian-to-occupancy conversion (fgl_gaussian_density, paper Sec.
    IV-A) on torch CUDA tensors: mu/scale [n,3], quat [n,4] (w,x,y,z),
    opacity [n].  Returns (density [nz,ny,nx] f32, occ u8, surf u8, stats);
    occ and surf are None when masks=False."""
    import torch
    n = int(mu.shape[0]) if mu.dim() > 1 else mu.numel() // 3
    nx, ny, nz = (int(d) for d in dims)
    nv = nx * ny * nz
    dev = mu.device
    if out_density is None:
        out_density = torch.empty((nz, ny, nx), dtype=torch.float32, device=dev)
    if masks and out_occ is None:
        out_occ = torch.empty((nz, ny, nx), dtype=torch.uint8, device=dev)
    if masks and out_surf is None:
        out_surf = torch.empty((nz, ny, nx), dtype=torch.uint8, device=dev)
    gs = Gaussians(_dev_ptr(mu, "float32", 3 * n, "mu") if n else None,
                   _dev_ptr(scale, "float32", 3 * n, "scale") if n else None,
                   _dev_ptr(quat, "float32", 4 * n, "quat") if n else None,
                   _dev_ptr(opacity, "float32", n, "opacity") if n else None, n)
    g = Grid((F32 * 3)(*[float(x) for x in origin]), float(h), (I32 * 3)(nx, ny, nz), int(tile))
    st = DensityStats()
    st.timing = 1 if timing else 0
    _check(lib().fgl_gaussian_density(ctypes.byref(gs), ctypes.byref(g), float(theta),
                                      _dev_ptr(out_density, "float32", nv, "out_density"),
                                      _dev_ptr(out_occ, "uint8", nv, "out_occ") if masks else None,
                                      _dev_ptr(out_surf, "uint8", nv, "out_surf") if masks else None,
                                      ctypes.byref(st), _stream_handle(stream)))
    return out_density, out_occ, out_surf, {"n_pairs": st.n_pairs, "n_tiles": st.n_tiles,
                                            "n_voxels": st.n_voxels, "ms_total": st.ms_total,
                                            "ms_density": st.ms_density,
                                            "n_launches": st.n_launches}


# ---------------------------------------------------------------------------
# mesh reconstruction (fgl_denoise, fgl_tsdf, fgl_marching_tets; Sec. IV-B)
# ---------------------------------------------------------------------------
class TsdfStats(ctypes.Structure):
    _fields_ = [("timing", I32), ("n_layers", I32), ("n_launches", I32), ("ms_total", F32),
                ("delta_mode", I32)]


def _grid_of(shape, origin, h):
    nz, ny, nx = (int(d) for d in shape)
    return Grid((F32 * 3)(*[float(x) for x in origin]), float(h), (I32 * 3)(nx, ny, nz), 0), nx * ny * nz


def denoise(surf, h: float, sigma: float, tau: float = 0.5, quantile=None, blur: bool = False,
            stream=None):
    """Eqs. V' and rethresh (fgl_denoise) on a u8 CUDA grid [nz, ny, nx]:
    blur by a Gaussian of sigma metres, keep V' >= tau (or V' >= the
    quantile-q order statistic when quantile is given).  Returns (mask u8,
    V' f32 or None, threshold used)."""
    import torch
    g, n = _grid_of(surf.shape, (0.0, 0.0, 0.0), h)
    mask = torch.empty(surf.shape, dtype=torch.uint8, device=surf.device)
    vp = torch.empty(surf.shape, dtype=torch.float32, device=surf.device) if blur else None
    thr = F32()
    mode, value = (1, float(quantile)) if quantile is not None else (0, float(tau))
    _check(lib().fgl_denoise(_dev_ptr(surf, "uint8", n, "surf"), ctypes.byref(g), float(sigma), mode,
                             value, _dev_ptr(vp, "float32", n, "blur") if blur else None,
                             _dev_ptr(mask, "uint8", n, "mask"), ctypes.byref(thr),
                             _stream_handle(stream)))
    return mask, vp, float(thr.value)


def tsdf(surf, h: float, trunc: float, outside: bool = False, shell: bool = False,
         timing: bool = False, stream=None, delta: str = "half"):
    """Narrow-band TSDF (fgl_tsdf) of a u8 surface grid [nz, ny, nx], eq.
    delta as (p + 1/2) h (delta="half") or literally p h (delta="literal"):
    returns (phi f32, outside u8 or None, shell index u8 or None, stats)."""
    if delta not in ("half", "literal"):
        raise ValueError("delta must be 'half' or 'literal'")
    import torch
    g, n = _grid_of(surf.shape, (0.0, 0.0, 0.0), h)
    dev = surf.device
    phi = torch.empty(surf.shape, dtype=torch.float32, device=dev)
    out = torch.empty(surf.shape, dtype=torch.uint8, device=dev) if outside else None
    sh = torch.empty(surf.shape, dtype=torch.uint8, device=dev) if shell else None
    st = TsdfStats()
    st.timing = 1 if timing else 0
    st.delta_mode = 1 if delta == "literal" else 0
    _check(lib().fgl_tsdf(_dev_ptr(surf, "uint8", n, "surf"), ctypes.byref(g), float(trunc),
                          _dev_ptr(phi, "float32", n, "phi"),
                          _dev_ptr(out, "uint8", n, "outside") if outside else None,
                          _dev_ptr(sh, "uint8", n, "shell") if shell else None, ctypes.byref(st),
                          _stream_handle(stream)))
    return phi, out, sh, {"n_layers": st.n_layers, "n_launches": st.n_launches,
                          "ms_total": st.ms_total}


def marching_tets(phi, origin, h: float, iso: float = 0.0, step: int = 1, normals: bool = False,
                  capacity=None, stream=None):
    """The phi = iso level set (fgl_marching_tets) of a float CUDA grid
    [nz, ny, nx] whose voxel (i, j, k) has centre origin + (idx + 1/2) h.
    Returns (verts f32 [nv, 3], tris i32 [nt, 3], normals f32 [nv, 3] or
    None).  capacity=(verts, tris) sizes the outputs up front; without it the
    call counts first (a second pass over the grid)."""
    import torch
    g, n = _grid_of(phi.shape, origin, h)
    dev = phi.device
    nv, nt = I64(), I64()
    L = lib()
    pphi = _dev_ptr(phi, "float32", n, "phi")
    hs = _stream_handle(stream)
    if capacity is None:
        _check(L.fgl_marching_tets(pphi, ctypes.byref(g), float(iso), int(step), None, 0, None, 0, None,
                                   ctypes.byref(nv), ctypes.byref(nt), hs))
        capacity = (nv.value, nt.value)
    for _ in range(2):
        vc, tc = max(int(capacity[0]), 1), max(int(capacity[1]), 1)
        verts = torch.empty((vc, 3), dtype=torch.float32, device=dev)
        tris = torch.empty((tc, 3), dtype=torch.int32, device=dev)
        nrm = torch.empty((vc, 3), dtype=torch.float32, device=dev) if normals else None
        st = L.fgl_marching_tets(pphi, ctypes.byref(g), float(iso), int(step),
                                 _dev_ptr(verts, "float32", 3 * vc, "verts"), vc,
                                 _dev_ptr(tris, "int32", 3 * tc, "tris"), tc,
                                 _dev_ptr(nrm, "float32", 3 * vc, "normals") if normals else None,
                                 ctypes.byref(nv), ctypes.byref(nt), hs)
        if st == FGL_ERR_CAPACITY:
            capacity = (nv.value, nt.value)
            continue
        _check(st)
        return (verts[:nv.value], tris[:nt.value], nrm[:nv.value] if normals else None)
    raise FglError(FGL_ERR_CAPACITY, "marching_tets: capacity retry failed")


def mesh_from_surface(surf, origin, h: float, trunc: float = 0.06, sigma=None, tau: float = 0.5,
                      quantile=None, iso: float = 0.0, step: int = 1, normals: bool = False,
                      capacity=None, stream=None):
    """Sec. IV-B from a surface grid: optional denoising (sigma metres; the
    paper leaves sigma and tau open), the narrow-band TSDF of half-width
    trunc, and its iso level set.  Returns (verts, tris, normals, phi)."""
    if sigma:
        surf, _, _ = denoise(surf, h, sigma, tau=tau, quantile=quantile, stream=stream)
    phi, _, _, _ = tsdf(surf, h, trunc, stream=stream)
    v, t, nrm = marching_tets(phi, origin, h, iso=iso, step=step, normals=normals, capacity=capacity,
                              stream=stream)
    return v, t, nrm, phi


def mesh_from_gaussians(mu, scale, quat, opacity, origin, h: float, dims, theta: float = 0.5,
                        trunc: float = 0.06, sigma="half-voxel", tau: float = 0.5, iso: float = 0.0,
                        step: int = 1, normals: bool = False, capacity=None, stream=None):
    """3D Gaussians to a watertight mesh on the GPU (Sec. IV-A then IV-B):
    density and surface shell (gaussian_density), denoising (default sigma =
    h / 2 with tau = 1/2: a lone voxel blurs below 1/2 while a one-voxel
    plane stays at 0.79; sigma=None skips it), TSDF and marching tetrahedra.
    Returns (verts, tris, normals)."""
    _, _, surf, _ = gaussian_density(mu, scale, quat, opacity, origin, h, dims, theta=theta,
                                     stream=stream)
    if isinstance(sigma, str):
        sigma = 0.5 * h
    v, t, nrm, _ = mesh_from_surface(surf, origin, h, trunc=trunc, sigma=sigma, tau=tau, iso=iso,
                                     step=step, normals=normals, capacity=capacity, stream=stream)
    return v, t, nrm


def work_counters():
    """(rays, node visits, triangle tests) counted by count_work launches."""
    r, n, t = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().fgl_work_counters(ctypes.byref(r), ctypes.byref(n), ctypes.byref(t)))
    return int(r.value), int(n.value), int(t.value)


class SensorEffects(ctypes.Structure):
    _fields_ = [("seed", U64), ("step", ctypes.c_uint32), ("env_offset", I32), ("drop_prob", F32),
                ("noise_sigma0", F32), ("noise_sigma1", F32), ("max_range", F32)]


def apply_sensor_effects(range_, tri, n_env: int, seed: int, step: int = 0, env_offset: int = 0,
                         drop_prob: float = 0.0, sigma0: float = 0.0, sigma1: float = 0.0,
                         max_range: float = 100.0, stream=None):
    """fgl_apply_sensor_effects in place on one cast item's CUDA outputs
    (range float32, tri int32, n_env * n_rays each)."""
    n = range_.numel()
    if n_env < 1 or n % n_env:
        raise ValueError("range must hold n_env * n_rays values")
    fx = SensorEffects(int(seed), int(step), int(env_offset), float(drop_prob), float(sigma0),
                       float(sigma1), float(max_range))
    _check(lib().fgl_apply_sensor_effects(ctypes.byref(fx), _dev_ptr(range_, "float32", n, "range"),
                                          _dev_ptr(tri, "int32", n, "tri"), int(n_env), n // n_env,
                                          _stream_handle(stream)))


def probe_l2_read(buf, reps: int, sink, stream=None):
    """fgl_probe_l2_read over a CUDA tensor `buf` (its whole storage), `reps`
    passes; `sink` a one-element int32 CUDA tensor."""
    nbytes = buf.numel() * buf.element_size()
    _check(lib().fgl_probe_l2_read(buf.data_ptr(), nbytes - nbytes % 16, int(reps), sink.data_ptr(),
                                   _stream_handle(stream)))


PHASE_COUNTERS = ("rays", "node_visits", "tri_tests", "warp_iterations", "active_lane_iterations",
                  "tri_rounds", "finish_pops", "packets")


def work_phase_counters() -> dict:
    """Every count_work counter (fgl_work_phase_counters), then reset."""
    out = (ctypes.c_uint64 * len(PHASE_COUNTERS))()
    _check(lib().fgl_work_phase_counters(out, len(PHASE_COUNTERS)))
    return {k: int(v) for k, v in zip(PHASE_COUNTERS, out)}


# ---------------------------------------------------------------------------
# serving (fgl_server_*)
# ---------------------------------------------------------------------------
class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", I64), ("tick_rays", I64), ("max_active", I32),
                ("mode", I32), ("opts", BatchOpts), ("env_capacity", I32)]


# fgl_pose_source
POSES_REQUEST, POSES_SLOTS, POSES_SLOTS_SET_HOST, POSES_SLOTS_SET_DEVICE = 0, 1, 2, 3


class Request(ctypes.Structure):
    _fields_ = [("scene_id", I32), ("sensor_id", I32), ("n_env", I32), ("max_range", F32),
                ("poses", P), ("out_range", P), ("out_tri", P), ("min_range", F32),
                ("pose_source", I32), ("env_first", I32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", I32), ("queue_ms", F64), ("latency_ms", F64), ("rays", I64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", I64), ("completed", I64), ("rejected", I64), ("cancelled", I64),
                ("evictions", I64), ("uploads", I64), ("ticks", I64), ("rays", I64),
                ("p50_ms", F64), ("p99_ms", F64), ("mean_ms", F64), ("busy_s", F64),
                ("rays_per_s", F64), ("device_bytes", I64), ("pending", I64), ("active", I64)]


class Server:
    """Continuous-batching scan server (fgl_server_*).  Scenes and sensors
    registered with it must stay alive until close()."""

    def __init__(self, hbm_budget_bytes: int = 0, tick_rays: int = 0, max_active: int = 0,
                 mode: int = 0, opts: Optional[BatchOpts] = None, env_capacity: int = 0):
        o = ServerOpts(hbm_budget_bytes, tick_rays, max_active, mode, opts or BatchOpts(),
                       env_capacity)
        h = P()
        _check(lib().fgl_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._keep = []

    def add_scene(self, scene: Scene) -> int:
        i = I32()
        _check(lib().fgl_server_add_scene(self._h, scene.handle, ctypes.byref(i)))
        self._keep.append(scene)
        return i.value

    def add_sensor(self, sensor: Sensor) -> int:
        i = I32()
        _check(lib().fgl_server_add_sensor(self._h, sensor.handle, ctypes.byref(i)))
        self._keep.append(sensor)
        return i.value

    def add_envs(self, poses) -> int:
        """Register environment slots holding `poses` (host float32
        [n_env, 3, 4]); returns the first slot id (fgl_server_add_envs)."""
        P_ = np.ascontiguousarray(poses, np.float32)
        first = I32()
        _check(lib().fgl_server_add_envs(self._h, P_.size // 12, P_.ctypes.data_as(P),
                                         ctypes.byref(first)))
        return first.value

    def read_poses(self, env_first: int, n_env: int) -> np.ndarray:
        """The slots' current poses as the admitted requests left them."""
        out = np.empty((n_env, 3, 4), np.float32)
        _check(lib().fgl_server_read_poses(self._h, env_first, n_env, out.ctypes.data_as(P)))
        return out

    def submit(self, scene_id: int, sensor_id: int, poses, max_range: float, out_range, out_tri,
               min_range: float = 0.0, env_first: Optional[int] = None, n_env: Optional[int] = None) -> int:
        """Without env_first: poses are host float32 [n_env,3,4] carried by the
        request.  With env_first: the request scans resident slots
        [env_first, env_first + n_env); poses None scans them as they are, a
        host array or a CUDA tensor overwrites them first.  Outputs: host
        arrays/tensors."""
        if env_first is None:
            src, first = POSES_REQUEST, 0
            n_env = int(np.prod(poses.shape)) // 12
            ptr = _host_ptr(poses)
        else:
            first = int(env_first)
            if poses is None:
                src, ptr = POSES_SLOTS, None
                assert n_env is not None, "n_env is needed when no poses are given"
            else:
                n_env = int(np.prod(poses.shape)) // 12
                dev = getattr(poses, "is_cuda", False)
                src = POSES_SLOTS_SET_DEVICE if dev else POSES_SLOTS_SET_HOST
                ptr = _dev_ptr(poses, "float32", n_env * 12, "poses") if dev else _host_ptr(poses)
        r = Request(scene_id, sensor_id, int(n_env), float(max_range), ptr,
                    _host_ptr(out_range), _host_ptr(out_tri), float(min_range), src, first)
        t = I64()
        _check(lib().fgl_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)))
        return t.value

    def wait(self, ticket: int, timeout_ms: int = -1, check: bool = True) -> dict:
        info = RequestInfo()
        st = lib().fgl_server_wait(self._h, ticket, timeout_ms, ctypes.byref(info))
        if check:
            _check(st)
        return {"status": st, "queue_ms": info.queue_ms, "latency_ms": info.latency_ms,
                "rays": info.rays}

    def cancel(self, ticket: int):
        _check(lib().fgl_server_cancel(self._h, ticket))

    def inject_alloc_failures(self, n: int):
        _check(lib().fgl_server_inject_alloc_failures(self._h, n))

    def inject_worker_faults(self, n: int):
        """The next n ticks with work throw a host exception in the worker
        (fgl_server_inject_worker_faults)."""
        _check(lib().fgl_server_inject_worker_faults(self._h, n))

    def stats(self) -> dict:
        s = ServerStats()
        _check(lib().fgl_server_get_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def reset_stats(self):
        _check(lib().fgl_server_reset_stats(self._h))

    def close(self):
        if getattr(self, "_h", None):
            lib().fgl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
