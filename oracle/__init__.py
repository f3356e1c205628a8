"""FP64 CPU oracle for first-hit LiDAR ray casting (paper Sec. IV-C), for
the Gaussian-to-occupancy conversion (Sec. IV-A) and for the mesh
reconstruction steps (Sec. IV-B: denoising, narrow-band TSDF, isosurface).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the library it checks.  It
shares no code with ``paper_2509_17390_gb300``.

The C++ sources (``oracle.cpp``, ``density.cpp``, ``tsdf.cpp``) are compiled on first use
(or by ``build()``) with ``-ffp-contract=off`` into ``oracle/_build/liboracle.so``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_SRC_DENSITY = os.path.join(_HERE, "density.cpp")
_SRC_TSDF = os.path.join(_HERE, "tsdf.cpp")
_SRC_EFFECTS = os.path.join(_HERE, "effects.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

FLAG_EDGE, FLAG_TIE, FLAG_RANGE = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(f) for f in (_SRC, _SRC_DENSITY, _SRC_TSDF, _SRC_EFFECTS))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-pthread", _SRC, _SRC_DENSITY, _SRC_TSDF, _SRC_EFFECTS, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.orc_version.restype = I32
            L.orc_sensor_dirs.argtypes = [P, P, I64, P]
            L.orc_world_rays.argtypes = [P, I64, P, I64, P, P]
            L.orc_scene_create.argtypes = [P, I64, P, I64, I32]
            L.orc_scene_create.restype = P
            L.orc_scene_free.argtypes = [P]
            L.orc_scene_depth.argtypes = [P]
            L.orc_scene_depth.restype = I32
            L.orc_cast.argtypes = [P, P, P, I64, D, D, I32, P, P, P]
            L.orc_validate.argtypes = [P, P, P, I64, D, D, P, P, I32, P]
            L.orc_tri_test.argtypes = [P, P, P, P, P, P]
            L.orc_edge_measure.argtypes = [P, P, P, I64, P, D, I32, P]
            L.orc_tri_test.restype = I32
            L.orc_instance_rays.argtypes = [P, P, P, I64, P, P]
            L.orc_gauss_tile_ranges.argtypes = [P, P, P, I64, P, ctypes.c_float, I32, P]
            L.orc_density.argtypes = [P, P, P, P, I64, P, ctypes.c_float, P, I32, I32, P, P]
            L.orc_occupancy.argtypes = [P, P, D, P, P]
            L.orc_density_tiles.argtypes = [P, P, P, P, I64, P, ctypes.c_float, P, I32, P, I64, I32, P, P]
            F = ctypes.c_float
            L.orc_blur.argtypes = [P, I64, I64, I64, D, I32, P]
            L.orc_outside.argtypes = [P, I64, I64, I64, P]
            L.orc_shell.argtypes = [P, I64, I64, I64, I32, P]
            L.orc_tsdf.argtypes = [P, P, I64, F, F, I32, P]
            L.orc_marching_tets.argtypes = [P, I64, I64, I64, P, F, F, I32, I32, P, P, P, P, P]
            L.orc_tsdf_free.argtypes = [P]
            U64 = ctypes.c_uint64
            L.orc_philox4x32.argtypes = [P, P, I32, P]
            L.orc_sensor_effects.argtypes = [U64, ctypes.c_uint32, ctypes.c_int32, D, D, D, D, I64, I64,
                                             P, P, P]
            _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def sensor_dirs(elev: np.ndarray, azim: np.ndarray) -> np.ndarray:
    """float32 [n,3] sensor-frame unit directions from (elev, azim)."""
    el = np.ascontiguousarray(elev, np.float32)
    az = np.ascontiguousarray(azim, np.float32)
    out = np.empty((len(el), 3), np.float32)
    lib().orc_sensor_dirs(_ptr(el), _ptr(az), len(el), _ptr(out))
    return out


def world_rays(dirs: np.ndarray, poses: np.ndarray):
    """float32 world rays (o, d), each [n_env * n_rays, 3], ray e*n_rays+j."""
    dirs = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    poses = np.ascontiguousarray(poses, np.float32).reshape(-1, 12)
    n = len(dirs) * len(poses)
    o = np.empty((n, 3), np.float32)
    d = np.empty((n, 3), np.float32)
    lib().orc_world_rays(_ptr(dirs), len(dirs), _ptr(poses), len(poses), _ptr(o), _ptr(d))
    return o, d


def tri_test(o, d, v0, v1, v2):
    """FP64 signed-volume test of one ray against one triangle: t or None."""
    args = [np.ascontiguousarray(x, np.float64) for x in (o, d, v0, v1, v2)]
    t = np.zeros(1, np.float64)
    hit = lib().orc_tri_test(*[_ptr(a) for a in args], _ptr(t))
    return float(t[0]) if hit else None


def instance_rays(o: np.ndarray, d: np.ndarray, poses: np.ndarray):
    """Rays moved into instance frames (float32, the fixed sequence of the C
    source): poses is world-from-local [R | t] per ray, [n, 3, 4] or [n, 12]."""
    o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
    P = np.ascontiguousarray(poses, np.float32).reshape(-1, 12)
    oo = np.empty_like(o)
    dd = np.empty_like(d)
    lib().orc_instance_rays(_ptr(o), _ptr(d), _ptr(P), len(o), _ptr(oo), _ptr(dd))
    return oo, dd


def cast_with_instances(static: "Scene", instances, o, d, inst_poses, n_rays, max_range,
                        min_range: float = 0.0):
    """Eq. t_j* over a scene plus per-environment rigid instances.

    inst_poses: [n_env, n_inst, 3, 4] world-from-local; rays env-major
    (n_env * n_rays).  Each instance is cast in its own frame (instance_rays);
    the return is the nearest, ties going to the scene, then to the lower
    instance.  Returns (range f64, tri id, instance (-1 = scene), flags): the
    flags of every part are combined (an ambiguity in any part may decide the
    nearest), and a ray is also TIE-flagged when two parts return within tol
    of each other."""
    r, i, fl = static.cast(o, d, max_range, min_range=min_range)
    inst = np.full(len(r), -1, np.int32)
    r = r.copy()
    i = i.copy()
    fl = fl.copy()
    P = np.asarray(inst_poses, np.float32)
    for k, sc in enumerate(instances):
        pk = np.repeat(P[:, k].reshape(-1, 12), n_rays, axis=0)
        lo, ld = instance_rays(o, d, pk)
        rk, ik, fk = sc.cast(lo, ld, max_range, min_range=min_range)
        hit_k = ik >= 0
        close = hit_k & (i >= 0) & (np.abs(rk - r) <= 1e-4 + 1e-6 * np.abs(r))
        take = hit_k & ((i < 0) | (rk < r))
        fl = fl | fk | np.where(close, FLAG_TIE, 0).astype(np.uint8)
        r = np.where(take, rk, r)
        i = np.where(take, ik, i)
        inst = np.where(take, k, inst).astype(np.int32)
    return r, i, inst, fl


def philox4x32(ctr, key, rounds: int = 10) -> np.ndarray:
    """Philox-4x32 (Salmon et al. 2011) of one counter (4 uint32) under one
    key (2 uint32): 4 uint32 words."""
    c = np.ascontiguousarray(ctr, np.uint32).reshape(4)
    k = np.ascontiguousarray(key, np.uint32).reshape(2)
    out = np.empty(4, np.uint32)
    lib().orc_philox4x32(_ptr(c), _ptr(k), int(rounds), _ptr(out))
    return out


def sensor_effects(range_, tri, n_env: int, seed: int, step: int = 0, env_offset: int = 0,
                   drop_prob: float = 0.0, sigma0: float = 0.0, sigma1: float = 0.0,
                   max_range: float = 100.0):
    """Seeded return dropout and range noise on cast returns [n_env * n_rays]
    (see effects.cpp): returns (range f32, tri i32, dropped u8) copies.  The
    parameters are float32 values (as a caller of the library passes them):
    they are rounded to float32 first."""
    f32 = lambda x: float(np.float32(x))
    drop_prob, sigma0, sigma1, max_range = f32(drop_prob), f32(sigma0), f32(sigma1), f32(max_range)
    r = np.array(range_, np.float32, copy=True).reshape(-1)
    t = np.array(tri, np.int32, copy=True).reshape(-1)
    if len(r) != len(t) or len(r) % max(1, n_env):
        raise ValueError("range and tri must hold n_env * n_rays values")
    dropped = np.empty(len(r), np.uint8)
    lib().orc_sensor_effects(int(seed), int(step), int(env_offset), float(drop_prob), float(sigma0),
                             float(sigma1), float(max_range), int(n_env), len(r) // max(1, n_env),
                             _ptr(r), _ptr(t), _ptr(dropped))
    return r, t, dropped


class Scene:
    """Oracle scene: brute force over all triangles (bvh=False) or a
    median-split FP64 BVH (bvh=True); both give identical answers."""

    def __init__(self, verts: np.ndarray, tris: np.ndarray, bvh: bool = True):
        self.verts = np.ascontiguousarray(verts, np.float32).reshape(-1, 3)
        self.tris = np.ascontiguousarray(tris, np.int32).reshape(-1, 3)
        self._h = lib().orc_scene_create(_ptr(self.verts), len(self.verts), _ptr(self.tris),
                                         len(self.tris), 1 if bvh else 0)
        if not self._h:
            raise ValueError("invalid scene (vertex id out of range or non-finite vertex)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_scene_free(h)
            self._h = None

    @property
    def depth(self) -> int:
        return lib().orc_scene_depth(self._h)

    def cast(self, o: np.ndarray, d: np.ndarray, max_range: float, flags: bool = True,
             nthreads: int = 0, min_range: float = 0.0):
        """Nearest hit (eq. t_j*) among intersections with t > 0 and
        min_range <= t <= max_range: (range f64, id i32, flags u8 or None)."""
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        n = len(o)
        t = np.empty(n, np.float64)
        ids = np.empty(n, np.int32)
        fl = np.empty(n, np.uint8) if flags else None
        lib().orc_cast(self._h, _ptr(o), _ptr(d), n, float(min_range), float(max_range), int(nthreads), _ptr(t),
                       _ptr(ids), _ptr(fl) if flags else None)
        return t, ids, fl

    def edge_measure(self, o, d, t_star, cap: float = 1e-5, nthreads: int = 0) -> np.ndarray:
        """Per ray: the smallest (ray-line to triangle-edge distance) / L_k over
        the EDGE flag's window [-1e-4, t* + tol(t*)], capped at `cap`; the EDGE
        flag is set exactly where this is below 1e-6."""
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        t = np.ascontiguousarray(t_star, np.float64)
        out = np.empty(len(o), np.float64)
        lib().orc_edge_measure(self._h, _ptr(o), _ptr(d), len(o), _ptr(t), float(cap), int(nthreads), _ptr(out))
        return out

    def validate(self, o, d, max_range, rng, ids, nthreads: int = 0, min_range: float = 0.0) -> np.ndarray:
        """Per ray: is (range, id) an acceptable FP32 answer?  (bool array)"""
        o = np.ascontiguousarray(o, np.float32).reshape(-1, 3)
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        r = np.ascontiguousarray(rng, np.float32)
        i = np.ascontiguousarray(ids, np.int32)
        ok = np.empty(len(o), np.uint8)
        lib().orc_validate(self._h, _ptr(o), _ptr(d), len(o), float(min_range), float(max_range), _ptr(r), _ptr(i),
                           int(nthreads), _ptr(ok))
        return ok.astype(bool)


def compare(range_gpu, id_gpu, range_orc, id_orc, flags, max_range):
    """Element-wise parity under the tolerance contract.

    Unflagged rays: hit/miss and triangle id equal, and
    |range_gpu - range_orc| <= 1e-4 + 1e-6 * range_orc (a miss must report
    max_range exactly).  TIE-flagged rays: range checked, id exempt.
    EDGE/RANGE-flagged rays: exempt here (check them with Scene.validate).
    Returns (bad_mask, checked_mask).
    """
    rg = np.asarray(range_gpu, np.float64)
    ig = np.asarray(id_gpu)
    ro = np.asarray(range_orc, np.float64)
    io = np.asarray(id_orc)
    fl = np.asarray(flags)
    hard = (fl & (FLAG_EDGE | FLAG_RANGE)) != 0
    tie = (fl & FLAG_TIE) != 0
    checked = ~hard
    tolr = 1e-4 + 1e-6 * np.abs(ro)
    bad = np.zeros(len(rg), bool)
    hit_o = io >= 0
    hit_g = ig >= 0
    bad |= checked & (hit_o != hit_g)
    bad |= checked & ~tie & (io != ig)
    bad |= checked & hit_o & hit_g & (np.abs(rg - ro) > tolr)
    bad |= checked & ~hit_o & ~hit_g & (rg != np.float32(max_range))
    return bad, checked


# ---------------------------------------------------------------------------
# Gaussian-to-occupancy (paper Sec. IV-A)
# ---------------------------------------------------------------------------
def _f32(a, cols):
    return np.ascontiguousarray(a, np.float32).reshape(-1, cols) if cols else np.ascontiguousarray(a, np.float32).reshape(-1)


def gauss_tile_ranges(mu, scale, quat, origin, h, B):
    """Candidate tile ranges [n, 6] (lo xyz, hi xyz; inclusive, unclamped)."""
    mu, scale, quat = _f32(mu, 3), _f32(scale, 3), _f32(quat, 4)
    o = np.ascontiguousarray(origin, np.float32)
    out = np.empty((len(mu), 6), np.int32)
    lib().orc_gauss_tile_ranges(_ptr(mu), _ptr(scale), _ptr(quat), len(mu), _ptr(o), float(h), int(B),
                                _ptr(out))
    return out


def density(mu, scale, quat, alpha, origin, h, dims, B, nthreads: int = 0):
    """Eq. D(v) over the grid (FP64) and A(v) = sum of alpha^2 over the
    candidates of v's tile; both shaped [nz, ny, nx]."""
    mu, scale, quat, alpha = _f32(mu, 3), _f32(scale, 3), _f32(quat, 4), _f32(alpha, 0)
    o = np.ascontiguousarray(origin, np.float32)
    dm = np.ascontiguousarray(dims, np.int32)
    nx, ny, nz = (int(x) for x in dims)
    D = np.empty((nz, ny, nx), np.float64)
    A = np.empty((nz, ny, nx), np.float64)
    lib().orc_density(_ptr(mu), _ptr(scale), _ptr(quat), _ptr(alpha), len(mu), _ptr(o), float(h),
                      _ptr(dm), int(B), int(nthreads), _ptr(D), _ptr(A))
    return D, A


def density_tiles(mu, scale, quat, alpha, origin, h, dims, B, tiles, nthreads: int = 0):
    """Eq. D(v) and A(v) on the voxels of the listed tiles only (tile id
    (c*ty + b)*tx + a): two arrays [n_tiles, B, B, B] indexed [tile, k, j, i]
    (voxel (aB + i, bB + j, cB + k)), NaN past the grid's faces."""
    mu, scale, quat, alpha = _f32(mu, 3), _f32(scale, 3), _f32(quat, 4), _f32(alpha, 0)
    o = np.ascontiguousarray(origin, np.float32)
    dm = np.ascontiguousarray(dims, np.int32)
    t = np.ascontiguousarray(tiles, np.int64)
    D = np.empty((len(t), B, B, B), np.float64)
    A = np.empty((len(t), B, B, B), np.float64)
    lib().orc_density_tiles(_ptr(mu), _ptr(scale), _ptr(quat), _ptr(alpha), len(mu), _ptr(o), float(h),
                            _ptr(dm), int(B), _ptr(t), len(t), int(nthreads), _ptr(D), _ptr(A))
    return D, A


def occupancy(D, theta):
    """Eqs. V_occ and Surf from a density grid [nz, ny, nx]: (occ u8, surf u8)."""
    D = np.ascontiguousarray(D, np.float64)
    nz, ny, nx = D.shape
    dm = np.array([nx, ny, nz], np.int32)
    occ = np.empty(D.shape, np.uint8)
    surf = np.empty(D.shape, np.uint8)
    lib().orc_occupancy(_ptr(D), _ptr(dm), float(theta), _ptr(occ), _ptr(surf))
    return occ, surf


def density_tolerance(D, A):
    """Per-voxel tolerance of a float32 implementation of eq. D(v): each term
    alpha^2 exp(-q/2) carries an error of at most alpha^2 * 3e-5 (float32
    voxel-to-mean offsets within 5e-7 m at coordinates up to 10 m, scales of
    at least 1 cm: |dq| <= 1e-4 sqrt(q), and max_q exp(-q/2) sqrt(q)/2 < 0.43,
    plus the exponential's own error), and the float32 sum adds 1e-6 relative."""
    return 3e-5 * np.asarray(A) + 1e-6 * np.abs(np.asarray(D)) + 1e-9


# ---------------------------------------------------------------------------
# Mesh reconstruction (Sec. IV-B)
# ---------------------------------------------------------------------------

def blur_radius(sigma_vox: float) -> int:
    """Taps of the eq. V' kernel on each side: ceil(3 sigma) (sigma in voxels)."""
    return int(np.ceil(3.0 * float(sigma_vox)))


def blur(V, sigma_vox: float, radius: int | None = None):
    """Eq. V': the normalised Gaussian of sigma_vox voxels (radius taps a side,
    default ceil(3 sigma)) over a binary grid [nz, ny, nx], 0 outside; FP64."""
    V = np.ascontiguousarray(V, np.uint8)
    nz, ny, nx = V.shape
    R = blur_radius(sigma_vox) if radius is None else int(radius)
    out = np.empty(V.shape, np.float64)
    rc = lib().orc_blur(_ptr(V), nx, ny, nz, float(sigma_vox), R, _ptr(out))
    if rc:
        raise ValueError("orc_blur: bad arguments")
    return out


def rethreshold(Vp, mode: str, value: float):
    """Eq. rethresh: V~ = [V' >= tau] (mode "fixed", value tau) or
    [V' >= Quantile_q(V')] (mode "quantile", value q), the quantile being the
    order statistic of rank floor(q (N - 1)) in ascending order.  Returns
    (V~ u8, threshold)."""
    Vp = np.asarray(Vp)
    if mode == "fixed":
        thr = float(value)
    elif mode == "quantile":
        flat = np.sort(Vp.ravel())
        thr = float(flat[int(np.floor(float(value) * (flat.size - 1)))])
    else:
        raise ValueError(mode)
    return (Vp >= thr).astype(np.uint8), thr


def outside(V):
    """Sign of eq. phi: 1 where the flood fill over free voxels from the padded
    frame reaches, else 0 ([nz, ny, nx] u8)."""
    V = np.ascontiguousarray(V, np.uint8)
    nz, ny, nx = V.shape
    out = np.empty(V.shape, np.uint8)
    if lib().orc_outside(_ptr(V), nx, ny, nz, _ptr(out)):
        raise ValueError("orc_outside: bad arguments")
    return out


def shell(V, L: int):
    """First-arrival shell index p(x) from eq. S_0, shells up to L; 255 beyond."""
    V = np.ascontiguousarray(V, np.uint8)
    nz, ny, nx = V.shape
    p = np.empty(V.shape, np.uint8)
    if lib().orc_shell(_ptr(V), nx, ny, nz, int(L), _ptr(p)):
        raise ValueError("orc_shell: bad arguments")
    return p


def band_layers(h: float, r: float) -> int:
    """Shells needed for the band: ceil(r / h) (a voxel first reached later has
    (p + 1/2) h > r and is clipped anyway)."""
    return int(np.ceil(np.float64(np.float32(r)) / np.float64(np.float32(h))))


def tsdf(V, h: float, r: float, delta: str = "half"):
    """Eq. phi = clip(s delta, -r, r) for a surface grid V [nz, ny, nx], with
    eq. delta read as (p + 1/2) h (delta="half", the default) or literally as
    p h (delta="literal"); returns (phi f32, outside u8, p u8)."""
    if delta not in ("half", "literal"):
        raise ValueError("delta must be 'half' or 'literal'")
    V = np.ascontiguousarray(V, np.uint8)
    L = min(band_layers(h, r), 254)
    out = outside(V)
    p = shell(V, L)
    phi = np.empty(V.shape, np.float32)
    if lib().orc_tsdf(_ptr(out), _ptr(p), V.size, float(h), float(r), 1 if delta == "literal" else 0,
                      _ptr(phi)):
        raise ValueError("orc_tsdf: bad arguments")
    return phi, out, p


def marching_tets(phi, origin, h: float, iso: float = 0.0, step: int = 1, normals: bool = False):
    """The phi = iso level set by marching tetrahedra (canonical vertex and
    triangle order, normals towards phi >= iso).  Returns (verts f32 [nv, 3],
    tris i32 [nt, 3], normals f32 [nv, 3] or None)."""
    phi = np.ascontiguousarray(phi, np.float32)
    nz, ny, nx = phi.shape
    o = np.ascontiguousarray(origin, np.float32)
    pv, pt, pn = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    L = lib()
    rc = L.orc_marching_tets(_ptr(phi), nx, ny, nz, _ptr(o), float(h), float(iso), int(step),
                             int(bool(normals)), ctypes.byref(pv), ctypes.byref(nv), ctypes.byref(pt),
                             ctypes.byref(nt), ctypes.byref(pn) if normals else None)
    if rc:
        raise ValueError("orc_marching_tets: bad arguments")
    try:
        verts = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_float)),
                                      (max(nv.value, 1) * 3,))[:nv.value * 3].reshape(-1, 3).copy()
        tris = np.ctypeslib.as_array(ctypes.cast(pt, ctypes.POINTER(ctypes.c_int32)),
                                     (max(nt.value, 1) * 3,))[:nt.value * 3].reshape(-1, 3).copy()
        nrm = None
        if normals:
            nrm = np.ctypeslib.as_array(ctypes.cast(pn, ctypes.POINTER(ctypes.c_float)),
                                        (max(nv.value, 1) * 3,))[:nv.value * 3].reshape(-1, 3).copy()
    finally:
        L.orc_tsdf_free(pv)
        L.orc_tsdf_free(pt)
        if normals:
            L.orc_tsdf_free(pn)
    return verts, tris, nrm


def mesh_from_gaussians(mu, scale, quat, alpha, origin, h: float, dims, theta: float = 0.5,
                        trunc: float = 0.06, sigma="half-voxel", tau: float = 0.5, iso: float = 0.0,
                        step: int = 1, B: int = 8):
    """Sec. IV-A then IV-B, the oracle's steps in order: eq. D(v), eqs. V_occ
    and Surf, eq. V' with eq. rethresh (default sigma = h / 2, tau = 1/2;
    sigma=None skips them), the TSDF and its iso level set.  Returns (verts,
    tris)."""
    D, _ = density(mu, scale, quat, alpha, origin, h, dims, B)
    _, surf = occupancy(D, theta)
    if isinstance(sigma, str):
        sigma = 0.5 * h
    if sigma:
        sv = np.float64(np.float32(sigma)) / np.float64(np.float32(h))
        surf, _ = rethreshold(blur(surf, sv), "fixed", tau)
    phi, _, _ = tsdf(surf, h, trunc)
    v, t, _ = marching_tets(phi, origin, h, iso=iso, step=step)
    return v, t


def blur_tolerance(radius: int) -> float:
    """Absolute tolerance of a float32 eq. V' (values in [0, 1]): three passes
    of 2R + 1 float32 products and sums, each within 2^-24 relative, on
    partial sums at most 1, plus the weights' own float32 rounding."""
    return 4.0 * 3 * (2 * radius + 2) * 2.0 ** -24


def vertex_tolerance(verts, h: float) -> float:
    """Absolute tolerance on a float32 marching-tetrahedra vertex: the voxel
    centre (o + (i + 1/2) h) and the step along the edge each round a few
    times at the coordinate's magnitude; tau's own float32 error moves the
    vertex by at most 4 ulp of h."""
    mag = float(np.max(np.abs(verts))) if len(verts) else 1.0
    return 8 * 2.0 ** -24 * max(mag, 1.0) + 8 * 2.0 ** -24 * float(h)
