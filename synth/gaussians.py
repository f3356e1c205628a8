"""Seeded 3D Gaussian scenes and their host mesher (TSDF + marching
tetrahedra), the input generator of the heterogeneous ray-casting workload.

The paper converts pretrained 3DGS assets to meshes (Sec. IV-A/B).  With no
assets available, Gaussians are drawn on the surfaces of a procedural room:
means area-weighted over the floor, the four walls (the ceiling is left open
so the outside flood fill reaches the interior and walls get both faces) and
the surfaces of boxes and spheres inside; scales log-normal (median 4.5 cm,
log-sigma 0.75, clipped to 1-20 cm) per axis; uniformly random rotations;
opacity uniform in [0.3, 1].
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mesher.cpp")
_LIB = os.path.join(_HERE, "_build", "libmesher.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread", _SRC, "-o", tmp],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
            L.mesher_run.argtypes = [P, P, P, P, I64, D, D, D, I32, P, P, P, P, P]
            L.mesher_run.restype = I32
            L.mesher_free.argtypes = [P]
            _lib = L
    return _lib


@dataclasses.dataclass
class GaussianSet:
    mu: np.ndarray       # [n,3]
    scale: np.ndarray    # [n,3]
    quat: np.ndarray     # [n,4] (w, x, y, z)
    alpha: np.ndarray    # [n]

    def __len__(self):
        return len(self.alpha)


def _sample_surfaces(rng, rects, spheres, n):
    """Area-weighted points on axis-aligned rectangles (lo, hi with one flat
    axis) and sphere surfaces (centre, radius)."""
    areas = []
    for lo, hi in rects:
        e = np.sort(hi - lo)[1:]
        areas.append(e[0] * e[1])
    for c, r in spheres:
        areas.append(4 * np.pi * r * r)
    areas = np.asarray(areas)
    counts = rng.multinomial(n, areas / areas.sum())
    pts = []
    for (lo, hi), k in zip(rects, counts[:len(rects)]):
        pts.append(lo + rng.uniform(0, 1, (k, 3)) * (hi - lo))
    for (c, r), k in zip(spheres, counts[len(rects):]):
        v = rng.standard_normal((k, 3))
        pts.append(c + r * v / np.linalg.norm(v, axis=1, keepdims=True))
    return np.concatenate(pts)


def gaussian_room(seed: int, room=(6.0, 5.0, 3.0), n_gauss: int = 200_000, n_boxes: int = 6,
                  n_spheres: int = 4, with_obstacles: bool = False):
    """Gaussians on the surfaces of an open-topped room with boxes and
    spheres; with_obstacles=True also returns the solid objects (for sampling
    free sensor poses)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(room, np.float64)
    rects = [(np.array([0, 0, 0.0]), np.array([L[0], L[1], 0.0]))]                 # floor
    rects += [(np.array([0, 0, 0.0]), np.array([0.0, L[1], L[2]])),
              (np.array([L[0], 0, 0.0]), np.array([L[0], L[1], L[2]])),
              (np.array([0, 0, 0.0]), np.array([L[0], 0.0, L[2]])),
              (np.array([0, L[1], 0.0]), np.array([L[0], L[1], L[2]]))]            # walls
    for _ in range(n_boxes):
        side = rng.uniform(0.3, 1.5, 3)
        lo = np.r_[rng.uniform(0.3, 1, 2) * (L[:2] - side[:2] - 0.3), 0.0]
        hi = lo + side
        for a in range(3):
            for v in (lo[a], hi[a]):
                l2, h2 = lo.copy(), hi.copy()
                l2[a] = h2[a] = v
                rects.append((l2, h2))
    boxes = []
    for b in range(n_boxes):
        fr = rects[5 + 6 * b: 11 + 6 * b]
        lo = np.min([f[0] for f in fr], axis=0)
        hi = np.max([f[1] for f in fr], axis=0)
        boxes.append((lo, hi))
    spheres = []
    for _ in range(n_spheres):
        r = rng.uniform(0.2, 0.6)
        c = np.r_[r + 0.3 + rng.uniform(0, 1, 2) * (L[:2] - 2 * r - 0.6), rng.uniform(r, L[2] - r)]
        spheres.append((c, r))
    mu = _sample_surfaces(rng, rects, spheres, n_gauss)
    scale = np.clip(np.exp(np.log(0.045) + 0.75 * rng.standard_normal((n_gauss, 3))), 0.01, 0.20)
    q = rng.standard_normal((n_gauss, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    alpha = rng.uniform(0.3, 1.0, n_gauss)
    gs = GaussianSet(mu.astype(np.float32), scale.astype(np.float32), q.astype(np.float32),
                     alpha.astype(np.float32))
    if not with_obstacles:
        return gs
    from .scenes import Obstacles
    obs = Obstacles(L, np.asarray([b[0] for b in boxes]).reshape(-1, 3),
                    np.asarray([b[1] for b in boxes]).reshape(-1, 3),
                    np.asarray([c for c, r in spheres]).reshape(-1, 3),
                    np.asarray([r for c, r in spheres]))
    return gs, obs


def mesh_from_gaussians(gs: GaussianSet, voxel: float, theta: float = 0.5, trunc: float = 0.06,
                        threads: int = 0):
    """Run the host mesher; returns (verts f32 [nv,3], tris i32 [nt,3], stats)."""
    L = _load()
    mu = np.ascontiguousarray(gs.mu, np.float32)
    sc = np.ascontiguousarray(gs.scale, np.float32)
    qu = np.ascontiguousarray(gs.quat, np.float32)
    al = np.ascontiguousarray(gs.alpha, np.float32)
    pv, pt = ctypes.c_void_p(), ctypes.c_void_p()
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    stats = np.zeros(8, np.float64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = L.mesher_run(p(mu), p(sc), p(qu), p(al), len(al), float(voxel), float(theta), float(trunc),
                      int(threads), ctypes.byref(pv), ctypes.byref(nv), ctypes.byref(pt),
                      ctypes.byref(nt), p(stats))
    if rc != 0:
        raise RuntimeError(f"mesher failed (code {rc})")
    try:
        v = np.ctypeslib.as_array(ctypes.cast(pv, ctypes.POINTER(ctypes.c_float)), (nv.value * 3,)).copy()
        t = np.ctypeslib.as_array(ctypes.cast(pt, ctypes.POINTER(ctypes.c_int32)), (nt.value * 3,)).copy()
    finally:
        L.mesher_free(pv)
        L.mesher_free(pt)
    st = {"grid": stats[:3].astype(int).tolist(), "occupied": int(stats[3]), "surface_voxels": int(stats[4]),
          "outside_voxels": int(stats[5])}
    return v.reshape(-1, 3), t.reshape(-1, 3), st


def edge_manifold_report(tris: np.ndarray):
    """Counts of undirected edges by how many triangles use them; a closed
    (watertight) surface has every edge used exactly twice."""
    t = np.asarray(tris, np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e.sort(axis=1)
    key = e[:, 0] * (int(t.max()) + 1) + e[:, 1]
    _, cnt = np.unique(key, return_counts=True)
    return np.bincount(cnt)
