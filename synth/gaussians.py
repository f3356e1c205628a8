"""Seeded 3D Gaussian scenes, the input of the Gaussian-to-occupancy and
mesh-reconstruction steps and (through a mesher passed in by the caller) of
the heterogeneous ray-casting workload.  No step of the method lives here.

The paper converts pretrained 3DGS assets to meshes (Sec. IV-A/B).  With no
assets available, Gaussians are drawn on the surfaces of a procedural room:
means area-weighted over the floor, the four walls (the ceiling is left open
so the outside flood fill reaches the interior and walls get both faces) and
the surfaces of boxes and spheres inside; scales log-normal (median 4.5 cm,
log-sigma 0.75, clipped to 1-20 cm) per axis; uniformly random rotations;
opacity uniform in [0.3, 1].
"""

from __future__ import annotations

import dataclasses

import numpy as np


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
        r = min(r, 0.5 * L[2] - 1e-3)             # a sphere fits under the room's height
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


def grid_around(lo, hi, h: float, margin: float):
    """A voxel grid (origin, dims) of spacing h covering the box [lo, hi]
    grown by margin on every side."""
    lo = np.asarray(lo, np.float64) - margin
    hi = np.asarray(hi, np.float64) + margin
    dims = tuple(int(np.ceil((hi[a] - lo[a]) / h)) for a in range(3))
    return tuple(float(x) for x in lo), dims


def edge_manifold_report(tris: np.ndarray):
    """Counts of undirected edges by how many triangles use them; a closed
    (watertight) surface has every edge used exactly twice."""
    t = np.asarray(tris, np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e.sort(axis=1)
    key = e[:, 0] * (int(t.max()) + 1) + e[:, 1]
    _, cnt = np.unique(key, return_counts=True)
    return np.bincount(cnt)
