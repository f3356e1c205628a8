"""Procedural indoor triangle meshes (seeded).

The paper casts LiDAR rays against watertight meshes extracted from 3DGS
indoor scenes (Sec. IV-B, IV-C).  Those assets are not available, so these
generators make indoor-shaped stand-ins: a closed box room cluttered with
closed objects (axis-aligned boxes, face-subdivided boxes and icospheres).
Objects may overlap one another; each object is itself a closed surface.
"""

from __future__ import annotations

import dataclasses
import numpy as np


# ----------------------------------------------------------------------------
# primitive meshes
# ----------------------------------------------------------------------------

def _unit_cube_surface(n: int):
    """Surface of [0,1]^3 with every face split into an n x n grid of quads
    (2 triangles each).  Vertices on shared edges are shared, so the surface
    is closed: every edge belongs to exactly two triangles."""
    ids = {}
    verts = []

    def vid(i, j, k):
        key = (i, j, k)
        if key not in ids:
            ids[key] = len(verts)
            verts.append((i / n, j / n, k / n))
        return ids[key]

    tris = []
    # each face: fixed axis a at value s (0 or n); grid over the other two axes
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        for s in (0, n):
            for u in range(n):
                for v in range(n):
                    def p(uu, vv):
                        idx = [0, 0, 0]
                        idx[a], idx[b], idx[c] = s, uu, vv
                        return vid(*idx)
                    q00, q10, q11, q01 = p(u, v), p(u + 1, v), p(u + 1, v + 1), p(u, v + 1)
                    if s == 0:
                        tris.append((q00, q01, q11))
                        tris.append((q00, q11, q10))
                    else:
                        tris.append((q00, q10, q11))
                        tris.append((q00, q11, q01))
    return np.asarray(verts, np.float64), np.asarray(tris, np.int32)


_CUBE_CACHE: dict = {}


def aabb_box(lo, hi, subdiv: int = 1):
    """Closed axis-aligned box [lo, hi] with each face split subdiv x subdiv
    (12 * subdiv^2 triangles)."""
    if subdiv not in _CUBE_CACHE:
        _CUBE_CACHE[subdiv] = _unit_cube_surface(subdiv)
    uv, ut = _CUBE_CACHE[subdiv]
    lo = np.asarray(lo, np.float64)
    hi = np.asarray(hi, np.float64)
    return (lo + uv * (hi - lo)).astype(np.float32), ut.copy()


def box_room(size=(10.0, 8.0, 3.0)):
    """Closed room [0,Lx]x[0,Ly]x[0,Lz]: 6 walls of 2 triangles = 12 tris."""
    return aabb_box((0.0, 0.0, 0.0), size, 1)


_ICO_CACHE: dict = {}


def icosphere_unit(level: int):
    """Unit icosphere: the icosahedron (20 faces) with every face split into
    4 by edge midpoints ``level`` times and the vertices pushed onto the unit
    sphere (20 * 4^level triangles).  Returns float64 verts, int32 tris."""
    if level in _ICO_CACHE:
        return _ICO_CACHE[level]
    g = (1.0 + 5.0 ** 0.5) / 2.0
    v = [(-1, g, 0), (1, g, 0), (-1, -g, 0), (1, -g, 0),
         (0, -1, g), (0, 1, g), (0, -1, -g), (0, 1, -g),
         (g, 0, -1), (g, 0, 1), (-g, 0, -1), (-g, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.asarray(p, np.float64) / np.linalg.norm(p) for p in v]
    faces = list(f)
    for _ in range(level):
        mid = {}

        def midpoint(a, b):
            key = (min(a, b), max(a, b))
            if key not in mid:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                mid[key] = len(verts) - 1
            return mid[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    out = (np.asarray(verts, np.float64), np.asarray(faces, np.int32))
    _ICO_CACHE[level] = out
    return out


def merge_meshes(parts):
    """Concatenate (verts, tris) pairs into one mesh (vertex ids re-based)."""
    vs, ts, off = [], [], 0
    for v, t in parts:
        vs.append(np.asarray(v, np.float32))
        ts.append(np.asarray(t, np.int64) + off)
        off += len(v)
    return np.concatenate(vs).astype(np.float32), np.concatenate(ts).astype(np.int32)


# ----------------------------------------------------------------------------
# obstacles (for free-space pose sampling)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Obstacles:
    """Closed objects of a scene, kept for rejecting sensor positions that
    fall inside an object.  ``room`` is the room's extent (metres)."""
    room: np.ndarray                 # (3,)
    box_lo: np.ndarray               # (nb, 3)
    box_hi: np.ndarray               # (nb, 3)
    sph_c: np.ndarray                # (ns, 3)
    sph_r: np.ndarray                # (ns,)

    def blocked(self, p: np.ndarray, margin: float = 0.05) -> np.ndarray:
        """Boolean per point: inside (or within ``margin`` of) an object."""
        p = np.atleast_2d(p)
        out = np.zeros(len(p), bool)
        for s in range(0, len(p), 256):
            q = p[s:s + 256, None, :]
            if len(self.box_lo):
                inb = np.all((q >= self.box_lo[None] - margin) & (q <= self.box_hi[None] + margin), axis=2)
                out[s:s + 256] |= inb.any(axis=1)
            if len(self.sph_c):
                d2 = np.sum((q - self.sph_c[None]) ** 2, axis=2)
                out[s:s + 256] |= (d2 < (self.sph_r[None] + margin) ** 2).any(axis=1)
        return out

    def occupancy_grid(self, cell: float = 0.1, margin: float = 0.05):
        """Conservative boolean grid over the room: a cell is set when it
        overlaps an object's bounding box grown by ``margin``."""
        n = np.maximum(1, np.ceil(self.room / cell).astype(int))
        occ = np.zeros(tuple(n), bool)
        los = np.concatenate([self.box_lo, self.sph_c - self.sph_r[:, None]])
        his = np.concatenate([self.box_hi, self.sph_c + self.sph_r[:, None]])
        for lo, hi in zip(los - margin, his + margin):
            a = np.clip(np.floor(lo / cell).astype(int), 0, n - 1)
            b = np.clip(np.floor(hi / cell).astype(int), 0, n - 1)
            occ[a[0]:b[0] + 1, a[1]:b[1] + 1, a[2]:b[2] + 1] = True
        return occ, cell


# ----------------------------------------------------------------------------
# the two procedural indoor workloads
# ----------------------------------------------------------------------------

def tiny_room_scene(seed: int, room=(10.0, 8.0, 3.0), n_boxes: int = 8,
                    side_lo: float = 0.2, side_hi: float = 1.5):
    """Closed 10x8x3 m room (12 tris) plus ``n_boxes`` axis-aligned boxes
    (12 tris each) with sides uniform in [side_lo, side_hi] m, fully inside the
    room and resting on the floor z=0.  Returns (verts, tris, obstacles)."""
    rng = np.random.default_rng(seed)
    room = np.asarray(room, np.float64)
    parts = [box_room(room)]
    los, his = [], []
    for _ in range(n_boxes):
        side = rng.uniform(side_lo, side_hi, 3)
        xy = rng.uniform(0.0, 1.0, 2) * (room[:2] - side[:2])
        lo = np.array([xy[0], xy[1], 0.0])
        hi = lo + side
        los.append(lo)
        his.append(hi)
        parts.append(aabb_box(lo, hi, 1))
    v, t = merge_meshes(parts)
    obs = Obstacles(room, np.asarray(los), np.asarray(his), np.zeros((0, 3)), np.zeros(0))
    return v, t, obs


def indoor_scene(seed: int, room=(20.0, 15.0, 4.0), n_spheres: int = 2000,
                 sphere_level: int = 2, radius_median: float = 0.3,
                 radius_sigma: float = 0.5, radius_clip=(0.05, 1.5),
                 n_boxes: int = 834, box_subdiv: int = 6,
                 side_lo: float = 0.2, side_hi: float = 1.5):
    """Cluttered indoor room: a closed 20x15x4 m room, ``n_spheres``
    icospheres (20*4^level tris; radius log-normal with the given median and
    log-sigma, clipped) and ``n_boxes`` boxes with faces split box_subdiv^2
    (12*box_subdiv^2 tris; sides uniform in [side_lo, side_hi]).  Every
    object lies fully inside the room; objects may overlap.  With the defaults
    the mesh has 12 + 2000*320 + 834*432 = 1,000,300 triangles."""
    rng = np.random.default_rng(seed)
    room = np.asarray(room, np.float64)
    r = np.exp(np.log(radius_median) + radius_sigma * rng.standard_normal(n_spheres))
    r = np.clip(r, radius_clip[0], np.minimum(radius_clip[1], room.min() / 2 - 1e-3))
    c = r[:, None] + rng.uniform(0.0, 1.0, (n_spheres, 3)) * (room[None] - 2 * r[:, None])
    uv, ut = icosphere_unit(sphere_level)
    sv = (c[:, None, :] + r[:, None, None] * uv[None]).astype(np.float32)
    nvs = len(uv)
    st = (ut[None].astype(np.int64) + (np.arange(n_spheres) * nvs)[:, None, None])

    side = rng.uniform(side_lo, side_hi, (n_boxes, 3))
    blo = rng.uniform(0.0, 1.0, (n_boxes, 3)) * (room[None] - side)
    bhi = blo + side
    if box_subdiv not in _CUBE_CACHE:
        _CUBE_CACHE[box_subdiv] = _unit_cube_surface(box_subdiv)
    cv, ct = _CUBE_CACHE[box_subdiv]
    bv = (blo[:, None, :] + cv[None] * side[:, None, :]).astype(np.float32)
    nvb = len(cv)
    bt = (ct[None].astype(np.int64) + (np.arange(n_boxes) * nvb)[:, None, None])

    rv, rt = box_room(room)
    verts = np.concatenate([rv, sv.reshape(-1, 3), bv.reshape(-1, 3)]).astype(np.float32)
    off_s = len(rv)
    off_b = off_s + n_spheres * nvs
    tris = np.concatenate([rt.astype(np.int64), st.reshape(-1, 3) + off_s,
                           bt.reshape(-1, 3) + off_b]).astype(np.int32)
    obs = Obstacles(room, blo, bhi, c, r)
    return verts, tris, obs
