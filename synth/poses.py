"""Sensor poses T_s in SE(3) as float32 row-major [R | t] (3x4).

Rotations are formed in float64 and rounded to float32 once.
"""

from __future__ import annotations

import numpy as np


def _axis_angle(axis: np.ndarray, ang: np.ndarray) -> np.ndarray:
    """Rodrigues rotation matrices for unit axes [n,3] and angles [n]."""
    axis = np.atleast_2d(axis)
    ang = np.atleast_1d(ang)
    x, y, z = axis[:, 0], axis[:, 1], axis[:, 2]
    c, s = np.cos(ang), np.sin(ang)
    C = 1.0 - c
    R = np.empty((len(ang), 3, 3))
    R[:, 0, 0] = c + x * x * C
    R[:, 0, 1] = x * y * C - z * s
    R[:, 0, 2] = x * z * C + y * s
    R[:, 1, 0] = y * x * C + z * s
    R[:, 1, 1] = c + y * y * C
    R[:, 1, 2] = y * z * C - x * s
    R[:, 2, 0] = z * x * C - y * s
    R[:, 2, 1] = z * y * C + x * s
    R[:, 2, 2] = c + z * z * C
    return R


def _pack(R: np.ndarray, t: np.ndarray) -> np.ndarray:
    R = np.atleast_3d(R).reshape(-1, 3, 3)
    t = np.atleast_2d(t).reshape(-1, 3)
    P = np.concatenate([R, t[:, :, None]], axis=2)
    return P.astype(np.float32)


def pose_from_yaw(pos, yaw) -> np.ndarray:
    """[n,3,4] poses with a rotation about +z by ``yaw`` radians."""
    yaw = np.atleast_1d(np.asarray(yaw, np.float64))
    R = _axis_angle(np.tile([0.0, 0.0, 1.0], (len(yaw), 1)), yaw)
    return _pack(R, np.asarray(pos, np.float64))


def _unit_vectors(rng, n):
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_rotation(rng, n: int) -> np.ndarray:
    """Uniformly distributed rotations (normalised Gaussian quaternions)."""
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.empty((n, 3, 3))
    R[:, 0] = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], 1)
    R[:, 1] = np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], 1)
    R[:, 2] = np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1)
    return R


def sample_free_pose(rng, obstacles, n: int = 1, margin: float = 0.3,
                     upright: bool = True, max_tries: int = 10000) -> np.ndarray:
    """``n`` poses with positions uniform in the room shrunk by ``margin``
    and outside every object; yaw-only (upright) or fully random rotation."""
    room = obstacles.room
    out = np.empty((0, 3))
    tries = 0
    while len(out) < n:
        k = max(64, 2 * (n - len(out)))
        p = margin + rng.uniform(0.0, 1.0, (k, 3)) * (room - 2 * margin)
        p = p[~obstacles.blocked(p)]
        out = np.concatenate([out, p])[:n]
        tries += k
        if tries > max_tries * max(1, n):
            raise RuntimeError("could not find free sensor positions")
    if upright:
        return pose_from_yaw(out, rng.uniform(0.0, 2 * np.pi, n))
    return _pack(random_rotation(rng, n), out)


def random_walk(rng, obstacles, n_env: int, n_steps: int, step: float = 0.1,
                rot_deg: float = 2.0, margin: float = 0.3, retries: int = 8) -> np.ndarray:
    """Seeded SE(3) random walks: each env starts at a free upright pose; at
    every step it translates ``step`` metres along a uniform random direction
    (reflected at the room walls shrunk by ``margin``; a step that lands in
    an occupied grid cell is redrawn up to ``retries`` times, else the env
    stays) and rotates ``rot_deg`` degrees about a uniform random axis.
    Returns float32 [n_steps, n_env, 3, 4]."""
    P0 = sample_free_pose(rng, obstacles, n_env)
    R = P0[:, :, :3].astype(np.float64)
    t = P0[:, :, 3].astype(np.float64)
    occ, cell = obstacles.occupancy_grid()
    nmax = np.array(occ.shape) - 1
    lo, hi = np.full(3, margin), obstacles.room - margin
    out = np.empty((n_steps, n_env, 3, 4), np.float32)
    for s in range(n_steps):
        out[s] = _pack(R, t)
        todo = np.ones(n_env, bool)
        newt = t.copy()
        for _ in range(retries):
            idx = np.nonzero(todo)[0]
            if len(idx) == 0:
                break
            cand = t[idx] + step * _unit_vectors(rng, len(idx))
            # reflect at the shrunk walls
            cand = np.where(cand < lo, 2 * lo - cand, cand)
            cand = np.where(cand > hi, 2 * hi - cand, cand)
            cand = np.clip(cand, lo, hi)
            cidx = np.clip(np.floor(cand / cell).astype(int), 0, nmax)
            ok = ~occ[cidx[:, 0], cidx[:, 1], cidx[:, 2]]
            newt[idx[ok]] = cand[ok]
            todo[idx[ok]] = False
        t = newt
        dR = _axis_angle(_unit_vectors(rng, n_env), np.full(n_env, np.deg2rad(rot_deg)))
        R = np.einsum("nij,njk->nik", R, dR)
        # re-orthonormalise (polar decomposition via SVD) to stop drift
        u, _, vt = np.linalg.svd(R)
        R = np.einsum("nij,njk->nik", u, vt)
    return out
