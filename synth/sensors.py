"""LiDAR scan patterns as per-ray (elevation, azimuth) tables.

The paper only says each beam has a unit direction fixed by the scanning
pattern (Sec. IV-C).  Grid sensors here use evenly spaced elevation rows
(inclusive of both end angles) and azimuth columns ``2*pi*k/n_az``; the
non-repetitive pattern is a rose curve around the forward (+x) axis.
Angles are returned as float32 radians; turning them into direction vectors
is the consumer's job.
"""

from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class SensorTable:
    elev: np.ndarray     # float32 [n_rays] radians
    azim: np.ndarray     # float32 [n_rays] radians
    rows: int            # grid rows (beams); 1 for non-grid patterns
    cols: int            # grid columns (azimuth steps); n_rays for non-grid
    name: str = ""

    @property
    def n_rays(self) -> int:
        return int(self.elev.shape[0])


def grid_sensor(n_beams: int, elev_lo_deg: float, elev_hi_deg: float, n_az: int,
                name: str = "") -> SensorTable:
    """Spinning-LiDAR grid: ``n_beams`` elevations evenly spaced over
    [elev_lo, elev_hi] (both included) x ``n_az`` azimuths 2*pi*k/n_az.
    Ray order is row-major: r = beam_row * n_az + az_col."""
    if n_beams == 1:
        el = np.array([np.deg2rad(elev_lo_deg)])
    else:
        el = np.deg2rad(np.linspace(elev_lo_deg, elev_hi_deg, n_beams))
    az = 2.0 * np.pi * np.arange(n_az) / n_az
    E, A = np.meshgrid(el, az, indexing="ij")
    return SensorTable(E.reshape(-1).astype(np.float32), A.reshape(-1).astype(np.float32),
                       n_beams, n_az, name or f"grid{n_beams}x{n_az}")


def rosette_sensor(n_rays: int = 20000, seed: int = 0, fov_deg: float = 35.0,
                   dt: float = 1e-3, w1: float = 2.0 * np.pi * 61.0) -> SensorTable:
    """Non-repetitive rosette (rose-curve) pattern around +x: the angle off
    the forward axis is rho = fov*sin(w1*t + phase) and the angle around it is
    psi = w2*t, with w1/w2 the golden ratio so the curve never closes.
    Converted to (elevation, azimuth) of the direction
    (cos rho, sin rho cos psi, sin rho sin psi)."""
    rng = np.random.default_rng(seed)
    phase = rng.uniform(0.0, 2.0 * np.pi)
    golden = (1.0 + 5.0 ** 0.5) / 2.0
    w2 = w1 / golden
    t = np.arange(n_rays) * dt
    rho = np.deg2rad(fov_deg) * np.sin(w1 * t + phase)
    psi = w2 * t
    dx = np.cos(rho)
    dy = np.sin(rho) * np.cos(psi)
    dz = np.sin(rho) * np.sin(psi)
    el = np.arcsin(np.clip(dz, -1.0, 1.0))
    az = np.arctan2(dy, dx)
    return SensorTable(el.astype(np.float32), az.astype(np.float32), 1, n_rays, f"rosette{n_rays}")


# The mixed sensor set of the heterogeneous workload: spinning LiDARs of
# 16/32/64/128 beams (VLP/HDL/OS-class elevation spans) at several azimuth
# resolutions, plus the rosette.
MIXED_BEAMS = {16: (-15.0, 15.0), 32: (-16.0, 15.0), 64: (-24.9, 2.0), 128: (-22.5, 22.5)}
MIXED_AZ = (360, 512, 1024, 1800, 2048)


def mixed_sensors(seed: int = 0):
    """One table per (beams, azimuth) pair of the mixed set, plus the
    20k-ray rosette."""
    out = []
    for b, (lo, hi) in MIXED_BEAMS.items():
        for a in MIXED_AZ:
            out.append(grid_sensor(b, lo, hi, a))
    out.append(rosette_sensor(20000, seed))
    return out
