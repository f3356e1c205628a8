"""Host mesher (input generator of the heterogeneous workload): seeded
Gaussians -> density -> occupancy -> surface shell -> outside flood fill ->
shell distance -> TSDF -> marching tetrahedra (paper Sec. IV-A/B)."""

import numpy as np

from synth import gaussians as G


def test_mesh_is_watertight_and_oriented():
    gs = G.gaussian_room(3, (2.0, 1.5, 1.0), 40_000, n_boxes=1, n_spheres=1)
    v, t, st = G.mesh_from_gaussians(gs, 0.05)
    assert len(t) > 10_000
    hist = G.edge_manifold_report(t)
    assert hist.sum() == hist[2], hist            # every edge in exactly two triangles
    # consistent orientation: each directed edge appears once (shared edges opposite)
    d = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]).astype(np.int64)
    key = d[:, 0] * (int(t.max()) + 1) + d[:, 1]
    assert len(np.unique(key)) == len(key)
    assert np.all(np.isfinite(v))


def test_single_isotropic_gaussian_gives_a_sphere():
    # one Gaussian, sigma 0.1, alpha 1: D(x) = exp(-|x|^2 / (2 sigma^2)) > theta is
    # a ball of radius sigma * sqrt(2 ln(1/theta)); the extracted surface sits
    # between the occupied shell and the first free voxels, within ~1.5 voxels
    s, theta, h = 0.1, 0.5, 0.01
    gs = G.GaussianSet(np.zeros((1, 3), np.float32), np.full((1, 3), s, np.float32),
                       np.array([[1, 0, 0, 0]], np.float32), np.ones(1, np.float32))
    v, t, st = G.mesh_from_gaussians(gs, h, theta=theta, trunc=0.03)
    r = np.linalg.norm(v, axis=1)
    R = s * np.sqrt(2 * np.log(1 / theta))
    assert abs(np.median(r) - R) < 1.5 * h and r.max() - r.min() < 3 * h
    assert G.edge_manifold_report(t)[2] == 3 * len(t) // 2


def test_interior_of_closed_object_is_inside():
    # a closed sphere of Gaussians: the mesh has an outer surface only near r
    rng = np.random.default_rng(1)
    n = 30_000
    p = rng.standard_normal((n, 3))
    p = 0.5 * p / np.linalg.norm(p, axis=1, keepdims=True)
    gs = G.GaussianSet(p.astype(np.float32), np.full((n, 3), 0.03, np.float32),
                       np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)), np.ones(n, np.float32))
    v, t, st = G.mesh_from_gaussians(gs, 0.02, theta=0.5)
    r = np.linalg.norm(v, axis=1)
    assert r.min() > 0.5 and r.max() < 0.62                    # outer surface of the shell only
    assert G.edge_manifold_report(t)[2] == 3 * len(t) // 2
