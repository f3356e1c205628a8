"""Pins for the FP64 Gaussian-to-occupancy oracle (paper Sec. IV-A) against
things other than itself.

Each pin targets a plausible mistake: the Gaussian kernel against SciPy's
multivariate normal density with SciPy's own quaternion rotation (a
transposed rotation, a wrong scale power, a missing factor 1/2 or alpha
instead of alpha^2), the tile rule of eq. C_tile against an ellipsoid AABB
derived independently (a 3-sigma box computed from the covariance diagonal
in FP64), linearity in the Gaussians, and closed forms of the surface mask
(eqs. Int, Surf) on boxes of occupied voxels.
"""

import numpy as np
import pytest

import oracle

scipy_stats = pytest.importorskip("scipy.stats")
scipy_rot = pytest.importorskip("scipy.spatial.transform")


def random_gaussians(rng, n, lo, hi, smin=0.02, smax=0.2):
    mu = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    scale = np.exp(rng.uniform(np.log(smin), np.log(smax), (n, 3))).astype(np.float32)
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    alpha = rng.uniform(0.2, 1.0, n).astype(np.float32)
    return mu, scale, q.astype(np.float32), alpha


def centres(origin, h, dims):
    """Voxel centres in FP64 from the float32 grid parameters (as given to
    the oracle)."""
    nx, ny, nz = dims
    o = np.asarray(origin, np.float32).astype(np.float64)
    h = float(np.float32(h))
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([o[0] + (i + 0.5) * h, o[1] + (j + 0.5) * h, o[2] + (k + 0.5) * h], -1)


def scipy_kernel(mu, scale, quat, alpha, pts):
    """alpha^2 exp(-q/2) through SciPy: the normal pdf times its normaliser."""
    w, x, y, z = (float(c) for c in quat)
    R = scipy_rot.Rotation.from_quat([x, y, z, w]).as_matrix()       # SciPy is scalar-last
    cov = R @ np.diag(np.asarray(scale, np.float64) ** 2) @ R.T
    mvn = scipy_stats.multivariate_normal(np.asarray(mu, np.float64), cov)
    norm = np.sqrt((2 * np.pi) ** 3 * np.linalg.det(cov))
    return float(alpha) ** 2 * mvn.pdf(pts.reshape(-1, 3)).reshape(pts.shape[:-1]) * norm


def test_single_gaussian_matches_scipy_when_one_tile_covers_the_grid():
    rng = np.random.default_rng(1)
    mu, sc, q, al = random_gaussians(rng, 6, 0.3, 0.9)
    dims, h, o = (12, 10, 9), 0.1, (0.0, 0.05, -0.1)
    pts = centres(o, h, dims)
    for g in range(6):
        D, A = oracle.density(mu[g:g + 1], sc[g:g + 1], q[g:g + 1], al[g:g + 1], o, h, dims, 16)
        ref = scipy_kernel(mu[g], sc[g], q[g], al[g], pts)
        np.testing.assert_allclose(D, ref, rtol=1e-10, atol=1e-14)
        assert np.all(A == np.float64(al[g]) ** 2)


def test_isotropic_closed_form_and_alpha_squared():
    mu = np.array([[0.55, 0.55, 0.55]], np.float32)
    sc = np.array([[0.1, 0.1, 0.1]], np.float32)
    q = np.array([[0.3, -0.2, 0.9, 0.1]], np.float32)          # any rotation of a sphere
    for a in (1.0, 0.5):
        D, _ = oracle.density(mu, sc, q, np.array([a], np.float32), (0, 0, 0), 0.1, (11, 11, 11), 11)
        # voxel (5,5,5) is the mean itself
        assert D[5, 5, 5] == pytest.approx(a * a, rel=1e-15)
        r2 = 3 * (0.1) ** 2                                       # voxel (6,6,6): one h along every axis
        assert D[6, 6, 6] == pytest.approx(a * a * np.exp(-0.5 * r2 / np.float64(np.float32(0.1)) ** 2), rel=1e-6)


def test_tile_rule_against_an_independent_3sigma_box():
    """A voxel receives a Gaussian's term exactly when the 3-sigma box of the
    Gaussian meets the voxel's tile (boxes placed away from tile borders)."""
    rng = np.random.default_rng(7)
    dims, h, B, o = (32, 24, 16), 0.05, 4, (0.0, 0.0, 0.0)
    cell = B * h
    pts = centres(o, h, dims)
    tested = 0
    for _ in range(40):
        mu, sc, q, al = random_gaussians(rng, 1, 0.2, 0.7, 0.01, 0.08)
        w, x, y, z = (float(c) for c in q[0])
        R = scipy_rot.Rotation.from_quat([x, y, z, w]).as_matrix()
        cov = R @ np.diag(sc[0].astype(np.float64) ** 2) @ R.T
        e = 3 * np.sqrt(np.diag(cov))
        lo = (mu[0] - e - np.asarray(o)) / float(np.float32(cell))
        hi = (mu[0] + e - np.asarray(o)) / float(np.float32(cell))
        if np.min(np.abs(np.concatenate([lo, hi]) - np.round(np.concatenate([lo, hi])))) < 1e-3:
            continue                                              # too close to a tile border
        tested += 1
        tlo, thi = np.floor(lo).astype(int), np.floor(hi).astype(int)
        k, j, i = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
        ti, tj, tk = i // B, j // B, k // B
        inside = ((tlo[0] <= ti) & (ti <= thi[0]) & (tlo[1] <= tj) & (tj <= thi[1]) &
                  (tlo[2] <= tk) & (tk <= thi[2]))
        D, A = oracle.density(mu, sc, q, al, o, h, dims, B)
        ref = scipy_kernel(mu[0], sc[0], q[0], al[0], pts)
        assert np.all(D[~inside] == 0.0) and np.all(A[~inside] == 0.0)
        np.testing.assert_allclose(D[inside], ref[inside], rtol=1e-10, atol=1e-15)
        rr = oracle.gauss_tile_ranges(mu, sc, q, o, h, B)[0]
        assert list(rr[:3]) == list(tlo) and list(rr[3:]) == list(thi)
    assert tested >= 20


def test_density_is_linear_in_the_gaussians():
    rng = np.random.default_rng(3)
    mu, sc, q, al = random_gaussians(rng, 30, 0.0, 1.0)
    dims, h, B, o = (20, 20, 20), 0.05, 4, (0, 0, 0)
    D, A = oracle.density(mu, sc, q, al, o, h, dims, B)
    D1, A1 = oracle.density(mu[:13], sc[:13], q[:13], al[:13], o, h, dims, B)
    D2, A2 = oracle.density(mu[13:], sc[13:], q[13:], al[13:], o, h, dims, B)
    np.testing.assert_allclose(D, D1 + D2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(A, A1 + A2, rtol=1e-12, atol=1e-15)


def test_invalid_gaussians_contribute_nothing():
    mu = np.array([[0.5, 0.5, 0.5]] * 4, np.float32)
    sc = np.array([[0.1, 0.1, 0.1], [0.0, 0.1, 0.1], [0.1, -1, 0.1], [0.1, 0.1, 0.1]], np.float32)
    q = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0]], np.float32)
    mu[3, 0] = np.nan
    D, A = oracle.density(mu, sc, q, np.ones(4, np.float32), (0, 0, 0), 0.1, (10, 10, 10), 4)
    assert np.all(D == 0) and np.all(A == 0)


@pytest.mark.parametrize("box", [((2, 3, 1), (7, 9, 6)), ((0, 0, 0), (5, 4, 3)), ((1, 1, 1), (2, 2, 2))])
def test_surface_mask_closed_form_on_boxes(box):
    """A solid a x b x c block of occupied voxels: its interior is the
    (a-2)(b-2)(c-2) block inside (faces on the grid border stay surface)."""
    dims = (10, 11, 8)
    D = np.zeros((dims[2], dims[1], dims[0]))
    (x0, y0, z0), (x1, y1, z1) = box
    D[z0:z1, y0:y1, x0:x1] = 1.0
    occ, surf = oracle.occupancy(D, 0.5)
    assert occ.sum() == (x1 - x0) * (y1 - y0) * (z1 - z0)
    a, b, c = x1 - x0, y1 - y0, z1 - z0
    interior = max(a - 2, 0) * max(b - 2, 0) * max(c - 2, 0)
    assert surf.sum() == a * b * c - interior
    assert np.all(surf <= occ)
    if interior:
        assert surf[z0 + 1:z1 - 1, y0 + 1:y1 - 1, x0 + 1:x1 - 1].sum() == 0


def test_threshold_is_strict():
    D = np.full((3, 3, 3), 0.5)
    D[1, 1, 1] = np.nextafter(0.5, 1)
    occ, surf = oracle.occupancy(D, 0.5)
    assert occ.sum() == 1 and surf.sum() == 1


def test_density_on_listed_tiles_equals_the_full_grid():
    """orc_density_tiles (the full-size GPU tests' sampled oracle) returns the
    full-grid density's values, bit for bit, on the listed tiles (ragged
    tiles past the faces marked NaN)."""
    rng = np.random.default_rng(1)
    n = 300
    mu = rng.uniform(0.1, 0.9, (n, 3)).astype(np.float32)
    sc = np.exp(rng.uniform(np.log(0.02), np.log(0.15), (n, 3))).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)
    al = rng.uniform(0.3, 1, n).astype(np.float32)
    dims, h, o = (21, 19, 17), 0.05, (0.0, 0.0, 0.0)
    D, A = oracle.density(mu, sc, q, al, o, h, dims, 8)
    tiles = np.array([0, 5, 13, 26])
    Dt, At = oracle.density_tiles(mu, sc, q, al, o, h, dims, 8, tiles)
    for k, t in enumerate(tiles):
        a, b, c = t % 3, (t // 3) % 3, t // 9
        sub = D[c * 8:c * 8 + 8, b * 8:b * 8 + 8, a * 8:a * 8 + 8]
        subA = A[c * 8:c * 8 + 8, b * 8:b * 8 + 8, a * 8:a * 8 + 8]
        blk = Dt[k][:sub.shape[0], :sub.shape[1], :sub.shape[2]]
        blkA = At[k][:sub.shape[0], :sub.shape[1], :sub.shape[2]]
        assert np.array_equal(sub, blk) and np.array_equal(subA, blkA)
        assert np.isnan(Dt[k]).sum() == 512 - sub.size
