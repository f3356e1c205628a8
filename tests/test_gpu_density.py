"""GPU parity of the Gaussian-to-occupancy conversion (paper Sec. IV-A)
against the FP64 oracle, through the C-ABI.

Contract: |D_gpu - D_oracle| <= oracle.density_tolerance(D, A) per voxel
(float32 offsets and exponentials, float32 sums); the candidate pair count is
an integer decided in float32 by the same operation sequence on both sides,
so it is compared exactly; occupancy and the surface mask are compared
exactly except where the oracle's density lies within the tolerance of theta
(and, for the surface mask, next to such a voxel).
"""

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

fgl = pytest.importorskip("paper_2509_17390_gb300")


def random_gaussians(rng, n, lo, hi, smin=0.01, smax=0.2):
    mu = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    scale = np.exp(rng.uniform(np.log(smin), np.log(smax), (n, 3))).astype(np.float32)
    q = rng.standard_normal((n, 4)).astype(np.float32)              # not normalised on purpose
    alpha = rng.uniform(0.2, 1.0, n).astype(np.float32)
    return mu, scale, q, alpha


def run_gpu(mu, scale, q, alpha, origin, h, dims, theta, tile):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    D, occ, surf, st = fgl.gaussian_density(t(mu), t(scale), t(q), t(alpha), origin, h, dims,
                                            theta=theta, tile=tile)
    torch.cuda.synchronize()
    return D.cpu().numpy(), occ.cpu().numpy(), surf.cpu().numpy(), st


def expected_pairs(mu, scale, q, origin, h, dims, tile):
    r = oracle.gauss_tile_ranges(mu, scale, q, origin, h, tile).astype(np.int64)
    nt = np.array([(d + tile - 1) // tile for d in dims])
    lo = np.maximum(r[:, :3], 0)
    hi = np.minimum(r[:, 3:], nt - 1)
    ext = np.clip(hi - lo + 1, 0, None)
    return int(np.prod(ext, axis=1).sum())


def check_parity(mu, scale, q, alpha, origin, h, dims, theta, tile):
    D, occ, surf, st = run_gpu(mu, scale, q, alpha, origin, h, dims, theta, tile)
    Do, Ao = oracle.density(mu, scale, q, alpha, origin, h, dims, tile)
    tol = oracle.density_tolerance(Do, Ao)
    err = np.abs(D.astype(np.float64) - Do)
    assert np.all(err <= tol), (float(err.max()), float((err / tol).max()))
    assert st["n_pairs"] == expected_pairs(mu, scale, q, origin, h, dims, tile)
    occ_o, surf_o = oracle.occupancy(Do, theta)
    amb = np.abs(Do - theta) <= tol
    assert np.array_equal(occ[~amb], occ_o[~amb])
    near = amb.copy()
    for ax in range(3):
        for sh in (-1, 1):
            near |= np.roll(amb, sh, axis=ax)
    assert np.array_equal(surf[~near], surf_o[~near])
    # the GPU's own masks follow from its own density exactly
    occ_g, surf_g = oracle.occupancy(D.astype(np.float64), np.float64(np.float32(theta)))
    assert np.array_equal(occ, occ_g) and np.array_equal(surf, surf_g)
    return D, st, amb.mean()


@pytest.mark.parametrize("tile", [8, 4])
def test_random_gaussians_vs_oracle(tile):
    rng = np.random.default_rng(10 + tile)
    mu, sc, q, al = random_gaussians(rng, 400, 0.0, 1.2)
    D, st, amb = check_parity(mu, sc, q, al, (-0.05, 0.02, 0.0), 0.04, (33, 29, 27), 0.5, tile)
    assert st["n_pairs"] > 400 and D.max() > 0.5 and amb < 0.01


def test_room_gaussians_vs_oracle():
    """Gaussians on the surfaces of a small procedural room (the heterogeneous
    workload's generator), 5 cm voxels."""
    from synth import gaussians
    gs = gaussians.gaussian_room(41, (2.0, 1.5, 1.0), 20_000, 1, 1)
    h = 0.05
    dims = (44, 34, 24)
    origin = (-0.1, -0.1, -0.1)
    D, st, amb = check_parity(gs.mu, gs.scale, gs.quat, gs.alpha, origin, h, dims, 0.5, 8)
    assert amb < 0.01 and (D > 0.5).mean() > 0.02


def test_deterministic_and_ragged_edges():
    rng = np.random.default_rng(3)
    mu, sc, q, al = random_gaussians(rng, 300, -0.1, 0.6)
    dims = (17, 9, 23)                                      # no dimension a multiple of 8
    a = run_gpu(mu, sc, q, al, (0, 0, 0), 0.03, dims, 0.4, 8)
    b = run_gpu(mu, sc, q, al, (0, 0, 0), 0.03, dims, 0.4, 8)
    assert all(np.array_equal(x, y) for x, y in zip(a[:3], b[:3]))
    check_parity(mu, sc, q, al, (0, 0, 0), 0.03, dims, 0.4, 8)


def test_edge_cases():
    z = np.zeros((0, 3), np.float32)
    D, occ, surf, st = run_gpu(z, z, np.zeros((0, 4), np.float32), np.zeros(0, np.float32),
                               (0, 0, 0), 0.1, (5, 6, 7), 0.5, 8)
    assert D.shape == (7, 6, 5) and np.all(D == 0) and occ.sum() == 0 and st["n_pairs"] == 0
    # invalid Gaussians and Gaussians entirely outside the grid contribute nothing
    mu = np.array([[0.3, 0.3, 0.3], [0.3, 0.3, 0.3], [50, 50, 50], [0.3, 0.3, 0.3]], np.float32)
    sc = np.array([[0.1, 0.1, 0.1], [0.1, 0.0, 0.1], [0.1, 0.1, 0.1], [0.1, 0.1, 0.1]], np.float32)
    q = np.array([[0, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0]], np.float32)
    mu[3, 2] = np.inf
    D, occ, surf, st = run_gpu(mu, sc, q, np.ones(4, np.float32), (0, 0, 0), 0.1, (6, 6, 6), 0.5, 8)
    assert np.all(D == 0) and st["n_pairs"] == 0
    # a single-voxel grid
    mu = np.array([[0.05, 0.05, 0.05]], np.float32)
    sc = np.array([[0.1, 0.1, 0.1]], np.float32)
    q = np.array([[1, 0, 0, 0]], np.float32)
    D, occ, surf, st = run_gpu(mu, sc, q, np.ones(1, np.float32), (0, 0, 0), 0.1, (1, 1, 1), 0.5, 4)
    assert D[0, 0, 0] == pytest.approx(1.0, rel=1e-5) and occ[0, 0, 0] == 1 and surf[0, 0, 0] == 1


def test_argument_errors():
    t = torch.zeros((1, 3), device="cuda")
    q = torch.zeros((1, 4), device="cuda")
    a = torch.zeros(1, device="cuda")
    for kw in ({"tile": 5}, {"h": 0.0}, {"dims": (0, 4, 4)}, {"h": float("nan")}):
        args = dict(origin=(0, 0, 0), h=0.1, dims=(4, 4, 4))
        args.update({k: v for k, v in kw.items() if k in args})
        with pytest.raises(fgl.FglError):
            fgl.gaussian_density(t, t, q, a, args["origin"], args["h"], args["dims"],
                                 tile=kw.get("tile", 0))


def test_largest_ladder_set_sampled_tiles_vs_oracle():
    """The occupancy bench's largest set (2 M Gaussians, 330 x 280 x 180
    voxels of 2 cm, 8^3 tiles) in the bench's launch configuration: the pair
    count exact, and 64 tiles (32 at random, 32 holding occupied voxels)
    voxel by voxel against the oracle's density on those tiles."""
    from synth import gaussians, workloads
    room, nb, ns, ng, h = workloads.HETERO_LADDER[7]
    gs = gaussians.gaussian_room(4 * 100 + 7, room, ng, nb, ns)
    origin = (-0.3, -0.3, -0.3)
    dims = tuple(int(np.ceil((room[a] + 0.6) / h)) for a in range(3))
    D, occ, surf, st = run_gpu(gs.mu, gs.scale, gs.quat, gs.alpha, origin, h, dims, 0.5, 8)
    assert st["n_pairs"] == expected_pairs(gs.mu, gs.scale, gs.quat, origin, h, dims, 8)
    nt = [(d + 7) // 8 for d in dims]
    rng = np.random.default_rng(77)
    occ_tiles = np.unique(((np.nonzero(occ)[0] // 8) * nt[1] + np.nonzero(occ)[1] // 8) * nt[0]
                          + np.nonzero(occ)[2] // 8)
    tiles = np.concatenate([rng.choice(nt[0] * nt[1] * nt[2], 32, replace=False),
                            rng.choice(occ_tiles, 32, replace=False)])
    Do, Ao = oracle.density_tiles(gs.mu, gs.scale, gs.quat, gs.alpha, origin, h, dims, 8, tiles)
    for q, t in enumerate(tiles):
        a, b, c = t % nt[0], (t // nt[0]) % nt[1], t // (nt[0] * nt[1])
        g = D[c * 8:c * 8 + 8, b * 8:b * 8 + 8, a * 8:a * 8 + 8].astype(np.float64)
        o = Do[q][:g.shape[0], :g.shape[1], :g.shape[2]]
        tol = oracle.density_tolerance(o, Ao[q][:g.shape[0], :g.shape[1], :g.shape[2]])
        assert np.all(np.abs(g - o) <= tol), (int(t), float(np.max(np.abs(g - o) / tol)))
