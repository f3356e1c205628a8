"""GPU parity of the mesh-reconstruction steps (paper Sec. IV-B) against the
FP64 oracle, through the C-ABI.

Contract:
  * TSDF (fgl_tsdf): sign, shell index and phi bit-exact (integer decisions;
    phi = s min((p + 1/2) h, r) rounds once on both sides);
  * denoise (fgl_denoise): |V'_gpu - V'_oracle| <= oracle.blur_tolerance(R);
    the mask equal wherever V'_oracle is farther than that from the
    threshold; the quantile threshold is exactly the order statistic of the
    GPU's own float32 V';
  * marching tetrahedra (fgl_marching_tets): vertex and triangle counts and
    every triangle's vertex ids exact (the inside test phi < iso is exact and
    the order canonical); vertices within oracle.vertex_tolerance; normals
    within 1e-4 where the gradient is not tiny.
"""

import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

fgl = pytest.importorskip("paper_2509_17390_gb300")


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def random_binary(rng, shape, p):
    return (rng.random(shape) < p).astype(np.uint8)


def hollow_sphere(n, c, r0, r1):
    z, y, x = np.indices(n)
    d = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    return ((d >= r0) & (d < r1)).astype(np.uint8)


# -- TSDF -----------------------------------------------------------------------

TSDF_CASES = [((23, 17, 70), 0.2, 0.02, 0.05), ((9, 40, 33), 0.45, 0.03, 0.09),
              ((30, 31, 65), 0.05, 0.015, 0.06), ((1, 1, 1), 0.5, 0.1, 0.1), ((1, 5, 1), 0.5, 0.1, 0.25),
              ((7, 1, 97), 0.3, 0.01, 0.035), ((4, 6, 1100), 0.08, 0.02, 0.05)]


@pytest.mark.parametrize("shape,p,h,r", TSDF_CASES)
def test_tsdf_bit_exact(shape, p, h, r):
    rng = np.random.default_rng(sum(shape))
    V = random_binary(rng, shape, p)
    phi, out, sh, st = fgl.tsdf(cu(V), h, r, outside=True, shell=True, timing=True)
    phi_o, out_o, p_o = oracle.tsdf(V, h, r)
    assert np.array_equal(out.cpu().numpy(), out_o)
    assert np.array_equal(sh.cpu().numpy(), p_o)
    assert np.array_equal(phi.cpu().numpy().view(np.uint32), phi_o.view(np.uint32))
    assert st["n_layers"] == oracle.band_layers(h, r) and st["ms_total"] > 0


@pytest.mark.parametrize("shape,p,h,r", TSDF_CASES[:3])
def test_tsdf_literal_delta_bit_exact_and_mesh(shape, p, h, r):
    """Eq. delta read literally (p h): phi bit-exact (signed zeros included),
    and its iso = 0 marching-tetrahedra mesh equal to the oracle's."""
    rng = np.random.default_rng(sum(shape) + 1)
    V = random_binary(rng, shape, p)
    phi, _, _, _ = fgl.tsdf(cu(V), h, r, delta="literal")
    phi_o, _, _ = oracle.tsdf(V, h, r, delta="literal")
    assert np.array_equal(phi.cpu().numpy().view(np.uint32), phi_o.view(np.uint32))
    v, t, _ = fgl.marching_tets(phi, (0.0, 0.0, 0.0), h)
    torch.cuda.synchronize()
    v_o, t_o, _ = oracle.marching_tets(phi_o, (0.0, 0.0, 0.0), h)
    assert np.array_equal(t.cpu().numpy(), t_o)
    assert np.max(np.abs(v.cpu().numpy() - v_o), initial=0.0) <= oracle.vertex_tolerance(v_o, h)
    with pytest.raises(ValueError):
        fgl.tsdf(cu(V), h, r, delta="p")


def test_tsdf_cavities_and_degenerate_grids():
    V = hollow_sphere((40, 36, 45), (22.3, 17.6, 20.1), 9.0, 10.5)
    V[2:6, 2:6, 2:6] = 1
    V[3:5, 3:5, 3:5] = 0                                     # a tiny closed box: second cavity
    for grid in (V, np.ones((5, 6, 7), np.uint8), np.zeros((5, 6, 7), np.uint8)):
        phi, out, sh, _ = fgl.tsdf(cu(grid), 0.02, 0.07, outside=True, shell=True)
        phi_o, out_o, p_o = oracle.tsdf(grid, 0.02, 0.07)
        assert np.array_equal(out.cpu().numpy(), out_o)
        assert np.array_equal(sh.cpu().numpy(), p_o)
        assert np.array_equal(phi.cpu().numpy(), phi_o)
    o = fgl.tsdf(cu(V), 0.02, 0.07, outside=True)[1].cpu().numpy()
    assert o[20, 17, 22] == 0 and o[4, 4, 4] == 0 and o[0, 0, 0] == 1


def test_tsdf_large_grid_vs_oracle():
    """A 160 x 150 x 170 grid (4.1 M voxels, 5 words a row) of thin shells,
    slabs and noise: bit-exact.  (Rows longer than 32 words -- two warp
    chunks -- are in the (4, 6, 1100) case above.)"""
    rng = np.random.default_rng(77)
    shape = (170, 150, 160)
    V = hollow_sphere(shape, (80.2, 75.5, 85.3), 50.0, 51.5)
    V |= hollow_sphere(shape, (40.0, 40.0, 40.0), 20.0, 21.0)
    V[:, 100:102, :] |= 1
    V |= random_binary(rng, shape, 0.002)
    phi, out, sh, _ = fgl.tsdf(cu(V), 0.015, 0.06, outside=True, shell=True)
    phi_o, out_o, p_o = oracle.tsdf(V, 0.015, 0.06)
    assert np.array_equal(out.cpu().numpy(), out_o)
    assert np.array_equal(sh.cpu().numpy(), p_o)
    assert np.array_equal(phi.cpu().numpy(), phi_o)


# -- denoise ----------------------------------------------------------------------

@pytest.mark.parametrize("shape,sigma_vox", [((21, 30, 47), 0.5), ((12, 13, 70), 1.3), ((5, 4, 3), 2.0)])
def test_denoise_fixed_threshold(shape, sigma_vox):
    rng = np.random.default_rng(int(sigma_vox * 10))
    V = random_binary(rng, shape, 0.2)
    V[V.shape[0] // 2] = 1                                   # a plane that survives
    h = 0.02
    sigma = np.float32(sigma_vox * h)
    mask, vp, thr = fgl.denoise(cu(V), h, float(sigma), tau=0.3, blur=True)
    sv = np.float64(sigma) / np.float64(np.float32(h))
    R = oracle.blur_radius(sv)
    vp_o = oracle.blur(V, sv, R)
    tol = oracle.blur_tolerance(R)
    err = np.abs(vp.cpu().numpy().astype(np.float64) - vp_o)
    assert err.max() <= tol, (err.max(), tol)
    m_o, _ = oracle.rethreshold(vp_o, "fixed", 0.3)
    clear = np.abs(vp_o - np.float32(0.3)) > tol
    assert np.array_equal(mask.cpu().numpy()[clear], m_o[clear]) and thr == np.float32(0.3)
    # the mask follows from the GPU's own V' exactly
    assert np.array_equal(mask.cpu().numpy(), (vp.cpu().numpy() >= np.float32(0.3)).astype(np.uint8))


@pytest.mark.parametrize("q", [0.0, 0.37, 0.9, 1.0])
def test_denoise_quantile_is_the_exact_order_statistic(q):
    rng = np.random.default_rng(5)
    V = random_binary(rng, (19, 23, 41), 0.3)
    mask, vp, thr = fgl.denoise(cu(V), 0.01, 0.012, quantile=q, blur=True)
    g = vp.cpu().numpy()
    m_own, thr_own = oracle.rethreshold(g, "quantile", q)
    assert np.float32(thr) == np.float32(thr_own)
    assert np.array_equal(mask.cpu().numpy(), m_own)
    # and within the blur tolerance of the oracle's FP64 quantile
    sv = np.float64(np.float32(0.012)) / np.float64(np.float32(0.01))
    _, thr_o = oracle.rethreshold(oracle.blur(V, sv), "quantile", q)
    assert abs(thr - thr_o) <= oracle.blur_tolerance(oracle.blur_radius(sv))


# -- marching tetrahedra ----------------------------------------------------------

def check_mt(phi, origin, h, iso=0.0, step=1, normals=True):
    v, t, n = fgl.marching_tets(cu(phi), origin, h, iso=iso, step=step, normals=normals)
    vo, to, no = oracle.marching_tets(phi, origin, h, iso=iso, step=step, normals=normals)
    v, t = v.cpu().numpy(), t.cpu().numpy()
    assert v.shape == vo.shape and t.shape == to.shape
    assert np.array_equal(t, to)
    if len(v):
        assert np.max(np.abs(v - vo)) <= oracle.vertex_tolerance(vo, h * step)
    if normals and len(v):
        n = n.cpu().numpy()
        ok = np.linalg.norm(no, axis=1) > 0.5                   # unit where the oracle's gradient is nonzero
        assert np.max(np.abs(n[ok] - no[ok]), initial=0) < 1e-4
    return v, t


def sphere_phi(shape, h, c, R):
    z, y, x = np.indices(shape)
    P = np.stack([x, y, z], -1) * h + h / 2
    return (np.linalg.norm(P - c, axis=-1) - R).astype(np.float32)


@pytest.mark.parametrize("step", [1, 2, 3])
def test_marching_tets_tsdf_field(step):
    V = hollow_sphere((41, 38, 70), (35.2, 19.1, 20.4), 11.0, 12.5)
    V[10:14, :, :] = 1
    phi, _, _ = oracle.tsdf(V, 0.02, 0.06)
    v, t = check_mt(phi, (-0.3, 0.1, 0.25), 0.02, step=step)
    assert len(t) > 100


@pytest.mark.parametrize("iso", [0.0, 0.013, -0.2])
def test_marching_tets_random_and_analytic_fields(iso):
    rng = np.random.default_rng(9)
    check_mt(rng.standard_normal((13, 9, 40)).astype(np.float32), (0.0, 0.0, 0.0), 0.1, iso=iso)
    check_mt(sphere_phi((36, 40, 66), 0.03, np.array([1.0, 0.6, 0.55]), 0.45), (0.0, 0.0, 0.0), 0.03,
             iso=iso)


def test_marching_tets_edge_cases_and_capacity():
    # no crossing, a single sample, one row, a degenerate thin grid
    for phi in (np.ones((4, 5, 6), np.float32), np.ones((1, 1, 1), np.float32),
                np.linspace(-1, 1, 70, dtype=np.float32).reshape(1, 1, 70),
                np.random.default_rng(1).standard_normal((2, 1, 33)).astype(np.float32)):
        check_mt(phi, (0.0, 0.0, 0.0), 0.5, normals=False)
    # undersized buffers through the C-ABI: FGL_ERR_CAPACITY with the counts
    phi = sphere_phi((20, 20, 20), 0.1, np.array([1.0, 1.0, 1.0]), 0.6)
    d = cu(phi)
    vo, to, _ = oracle.marching_tets(phi, (0, 0, 0), 0.1)
    g = fgl.Grid((ctypes.c_float * 3)(0, 0, 0), 0.1, (ctypes.c_int32 * 3)(20, 20, 20), 0)
    vb = torch.empty((4, 3), dtype=torch.float32, device="cuda")
    tb = torch.empty((4, 3), dtype=torch.int32, device="cuda")
    nv, nt = ctypes.c_int64(), ctypes.c_int64()
    st = fgl.lib().fgl_marching_tets(ctypes.c_void_p(d.data_ptr()), ctypes.byref(g), 0.0, 1,
                                     ctypes.c_void_p(vb.data_ptr()), 4, ctypes.c_void_p(tb.data_ptr()), 4,
                                     None, ctypes.byref(nv), ctypes.byref(nt), None)
    assert st == fgl.FGL_ERR_CAPACITY and (nv.value, nt.value) == (len(vo), len(to))
    v, t, _ = fgl.marching_tets(d, (0, 0, 0), 0.1, capacity=(10, 10))   # retried at the counts
    assert np.array_equal(t.cpu().numpy(), to)
    with pytest.raises(fgl.FglError):
        fgl.marching_tets(d, (0, 0, 0), 0.1, step=0)


# -- the GPU pipeline: Gaussians -> mesh -------------------------------------------

def edge_stats(tris):
    """(every undirected edge in exactly two triangles, every directed edge in one)."""
    t = np.asarray(tris, np.int64)
    a = np.concatenate([t[:, 0], t[:, 1], t[:, 2]])
    b = np.concatenate([t[:, 1], t[:, 2], t[:, 0]])
    n = int(t.max()) + 1 if len(t) else 1
    _, cu_ = np.unique(np.minimum(a, b) * n + np.maximum(a, b), return_counts=True)
    _, cd = np.unique(a * n + b, return_counts=True)
    return bool(np.all(cu_ == 2)), bool(np.all(cd == 1))


def test_pipeline_from_gaussians_matches_oracle_steps():
    """Gaussians on a small open-topped room: the GPU's surface grid goes
    through the oracle's blur (within tolerance, mask equal away from the
    threshold), then the GPU's mask through the oracle's TSDF and marching
    tetrahedra, which the GPU pipeline's mesh matches exactly; the mesh is
    closed and consistently oriented."""
    from synth import gaussians
    gs = gaussians.gaussian_room(12, (2.0, 1.5, 1.0), 40_000, 1, 1)
    h = 0.04
    origin = (-0.6, -0.6, -0.6)                              # 3 sigma of the largest Gaussian
    dims = (int(np.ceil(3.2 / h)), int(np.ceil(2.7 / h)), int(np.ceil(2.2 / h)))
    t = lambda a: cu(a)
    D, occ, surf, _ = fgl.gaussian_density(t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha), origin, h, dims)
    S = surf.cpu().numpy()
    mask, vp, _ = fgl.denoise(surf, h, 0.5 * h, tau=0.5, blur=True)
    sv = np.float64(np.float32(0.5 * h)) / np.float64(np.float32(h))
    vp_o = oracle.blur(S, sv)
    tol = oracle.blur_tolerance(oracle.blur_radius(sv))
    assert np.abs(vp.cpu().numpy() - vp_o).max() <= tol
    M = mask.cpu().numpy()
    clear = np.abs(vp_o - 0.5) > tol
    assert np.array_equal(M[clear], oracle.rethreshold(vp_o, "fixed", 0.5)[0][clear])
    # downstream of the GPU's own mask the steps are exact
    phi_o, _, _ = oracle.tsdf(M, h, 0.06)
    vo, to, _ = oracle.marching_tets(phi_o, origin, h)
    v, tr, _ = fgl.mesh_from_gaussians(t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha), origin, h, dims,
                                       trunc=0.06)
    tr = tr.cpu().numpy()
    assert np.array_equal(tr, to)
    assert np.max(np.abs(v.cpu().numpy() - vo)) <= oracle.vertex_tolerance(vo, h)
    closed, oriented = edge_stats(tr)
    assert closed and oriented and len(tr) > 10_000


def test_fullsize_mesh_steps_vs_oracle():
    """The mesh bench's largest set (2 M Gaussians, 375 x 325 x 225 voxels of
    2 cm = 27.4 M voxels) in the bench's configuration, from the GPU's own
    surface grid: V' within the blur bound and the mask exact away from the
    threshold; the TSDF of the GPU's mask bit-exact; its marching-tetrahedra
    mesh (5 M triangles) triangle for triangle, vertices within tolerance,
    closed and consistently oriented."""
    from synth import gaussians, workloads
    room, nb, ns, ng, h = workloads.HETERO_LADDER[7]
    gs = gaussians.gaussian_room(4 * 100 + 7, room, ng, nb, ns)
    origin, dims = workloads.hetero_grid(room, h)
    t = lambda a: cu(a)
    _, _, surf, _ = fgl.gaussian_density(t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha), origin, h, dims)
    mask, vp, _ = fgl.denoise(surf, h, 0.5 * h, tau=0.5, blur=True)
    S = surf.cpu().numpy()
    sv = np.float64(np.float32(0.5 * h)) / np.float64(np.float32(h))
    vp_o = oracle.blur(S, sv)
    tol = oracle.blur_tolerance(oracle.blur_radius(sv))
    assert np.abs(vp.cpu().numpy() - vp_o).max() <= tol
    M = mask.cpu().numpy()
    clear = np.abs(vp_o - 0.5) > tol
    assert np.array_equal(M[clear], (vp_o[clear] >= 0.5).astype(np.uint8))
    del vp, vp_o, clear
    phi, _, _, _ = fgl.tsdf(mask, h, 0.06)
    phi_o, _, _ = oracle.tsdf(M, h, 0.06)
    assert np.array_equal(phi.cpu().numpy(), phi_o)
    v, tr, _ = fgl.marching_tets(phi, origin, h)
    vo, to, _ = oracle.marching_tets(phi_o, origin, h)
    tr = tr.cpu().numpy()
    assert len(to) > 4_000_000 and np.array_equal(tr, to)
    assert np.max(np.abs(v.cpu().numpy() - vo)) <= oracle.vertex_tolerance(vo, h)
    closed, oriented = edge_stats(tr)
    assert closed and oriented


@pytest.mark.parametrize("h,r", [(0.01, 0.5), (0.01, 2.535)])
def test_tsdf_wide_bands(h, r):
    """Bands of L = 51 and the maximum 254 shells (6 and 8 count planes)."""
    V = hollow_sphere((60, 70, 90), (40.3, 33.1, 28.7), 15.0, 16.0)
    V[:, 5, :] = 1
    phi, out, sh, st = fgl.tsdf(cu(V), h, r, outside=True, shell=True)
    phi_o, out_o, p_o = oracle.tsdf(V, h, r)
    assert st["n_layers"] == oracle.band_layers(h, r)
    assert np.array_equal(out.cpu().numpy(), out_o)
    assert np.array_equal(sh.cpu().numpy(), p_o)
    assert np.array_equal(phi.cpu().numpy(), phi_o)


@pytest.mark.parametrize("quantile", [None, 0.8])
def test_denoise_three_pass_path(quantile):
    """sigma of 1.7 voxels (6 taps a side): the three-pass blur, at a grid of
    several hundred thousand voxels, with a fixed and a quantile threshold."""
    rng = np.random.default_rng(8)
    V = random_binary(rng, (40, 60, 150), 0.1)
    h, sigma = 0.02, np.float32(1.7 * 0.02)
    mask, vp, thr = fgl.denoise(cu(V), h, float(sigma), tau=0.2, quantile=quantile, blur=True)
    sv = np.float64(sigma) / np.float64(np.float32(h))
    R = oracle.blur_radius(sv)
    assert R == 6
    vp_o = oracle.blur(V, sv, R)
    tol = oracle.blur_tolerance(R)
    g = vp.cpu().numpy()
    assert np.abs(g.astype(np.float64) - vp_o).max() <= tol
    if quantile is None:
        clear = np.abs(vp_o - np.float32(0.2)) > tol
        assert np.array_equal(mask.cpu().numpy()[clear], (vp_o[clear] >= np.float32(0.2)).astype(np.uint8))
    else:
        m_own, thr_own = oracle.rethreshold(g, "quantile", quantile)
        assert np.float32(thr) == np.float32(thr_own) and np.array_equal(mask.cpu().numpy(), m_own)


def test_pipeline_mc_step_two():
    """mesh_from_gaussians with mc_step 2 equals the oracle's marching
    tetrahedra at step 2 on the GPU's TSDF, and stays closed."""
    from synth import gaussians
    gs = gaussians.gaussian_room(12, (2.0, 1.5, 1.0), 30_000, 1, 1)
    h = 0.03
    origin, dims = gaussians.grid_around((0, 0, 0), (2.0, 1.5, 1.0), h, 0.6)
    t = lambda a: cu(a)
    _, _, surf, _ = fgl.gaussian_density(t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha), origin, h, dims)
    mask, _, _ = fgl.denoise(surf, h, 0.5 * h)
    phi, _, _, _ = fgl.tsdf(mask, h, 0.06)
    v2, t2, _ = fgl.mesh_from_gaussians(t(gs.mu), t(gs.scale), t(gs.quat), t(gs.alpha), origin, h, dims,
                                        step=2)
    vo, to, _ = oracle.marching_tets(phi.cpu().numpy(), origin, h, step=2)
    t2 = t2.cpu().numpy()
    assert np.array_equal(t2, to) and len(to) > 5000
    assert np.max(np.abs(v2.cpu().numpy() - vo)) <= oracle.vertex_tolerance(vo, 2 * h)
    closed, oriented = edge_stats(t2)
    assert closed and oriented


# -- tiled sign, z-marching blur, chunked mesh offsets -----------------------------

def boxes_with_corridors(shape, rng):
    """Dense noise in the low z slab (many runs a row: those row tiles take
    the global union-find path) and, above it, two hollow boxes split by
    walls every 10 rows in y, each wall open at alternating x ends, so the
    free space winds through many row tiles.  Box A has a hole in its outer
    wall (its inside is reached from the frame only along the winding
    corridor); box B is closed (its inside is not), and holds a closed cell
    of its own."""
    nz, ny, nx = shape
    V = np.zeros(shape, np.uint8)
    zs = nz // 3
    V[:zs] = (rng.random((zs, ny, nx)) < 0.45).astype(np.uint8)
    half = nx // 2
    for x0, x1, hole in ((2, half - 2, True), (half + 2, nx - 2, False)):
        z0, z1, y0, y1 = zs + 3, nz - 3, 3, ny - 3
        V[z0:z1, y0:y1, x0:x1] = 1
        V[z0 + 1:z1 - 1, y0 + 1:y1 - 1, x0 + 1:x1 - 1] = 0
        for i, yw in enumerate(range(y0 + 10, y1 - 2, 10)):
            V[z0:z1, yw, x0:x1] = 1
            xo = x0 + 2 if i % 2 == 0 else x1 - 3
            V[(z0 + z1) // 2, yw, xo] = 0                       # a one-voxel door
        if hole:
            V[(z0 + z1) // 2, y0, x0 + 2] = 0
        else:
            c = ((z0 + z1) // 2, y0 + 5, (x0 + x1) // 2)
            V[c[0] - 2:c[0] + 3, c[1] - 2:c[1] + 3, c[2] - 2:c[2] + 3] = 1
            V[c[0] - 1:c[0] + 2, c[1] - 1:c[1] + 2, c[2] - 1:c[2] + 2] = 0
    return V


@pytest.mark.parametrize("shape", [(100, 110, 200), (30, 40, 70), (14, 130, 1000)])
def test_tsdf_tiles_mixed_paths_vs_oracle(shape):
    """Row tiles of 8 x 8 (the first shape), 4 x 4 (the second; too few 8 x 8
    tiles) and rows of 32 words (the third): tiles solved in shared memory
    next to tiles on the global path, components crossing many tile faces,
    a winding corridor to the frame and a closed box: sign, shells and phi
    bit-exact."""
    rng = np.random.default_rng(shape[0])
    V = boxes_with_corridors(shape, rng)
    phi, out, sh, _ = fgl.tsdf(cu(V), 0.02, 0.05, outside=True, shell=True)
    phi_o, out_o, p_o = oracle.tsdf(V, 0.02, 0.05)
    o = out.cpu().numpy()
    assert np.array_equal(o, out_o)
    assert np.array_equal(sh.cpu().numpy(), p_o)
    assert np.array_equal(phi.cpu().numpy().view(np.uint32), phi_o.view(np.uint32))
    nz, ny, nx = shape
    zm = (nz // 3 + 3 + nz - 3) // 2
    assert o[zm, ny // 2, nx // 4] == 1 and o[zm, ny // 2, 3 * nx // 4] == 0


@pytest.mark.parametrize("sigma_vox", [0.3, 0.6, 0.9, 1.2])
def test_denoise_many_z_chunks(sigma_vox):
    """Taps R = 1..4 on 6 M voxels: the fused blur's z columns (32 planes, the
    last one ragged) within the FP64 blur's tolerance, the mask exactly
    V' >= tau of the GPU's own V'."""
    rng = np.random.default_rng(21)
    V = random_binary(rng, (100, 200, 300), 0.15)
    h = 0.02
    sigma = np.float32(sigma_vox * h)
    mask, vp, _ = fgl.denoise(cu(V), h, float(sigma), tau=0.25, blur=True)
    sv = np.float64(sigma) / np.float64(np.float32(h))
    R = oracle.blur_radius(sv)
    assert R == round(sigma_vox / 0.3)
    g = vp.cpu().numpy()
    assert np.abs(g.astype(np.float64) - oracle.blur(V, sv, R)).max() <= oracle.blur_tolerance(R)
    assert np.array_equal(mask.cpu().numpy(), (g >= np.float32(0.25)).astype(np.uint8))


@pytest.mark.parametrize("shape", [(32, 32, 128), (39, 35, 96), (1, 2049, 20), (1, 2048, 20), (3, 700, 64)])
def test_marching_tets_chunk_boundaries(shape):
    """Sample grids of 4096, 4095, 2049, 2048 and 4200 words (offsets are
    scanned in chunks of 2048 words, the end position included): triangle
    lists exact, vertices within tolerance."""
    rng = np.random.default_rng(shape[1])
    check_mt(rng.standard_normal(shape).astype(np.float32), (0.1, -0.2, 0.3), 0.05, normals=True)
