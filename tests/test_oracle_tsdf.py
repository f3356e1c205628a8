"""Pins of the mesh-reconstruction oracle (paper Sec. IV-B) against things
other than itself: scipy's Gaussian filter, connected-component labelling and
taxicab distance transform, closed forms (a single voxel's shells, a sphere's
signed distance), and topological invariants of the extracted surface
(watertight, consistently oriented, Euler characteristic 2 per sphere-like
component, enclosed volume)."""

import numpy as np
import pytest

import oracle

ndi = pytest.importorskip("scipy.ndimage")


def random_binary(rng, shape, p):
    return (rng.random(shape) < p).astype(np.uint8)


# -- eq. V' -----------------------------------------------------------------

@pytest.mark.parametrize("sigma", [0.5, 1.0, 1.7])
def test_blur_matches_scipy_gaussian_filter(sigma):
    rng = np.random.default_rng(1)
    V = random_binary(rng, (9, 11, 13), 0.3)
    R = oracle.blur_radius(sigma)
    got = oracle.blur(V, sigma)
    ref = ndi.gaussian_filter(V.astype(np.float64), sigma, mode="constant", cval=0.0, truncate=R / sigma)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_blur_brute_force_3d_sum_and_mass():
    rng = np.random.default_rng(2)
    V = random_binary(rng, (5, 6, 7), 0.4)
    sigma, R = 0.8, 3
    got = oracle.blur(V, sigma, R)
    k = np.arange(-R, R + 1)
    g = np.exp(-k ** 2 / (2 * sigma ** 2))
    g /= g.sum()
    ref = np.zeros(V.shape)
    nz, ny, nx = V.shape
    for z, y, x in zip(*np.nonzero(V)):          # scatter every set voxel's kernel
        for dz in k:
            for dy in k:
                for dx in k:
                    zz, yy, xx = z + dz, y + dy, x + dx
                    if 0 <= zz < nz and 0 <= yy < ny and 0 <= xx < nx:
                        ref[zz, yy, xx] += g[dz + R] * g[dy + R] * g[dx + R]
    assert np.max(np.abs(got - ref)) < 1e-13
    # far from the borders a single voxel keeps its unit mass
    one = np.zeros((15, 15, 15), np.uint8)
    one[7, 7, 7] = 1
    assert abs(oracle.blur(one, 1.2).sum() - 1.0) < 1e-12


def test_rethreshold_quantile_is_the_lower_order_statistic():
    rng = np.random.default_rng(3)
    Vp = rng.random((4, 5, 6))
    for q in (0.0, 0.3, 0.9, 1.0):
        Vt, thr = oracle.rethreshold(Vp, "quantile", q)
        assert thr == np.quantile(Vp, q, method="lower")
        assert np.array_equal(Vt, (Vp >= thr).astype(np.uint8))
    Vt, thr = oracle.rethreshold(Vp, "fixed", 0.5)
    assert thr == 0.5 and Vt.sum() == (Vp >= 0.5).sum()


def test_isolated_voxel_removed_plane_kept_at_half_voxel_sigma():
    """sigma = h / 2, tau = 1/2 (the pipeline's default): a lone voxel blurs
    to 0.787^3 < 1/2, a one-voxel plane keeps 0.787."""
    V = np.zeros((12, 12, 12), np.uint8)
    V[6, :, :] = 1
    V[2, 3, 3] = 1
    Vp = oracle.blur(V, 0.5)
    Vt, _ = oracle.rethreshold(Vp, "fixed", 0.5)
    assert Vt[2, 3, 3] == 0 and np.array_equal(Vt[6], np.ones((12, 12), np.uint8))
    assert Vt.sum() == 144


# -- sign: outside flood fill ---------------------------------------------------

@pytest.mark.parametrize("p", [0.25, 0.45, 0.6])
def test_outside_matches_scipy_labels(p):
    rng = np.random.default_rng(int(p * 100))
    V = random_binary(rng, (10, 12, 9), p)
    got = oracle.outside(V)
    free = np.pad(V == 0, 1, constant_values=True)           # the padded frame is free
    lab, _ = ndi.label(free, structure=ndi.generate_binary_structure(3, 1))
    frame_label = lab[0, 0, 0]
    ref = (lab == frame_label)[1:-1, 1:-1, 1:-1].astype(np.uint8)
    assert np.array_equal(got, ref)


def test_outside_enclosed_cavity_and_tunnel():
    V = np.zeros((9, 9, 9), np.uint8)
    V[2:7, 2:7, 2:7] = 1
    V[3:6, 3:6, 3:6] = 0                                      # hollow box: cavity enclosed
    out = oracle.outside(V)
    assert out[4, 4, 4] == 0 and out[0, 0, 0] == 1 and out[3:6, 3:6, 3:6].sum() == 0
    V[4, 4, 2] = 0                                            # drill a hole: cavity opens
    out = oracle.outside(V)
    assert out[4, 4, 4] == 1 and out[3:6, 3:6, 3:6].sum() == 27


# -- shells ---------------------------------------------------------------------

def test_shell_single_voxel_closed_form():
    V = np.zeros((11, 11, 11), np.uint8)
    c = 5
    V[c, c, c] = 1
    p = oracle.shell(V, 20)
    z, y, x = np.indices(V.shape)
    d1 = np.abs(z - c) + np.abs(y - c) + np.abs(x - c)
    assert np.array_equal(p, np.maximum(d1 - 1, 0).astype(np.uint8))
    p3 = oracle.shell(V, 3)
    assert np.array_equal(p3, np.where(d1 - 1 <= 3, np.maximum(d1 - 1, 0), 255).astype(np.uint8))


@pytest.mark.parametrize("seed", [0, 1])
def test_shell_matches_taxicab_distance_transform(seed):
    rng = np.random.default_rng(seed)
    V = random_binary(rng, (12, 10, 14), 0.08)
    st = ndi.generate_binary_structure(3, 1)
    Vb = V.astype(bool)
    s0 = (Vb & ~ndi.binary_erosion(Vb, st, border_value=1)) | (~Vb & ndi.binary_dilation(Vb, st))
    d = ndi.distance_transform_cdt(~s0, metric="taxicab")
    L = 4
    ref = np.where(d <= L, d, 255).astype(np.uint8)
    assert np.array_equal(oracle.shell(V, L), ref)


def test_tsdf_values_and_band():
    V = np.zeros((14, 14, 14), np.uint8)
    V[3:11, 3:11, 3:11] = 1
    V[4:10, 4:10, 4:10] = 0                                   # hollow cube, one voxel walls
    h, r = 0.02, 0.05
    phi, out, p = oracle.tsdf(V, h, r)
    assert phi.dtype == np.float32
    s = np.where(out == 1, 1.0, -1.0)
    delta = np.where(p == 255, r, (p.astype(np.float64) + 0.5) * np.float64(np.float32(h)))
    ref = (s * np.minimum(delta, np.float64(np.float32(r)))).astype(np.float32)
    assert np.array_equal(phi, ref)
    assert phi[0, 0, 0] == np.float32(0.05)                   # beyond the band: clipped to r
    assert p[7, 7, 7] == 2 and phi[7, 7, 7] == np.float32(-2.5 * np.float64(np.float32(h)))
    # wall voxels and the enclosed cavity are negative, the outside positive
    assert np.all(phi[V == 1] < 0) and np.all(phi[4:10, 4:10, 4:10] < 0) and np.all(phi[out == 1] > 0)
    assert np.all(np.abs(phi) <= np.float32(r))


def test_tsdf_literal_delta_single_voxel_closed_form():
    """Eq. delta read literally (p h): one occupied voxel gives phi = -0 on it,
    +0 on its six face neighbours (both sides of S_0 at zero) and (D - 1) h at
    taxicab distance D >= 1, clipped to r; the default reading is the same
    field moved by h/2 away from zero (-h/2 on the voxel, (D - 1/2) h around)."""
    V = np.zeros((11, 11, 11), np.uint8)
    c = 5
    V[c, c, c] = 1
    h, r = 0.01, 0.035
    z, y, x = np.indices(V.shape)
    D = (np.abs(z - c) + np.abs(y - c) + np.abs(x - c)).astype(np.float64)
    hf, rf = np.float64(np.float32(h)), np.float64(np.float32(r))
    lit, out, p = oracle.tsdf(V, h, r, delta="literal")
    ref = np.where(D == 0, -0.0, np.minimum(np.maximum(D - 1, 0) * hf, rf)).astype(np.float32)
    assert np.array_equal(lit, ref)
    assert np.signbit(lit[c, c, c]) and not np.signbit(lit[c, c, c + 1]) and lit[c, c, c + 1] == 0
    half, _, _ = oracle.tsdf(V, h, r)
    ref_h = np.where(D == 0, -0.5 * hf, np.minimum((np.maximum(D - 1, 0) + 0.5) * hf, rf)).astype(np.float32)
    assert np.array_equal(half, ref_h)
    with pytest.raises(ValueError):
        oracle.tsdf(V, h, r, delta="p")


def test_tsdf_literal_delta_surface_offset():
    """A 6-voxel-thick slab: with the literal eq. delta the iso = 0 surface
    runs through the centres of the slab's outer voxel layers, h/2 inside the
    default reading's, which lies on the slab's faces."""
    V = np.zeros((20, 12, 12), np.uint8)
    V[7:13, :, :] = 1
    h, r = 0.1, 0.35
    z_lo_face, z_hi_face = 7 * h, 13 * h              # the slab's faces (voxel k spans [k h, (k+1) h])
    for delta, lo, hi in (("half", z_lo_face, z_hi_face), ("literal", z_lo_face + h / 2, z_hi_face - h / 2)):
        phi, _, _ = oracle.tsdf(V, h, r, delta=delta)
        v, t, _ = oracle.marching_tets(phi, (0.0, 0.0, 0.0), h)
        # away from the grid's side faces the surface is the two planes
        inner = (v[:, 0] > 2 * h) & (v[:, 0] < 9 * h) & (v[:, 1] > 2 * h) & (v[:, 1] < 9 * h)
        zs = np.unique(np.round(v[inner, 2].astype(np.float64), 6))
        assert np.allclose(zs, [lo, hi], atol=1e-6), (delta, zs)


# -- isosurface -----------------------------------------------------------------

def edge_stats(tris):
    """(every undirected edge used twice, every directed edge once)."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    und = np.sort(e, axis=1)
    _, cu = np.unique(und, axis=0, return_counts=True)
    _, cd = np.unique(e, axis=0, return_counts=True)
    return bool(np.all(cu == 2)), bool(np.all(cd == 1)), len(cu)


def signed_volume(v, t):
    a, b, c = v[t[:, 0]].astype(np.float64), v[t[:, 1]].astype(np.float64), v[t[:, 2]].astype(np.float64)
    return float(np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0)


def sphere_phi(n, h, c, R):
    z, y, x = np.indices((n, n, n))
    P = np.stack([x, y, z], -1) * h + h / 2
    return (np.linalg.norm(P - c, axis=-1) - R).astype(np.float32)


def test_sphere_watertight_oriented_euler_volume_normals():
    n, h, R = 40, 0.05, 0.8
    c = np.array([1.0, 1.02, 0.97])
    phi = sphere_phi(n, h, c, R)
    v, t, nrm = oracle.marching_tets(phi, (0, 0, 0), h, normals=True)
    closed, oriented, ne = edge_stats(t)
    assert closed and oriented
    assert len(v) - ne + len(t) == 2                            # Euler characteristic of a sphere
    vol = signed_volume(v, t)
    assert abs(vol - 4 / 3 * np.pi * R ** 3) < 0.01 * 4 / 3 * np.pi * R ** 3   # outward: positive
    rad = np.linalg.norm(v - c, axis=1)
    assert np.max(np.abs(rad - R)) < 0.1 * h                    # linear interpolation of a smooth field
    radial = (v - c) / rad[:, None]
    assert np.min(np.einsum("ij,ij->i", nrm, radial)) > np.cos(np.radians(6))
    # each triangle's own normal points outwards
    a, b, cc = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    fn = np.cross(b - a, cc - a)
    assert np.all(np.einsum("ij,ij->i", fn, (a + b + cc) / 3 - c) > 0)


def test_vertices_lie_on_the_linear_zero_of_their_edge():
    """Vertex k is the k-th sign-changing edge in (sample, type) order, at the
    zero of phi's linear interpolation along that edge (enumerated here with
    numpy, edge type by edge type)."""
    rng = np.random.default_rng(5)
    phi = rng.standard_normal((6, 7, 8)).astype(np.float32)
    h, o = 0.1, np.array([0.3, -0.2, 1.0], np.float32)
    v, t, _ = oracle.marching_tets(phi, o, h)
    nz, ny, nx = phi.shape
    rows = []
    for typ in range(1, 8):
        dx, dy, dz = typ & 1, (typ >> 1) & 1, (typ >> 2) & 1
        fa = phi[:nz - dz, :ny - dy, :nx - dx].astype(np.float64)
        fb = phi[dz:, dy:, dx:].astype(np.float64)
        kz, ky, kx = np.nonzero((fa < 0) != (fb < 0))
        for z, y, x in zip(kz, ky, kx):
            rows.append(((z * ny + y) * nx + x, typ, x, y, z, dx, dy, dz, fa[z, y, x], fb[z, y, x]))
    rows.sort(key=lambda r: (r[0], r[1]))
    assert len(rows) == len(v)
    for k, (_, _, x, y, z, dx, dy, dz, fa, fb) in enumerate(rows):
        tau = -fa / (fb - fa)
        assert 0 < tau <= 1 or 0 <= tau < 1
        pa = o.astype(np.float64) + (np.array([x, y, z]) + 0.5) * np.float64(np.float32(h))
        want = pa + tau * np.array([dx, dy, dz]) * np.float64(np.float32(h))
        assert np.max(np.abs(v[k] - want)) < 1e-6
    assert len(t) > 0 and t.min() >= 0 and t.max() < len(v)


def test_random_field_closed_surface():
    """A random field forced positive on the border: the level set is closed
    and consistently oriented whatever its topology."""
    rng = np.random.default_rng(6)
    phi = rng.standard_normal((12, 13, 11)).astype(np.float32)
    phi[0], phi[-1], phi[:, 0], phi[:, -1], phi[:, :, 0], phi[:, :, -1] = 1, 1, 1, 1, 1, 1
    v, t, _ = oracle.marching_tets(phi, (0, 0, 0), 1.0)
    closed, oriented, _ = edge_stats(t)
    assert closed and oriented and len(t) > 100
    # no vertex is unused and none is duplicated
    assert np.array_equal(np.unique(t), np.arange(len(v)))
    assert len(np.unique(v, axis=0)) == len(v)


def test_all_single_cube_configurations():
    """Every sign pattern of one cube: triangles separate the inside corners
    from the outside ones, counts follow the six tetrahedra, and the cube's
    surface is closed except on the cube's faces."""
    tets = [(0, 1, 3, 7), (0, 1, 5, 7), (0, 2, 3, 7), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 6, 7)]
    for cfg in range(256):
        phi = np.empty((2, 2, 2), np.float32)
        for c in range(8):
            phi[(c >> 2) & 1, (c >> 1) & 1, c & 1] = -1.0 if (cfg >> c) & 1 else 1.0
        v, t, _ = oracle.marching_tets(phi, (0, 0, 0), 1.0)
        inside = [(cfg >> c) & 1 for c in range(8)]
        want = 0
        for T in tets:
            k = sum(inside[c] for c in T)
            want += {0: 0, 1: 1, 2: 2, 3: 1, 4: 0}[k]
        assert len(t) == want, cfg
        ctr = lambda c: np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], np.float64) + 0.5
        ins = [ctr(c) for c in range(8) if inside[c]]
        outs = [ctr(c) for c in range(8) if not inside[c]]
        for tri in t:
            a, b, c = v[tri].astype(np.float64)
            fn = np.cross(b - a, c - a)
            assert np.linalg.norm(fn) > 0
            # inside corners on the back side of some triangle of theirs
        if ins and outs:
            # with +-1 corners every vertex is an edge midpoint
            assert np.allclose((v - 0.5) * 2 % 1, 0)
        if len(t):
            e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
            _, cd = np.unique(e, axis=0, return_counts=True)
            assert np.all(cd == 1), cfg                         # no directed edge twice


def test_orientation_matches_a_signed_distance():
    """Triangles of a plane phi = x - x0: every normal is +x."""
    z, y, x = np.indices((5, 6, 7))
    phi = (x + 0.5 - 3.3).astype(np.float32)
    v, t, _ = oracle.marching_tets(phi, (0, 0, 0), 1.0)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    fn = np.cross(b - a, c - a)
    assert np.all(fn[:, 0] > 0) and np.allclose(fn[:, 1:], 0, atol=1e-6)
    assert np.allclose(v[:, 0], 3.3, atol=1e-6)


def test_step_equals_subsampled_grid():
    n, h = 33, 0.04
    phi = sphere_phi(n, h, np.array([0.66, 0.6, 0.7]), 0.45)
    o = np.array([0.1, 0.2, -0.3], np.float32)
    v2, t2, _ = oracle.marching_tets(phi, o, h, step=2)
    vs, ts, _ = oracle.marching_tets(phi[::2, ::2, ::2], o - np.float32(h / 2), 2 * h)
    assert np.array_equal(t2, ts)
    assert np.max(np.abs(v2 - vs)) < 1e-6
    assert edge_stats(t2)[:2] == (True, True)


def test_hollow_shell_pipeline_gives_one_outer_surface():
    """A closed one-voxel shell around an enclosed cavity: the cavity is
    inside (s = -1), so only the outer surface is extracted -- one closed,
    outward-oriented sphere-like component."""
    n = 30
    z, y, x = np.indices((n, n, n))
    d = np.sqrt((x - 14.7) ** 2 + (y - 15.2) ** 2 + (z - 14.9) ** 2)
    V = ((d >= 8.0) & (d < 9.0)).astype(np.uint8)
    outside = oracle.outside(V)
    assert np.all(outside[d < 8.0] == 0)
    phi, _, _ = oracle.tsdf(V, 0.01, 0.04)
    v, t, _ = oracle.marching_tets(phi, (0, 0, 0), 0.01)
    closed, oriented, ne = edge_stats(t)
    assert closed and oriented and len(v) - ne + len(t) == 2
    assert signed_volume(v, t) > 0
    rad = np.linalg.norm(v - np.array([14.7, 15.2, 14.9]) * 0.01 - 0.005, axis=1)
    # one component (Euler 2, not 4 for two nested spheres), around the shell's
    # outer face at 9 voxels (staircase: within a voxel diagonal)
    assert rad.min() > 7.9 * 0.01 and rad.max() < 10.0 * 0.01


# -- the whole oracle pipeline from Gaussians (Sec. IV-A then IV-B) ---------------

def test_pipeline_single_gaussian_gives_its_level_ball():
    """One isotropic Gaussian (sigma s, alpha 1): D(x) = exp(-|x|^2 / (2 s^2))
    exceeds theta inside the ball of radius s sqrt(2 ln(1/theta)).  The mesh
    wraps that ball's one-voxel surface shell: a closed sphere-like surface
    within a voxel and a half of the radius, with or without the denoising."""
    from synth.gaussians import grid_around
    s, theta, h = 0.1, 0.5, 0.01
    R = s * np.sqrt(2 * np.log(1 / theta))
    origin, dims = grid_around((0, 0, 0), (0, 0, 0), h, 0.2)
    one = lambda a: np.asarray(a, np.float32).reshape(1, -1)
    for sigma in (None, "half-voxel"):
        v, t = oracle.mesh_from_gaussians(one([0, 0, 0]), one([s, s, s]), one([1, 0, 0, 0]), one([1.0]),
                                          origin, h, dims, theta=theta, trunc=0.03, sigma=sigma)
        r = np.linalg.norm(v, axis=1)
        assert abs(np.median(r) - R) < 1.5 * h and r.max() - r.min() < 3 * h
        closed, oriented, ne = edge_stats(t)
        assert closed and oriented and len(v) - ne + len(t) == 2


def test_pipeline_closed_shell_of_gaussians_keeps_its_cavity_inside():
    """Gaussians on a closed sphere of radius 0.5 m: the flood fill never
    reaches the inside, so the mesh is one outward surface just outside the
    shell (no inner surface)."""
    from synth.gaussians import grid_around
    rng = np.random.default_rng(1)
    n = 30_000
    p = rng.standard_normal((n, 3))
    p = 0.5 * p / np.linalg.norm(p, axis=1, keepdims=True)
    origin, dims = grid_around((-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), 0.02, 0.25)
    v, t = oracle.mesh_from_gaussians(p.astype(np.float32), np.full((n, 3), 0.03, np.float32),
                                      np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                                      np.ones(n, np.float32), origin, 0.02, dims, theta=0.5)
    r = np.linalg.norm(v, axis=1)
    assert r.min() > 0.5 and r.max() < 0.62
    closed, oriented, ne = edge_stats(t)
    assert closed and oriented and len(v) - ne + len(t) == 2 and signed_volume(v, t) > 0
