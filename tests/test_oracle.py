"""Pins for the FP64 oracle against things other than itself.

Each pin targets a plausible mistake: closed forms (wrong sign/axis, wrong t
formula), an independent textbook intersection routine (Moller-Trumbore) on
tiny scenes (dropped term, wrong edge test), BVH vs brute force (bad
pruning), invariants (transposed operand in ray generation, hit point off
the triangle), and hand-built ambiguous cases (flags).
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# independent brute force: Moller & Trumbore (1997), FP64, vectorised numpy
# ---------------------------------------------------------------------------
def mt_nearest(verts, tris, o, d, max_range, min_range=0.0):
    v = verts.astype(np.float64)[tris.astype(np.int64)]          # [nt,3,3]
    o = o.astype(np.float64)
    d = d.astype(np.float64)
    e1 = v[:, 1] - v[:, 0]
    e2 = v[:, 2] - v[:, 0]
    out_t = np.full(len(o), float(max_range))
    out_id = np.full(len(o), -1, np.int64)
    for i in range(len(o)):
        p = np.cross(d[i][None], e2)
        det = np.einsum("ij,ij->i", e1, p)
        ok = det != 0
        inv = np.where(ok, 1.0 / np.where(ok, det, 1.0), 0.0)
        s = o[i][None] - v[:, 0]
        u = np.einsum("ij,ij->i", s, p) * inv
        q = np.cross(s, e1)
        w = np.einsum("j,ij->i", d[i], q) * inv
        t = np.einsum("ij,ij->i", e2, q) * inv
        hit = ok & (u >= 0) & (w >= 0) & (u + w <= 1) & (t > 0) & (t >= min_range) & (t <= max_range)
        if hit.any():
            tt = np.where(hit, t, np.inf)
            m = tt.min()
            k = np.nonzero(tt == m)[0].min()
            out_t[i], out_id[i] = m, k
    return out_t, out_id


def random_soup(rng, n_tris, extent=10.0, size_lo=0.02, size_hi=2.0):
    c = rng.uniform(0, extent, (n_tris, 1, 3))
    s = np.exp(rng.uniform(np.log(size_lo), np.log(size_hi), (n_tris, 1, 1)))
    v = (c + s * rng.standard_normal((n_tris, 3, 3))).reshape(-1, 3).astype(np.float32)
    t = np.arange(3 * n_tris, dtype=np.int32).reshape(-1, 3)
    return v, t


def random_rays(rng, n, lo=0.0, hi=10.0):
    o = rng.uniform(lo, hi, (n, 3)).astype(np.float32)
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return o, d.astype(np.float32)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------
def test_golden_box_room_closed_form():
    g = json.load(open(os.path.join(GOLDEN, "box_room_closed_form.json")))
    v, t = synth.box_room(g["room"])
    for bvh in (False, True):
        sc = oracle.Scene(v, t, bvh=bvh)
        for case in g["cases"]:
            o = np.array([g["origin"]], np.float32)
            d = np.array([case["d"]], np.float32)
            rng, ids, fl = sc.cast(o, d, case["max_range"])
            assert rng[0] == case["t"], case
            if case["wall"] is None:
                assert ids[0] == -1
            else:
                axis, val = case["wall"]
                tv = v[t[ids[0]]]
                assert np.all(tv[:, axis] == val), (case, tv)


def test_box_room_random_rays_closed_form():
    rng = np.random.default_rng(11)
    L = np.array([10.0, 8.0, 3.0])
    v, t = synth.box_room(L)
    sc = oracle.Scene(v, t, bvh=False)
    o = (0.1 + rng.uniform(0, 1, (4000, 3)) * (L - 0.2)).astype(np.float32)
    d = rng.standard_normal((4000, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r, ids, fl = sc.cast(o, d, 1000.0)
    od, dd = o.astype(np.float64), d.astype(np.float64)
    with np.errstate(divide="ignore"):
        tb = np.where(dd > 0, (L - od) / dd, np.where(dd < 0, -od / dd, np.inf))
    cf = tb.min(axis=1)
    assert np.all(ids >= 0)
    np.testing.assert_allclose(r, cf, rtol=1e-12, atol=0)
    # the hit triangle lies on the wall of the minimising axis
    ax = tb.argmin(axis=1)
    side = np.where(dd[np.arange(len(d)), ax] > 0, L[ax], 0.0)
    tv = v[t[ids]]
    assert np.all(tv[np.arange(len(d)), :, ax] == side[:, None])


def test_plane_quad_closed_form():
    rng = np.random.default_rng(3)
    h = float(np.float32(1.7))            # the plane height as stored in float32
    v = np.array([[-50, -50, h], [50, -50, h], [50, 50, h], [-50, 50, h]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    sc = oracle.Scene(v, t, bvh=True)
    o = np.c_[rng.uniform(-5, 5, (2000, 2)), rng.uniform(-3, 1.5, 2000)].astype(np.float32)
    d = rng.standard_normal((2000, 3))
    d[:, 2] = np.abs(d[:, 2]) + 1.0
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    cf = (h - o[:, 2].astype(np.float64)) / d[:, 2].astype(np.float64)
    p = o.astype(np.float64) + cf[:, None] * d.astype(np.float64)
    keep = np.all(np.abs(p[:, :2]) < 49.0, axis=1)       # lands well inside the quad
    o, d, cf = o[keep], d[keep], cf[keep]
    r, ids, fl = sc.cast(o, d, 500.0)
    assert np.all(ids >= 0)
    np.testing.assert_allclose(r, cf, rtol=1e-12)
    # rays going down miss, and report (max_range, -1)
    r2, i2, _ = sc.cast(o, -d, 500.0)
    assert np.all(i2 == -1) and np.all(r2 == 500.0)


def test_icosphere_from_centre_within_sagitta_bound():
    level, radius = 2, 0.75
    uv, ut = synth.icosphere_unit(level)
    c = np.array([1.0, -2.0, 0.5])
    v = (c + radius * uv).astype(np.float32)
    sc = oracle.Scene(v, ut, bvh=True)
    # largest angular circumradius of a face bounds the face's depth below the sphere
    tri = uv[ut]
    cen = tri.mean(axis=1)
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    cosmin = np.min(np.einsum("fj,fkj->fk", cen, tri))
    rng = np.random.default_rng(5)
    d = rng.standard_normal((5000, 3))
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    o = np.tile(c.astype(np.float32), (5000, 1))
    r, ids, fl = sc.cast(o, d, 10.0)
    assert np.all(ids >= 0)
    assert np.all(r <= radius * (1 + 1e-6) + 1e-6)
    assert np.all(r >= radius * cosmin * (1 - 1e-6))


def test_icosphere_from_outside_against_analytic_sphere():
    level, radius = 3, 1.0
    uv, ut = synth.icosphere_unit(level)
    v = (radius * uv).astype(np.float32)
    sc = oracle.Scene(v, ut, bvh=True)
    rng = np.random.default_rng(9)
    n = 3000
    o = rng.standard_normal((n, 3))
    o = (4.0 * o / np.linalg.norm(o, axis=1, keepdims=True)).astype(np.float32)
    # aim at points within 0.5 of the centre so the incidence stays steep
    tgt = 0.5 * rng.uniform(-1, 1, (n, 3)) / np.sqrt(3)
    d = tgt - o
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    r, ids, _ = sc.cast(o, d, 100.0)
    od, dd = o.astype(np.float64), d.astype(np.float64)
    b = np.einsum("ij,ij->i", od, dd)
    cc = np.einsum("ij,ij->i", od, od) - radius ** 2
    ts = -b - np.sqrt(b * b - cc)                       # analytic entry
    cos_inc = np.abs(np.einsum("ij,ij->i", dd, (od + ts[:, None] * dd) / radius))
    tri = uv[ut]
    cen = tri.mean(axis=1)
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    sag = radius * (1 - np.min(np.einsum("fj,fkj->fk", cen, tri)))
    assert np.all(ids >= 0)
    assert np.all(r >= ts - 1e-9)                      # polyhedron lies inside the sphere
    assert np.all(r - ts <= sag / cos_inc + 1e-9)


# ---------------------------------------------------------------------------
# brute force against an independent routine, BVH against brute force
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_matches_moller_trumbore(seed):
    rng = np.random.default_rng(seed)
    v, t = random_soup(rng, 60)
    o, d = random_rays(rng, 400)
    sc = oracle.Scene(v, t, bvh=False)
    r, ids, fl = sc.cast(o, d, 30.0)
    mr, mid = mt_nearest(v, t, o, d, 30.0)
    unflagged = fl == 0
    assert unflagged.mean() > 0.95
    assert np.array_equal(ids[unflagged], mid[unflagged])
    np.testing.assert_allclose(r[unflagged], mr[unflagged], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("seed", [0, 1])
def test_bvh_bit_identical_to_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    v, t = random_soup(rng, 3000, size_lo=0.01, size_hi=1.0)
    o, d = random_rays(rng, 3000)
    a = oracle.Scene(v, t, bvh=False).cast(o, d, 25.0)
    b = oracle.Scene(v, t, bvh=True).cast(o, d, 25.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------------------
# minimum range t_min (eq. t_j*: intersections outside [t_min, t_max] are
# discarded; a surface nearer than t_min is passed through)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("bvh", [False, True])
def test_min_range_closed_form_box(bvh):
    """Rays along +x from x = -1 through the closed box [0,1]^3: entry face at
    t = 1, exit face at t = 2.  t_min <= 1 returns the entry face (t_min = 1
    inclusive), 1 < t_min <= 2 the exit face, t_min > 2 a miss."""
    v, t = synth.aabb_box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 2)
    sc = oracle.Scene(v, t, bvh=bvh)
    rng = np.random.default_rng(5)
    yz = rng.uniform(0.05, 0.95, (200, 2))
    o = np.concatenate([np.full((200, 1), -1.0), yz], 1).astype(np.float32)
    d = np.tile(np.array([[1.0, 0.0, 0.0]], np.float32), (200, 1))
    for tmin, want, plane in ((0.0, 1.0, 0.0), (0.5, 1.0, 0.0), (1.0, 1.0, 0.0), (1.5, 2.0, 1.0),
                              (2.0, 2.0, 1.0), (2.5, None, None)):
        r, ids, fl = sc.cast(o, d, 10.0, min_range=tmin)
        if want is None:
            assert np.all(ids == -1) and np.all(r == 10.0)
            continue
        assert np.all(r == want), tmin
        assert np.all(v[t[ids]][:, :, 0] == plane), tmin               # the hit lies on that face
        if tmin == want:
            assert np.all(fl & oracle.FLAG_RANGE)                      # hit exactly at t_min


@pytest.mark.parametrize("seed", [0, 1])
def test_min_range_bvh_equals_brute_force_and_moller_trumbore(seed):
    rng = np.random.default_rng(300 + seed)
    v, t = random_soup(rng, 600, size_lo=0.05, size_hi=1.5)
    o, d = random_rays(rng, 500)
    for tmin in (0.0, 0.7, 3.0):
        a = oracle.Scene(v, t, bvh=False).cast(o, d, 25.0, min_range=tmin)
        b = oracle.Scene(v, t, bvh=True).cast(o, d, 25.0, min_range=tmin)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
        r, ids, fl = a
        mr, mi = mt_nearest(v, t, o, d, 25.0, min_range=tmin)
        unflagged = fl == 0
        assert np.array_equal(ids[unflagged], mi[unflagged]), tmin
        np.testing.assert_allclose(r[unflagged], mr[unflagged], rtol=1e-9, atol=1e-12)
        if tmin > 0:
            assert np.all(r[ids >= 0] >= tmin)
            # without t_min the same rays return something at least as near
            r0, i0, _ = oracle.Scene(v, t, bvh=True).cast(o, d, 25.0)
            assert np.all(r0 <= r)


def test_min_range_validator():
    """The plausibility check honours t_min: the exit face is a valid answer
    for t_min between the faces, the entry face is not."""
    v, t = synth.aabb_box((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), 1)
    sc = oracle.Scene(v, t)
    o = np.array([[-1.0, 0.3, 0.6]], np.float32)
    d = np.array([[1.0, 0.0, 0.0]], np.float32)
    r, ids, _ = sc.cast(o, d, 10.0, min_range=1.5)
    r0, i0, _ = sc.cast(o, d, 10.0)
    assert sc.validate(o, d, 10.0, r.astype(np.float32), ids, min_range=1.5)[0]
    assert not sc.validate(o, d, 10.0, r0.astype(np.float32), i0, min_range=1.5)[0]
    assert not sc.validate(o, d, 10.0, r.astype(np.float32), ids)[0]        # skipped the entry face


def test_bvh_bit_identical_on_tiny_room_workload():
    v, t, obs = synth.tiny_room_scene(1)
    P = synth.sample_free_pose(np.random.default_rng(2), obs, 3)
    s = synth.grid_sensor(16, -15, 15, 360)
    o, d = oracle.world_rays(oracle.sensor_dirs(s.elev, s.azim), P)
    a = oracle.Scene(v, t, bvh=False).cast(o, d, 100.0)
    b = oracle.Scene(v, t, bvh=True).cast(o, d, 100.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


# ---------------------------------------------------------------------------
# ray generation (eq. r_j)
# ---------------------------------------------------------------------------
def test_sensor_dirs_closed_form():
    el = np.array([0.0, 0.0, np.pi / 2, -np.pi / 2, 0.0], np.float32)
    az = np.array([0.0, np.pi, 0.0, 0.0, np.pi / 2], np.float32)
    d = oracle.sensor_dirs(el, az).astype(np.float64)
    ref = np.array([[1, 0, 0], [-1, 0, 0], [0, 0, 1], [0, 0, -1], [0, 1, 0]], np.float64)
    np.testing.assert_allclose(d, ref, atol=1e-7)
    # unit length within float32 rounding, and elevation/azimuth recovered
    s = synth.grid_sensor(32, -16, 15, 1800)
    d = oracle.sensor_dirs(s.elev, s.azim).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), 1.0, atol=2e-7)
    np.testing.assert_allclose(np.arcsin(d[:, 2]), s.elev, atol=1e-6)
    az = np.mod(np.arctan2(d[:, 1], d[:, 0]), 2 * np.pi)
    err = np.abs(np.angle(np.exp(1j * (az - s.azim))))
    assert err.max() < 1e-6


def test_world_rays_pose_closed_forms():
    s = synth.grid_sensor(4, -10, 10, 16)
    dirs = oracle.sensor_dirs(s.elev, s.azim)
    ident = np.zeros((1, 3, 4), np.float32)
    ident[0, :, :3] = np.eye(3)
    ident[0, :, 3] = [1.5, -2.0, 0.25]
    o, d = oracle.world_rays(dirs, ident)
    assert np.array_equal(d, dirs) and np.all(o == ident[0, :, 3])
    rz = np.zeros((1, 3, 4), np.float32)
    rz[0, :, :3] = [[0, -1, 0], [1, 0, 0], [0, 0, 1]]      # +90 deg about z
    o, d = oracle.world_rays(dirs, rz)
    assert np.array_equal(d, np.stack([-dirs[:, 1], dirs[:, 0], dirs[:, 2]], 1))
    # general pose: d_w = R d within float32 rounding, and env-major layout
    P = synth.sample_free_pose(np.random.default_rng(1), synth.tiny_room_scene(0)[2], 3, upright=False)
    o, d = oracle.world_rays(dirs, P)
    ref = np.einsum("eij,rj->eri", P[:, :, :3].astype(np.float64), dirs.astype(np.float64)).reshape(-1, 3)
    np.testing.assert_allclose(d, ref, atol=3e-7)
    assert np.array_equal(o, np.repeat(P[:, :, 3], len(dirs), axis=0))


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------
def test_range_bound_and_hit_point_on_triangle():
    v, t, obs = synth.tiny_room_scene(4)
    P = synth.sample_free_pose(np.random.default_rng(8), obs, 4, upright=False)
    s = synth.grid_sensor(16, -15, 15, 360)
    o, d = oracle.world_rays(oracle.sensor_dirs(s.elev, s.azim), P)
    R = 6.0
    r, ids, fl = oracle.Scene(v, t).cast(o, d, R)
    assert np.all(r <= R)
    miss = ids < 0
    assert np.all(r[miss] == R) and miss.any() and (~miss).any()
    h = ~miss
    p = o[h].astype(np.float64) + r[h, None] * d[h].astype(np.float64)
    tv = v[t[ids[h]]].astype(np.float64)
    # barycentric coordinates by an independent least-squares solve
    M = np.stack([tv[:, 1] - tv[:, 0], tv[:, 2] - tv[:, 0]], axis=2)
    rhs = p - tv[:, 0]
    sol = np.stack([np.linalg.lstsq(M[i], rhs[i], rcond=None)[0] for i in range(len(M))])
    b1, b2 = sol[:, 0], sol[:, 1]
    assert np.all(b1 >= -1e-9) and np.all(b2 >= -1e-9) and np.all(b1 + b2 <= 1 + 1e-9)
    resid = np.linalg.norm(np.einsum("nij,nj->ni", M, sol) - rhs, axis=1)
    assert resid.max() < 1e-9


def _rz90(x):
    return np.stack([-x[..., 1], x[..., 0], x[..., 2]], axis=-1)


@pytest.mark.parametrize("bvh", [False, True])
def test_exact_rigid_transform_leaves_ranges_bit_identical(bvh):
    # vertices and origins on a 2^-10 grid: +90 deg about z and a translation
    # by (8, -16, 4) are exact in float32, so the oracle must agree bit for bit
    rng = np.random.default_rng(21)
    v, t, obs = synth.tiny_room_scene(6)
    v = (np.round(v * 1024) / 1024).astype(np.float32)
    P = synth.sample_free_pose(rng, obs, 2, upright=False)
    P[:, :, 3] = np.round(P[:, :, 3] * 1024) / 1024
    s = synth.grid_sensor(16, -15, 15, 90)
    dirs = oracle.sensor_dirs(s.elev, s.azim)
    T = np.array([8.0, -16.0, 4.0], np.float32)
    v2 = (_rz90(v) + T).astype(np.float32)
    P2 = P.copy()
    P2[:, :, :3] = np.stack([-P[:, 1, :3], P[:, 0, :3], P[:, 2, :3]], axis=1)
    P2[:, :, 3] = _rz90(P[:, :, 3]) + T
    o1, d1 = oracle.world_rays(dirs, P)
    o2, d2 = oracle.world_rays(dirs, P2)
    assert np.array_equal(d2, _rz90(d1))
    r1, i1, _ = oracle.Scene(v, t, bvh).cast(o1, d1, 100.0)
    r2, i2, _ = oracle.Scene(v2, t, bvh).cast(o2, d2, 100.0)
    assert np.array_equal(r1, r2) and np.array_equal(i1, i2)


def test_random_rigid_transform_within_tolerance():
    rng = np.random.default_rng(22)
    v, t, obs = synth.tiny_room_scene(7)
    P = synth.sample_free_pose(rng, obs, 2, upright=False)
    s = synth.grid_sensor(16, -15, 15, 180)
    dirs = oracle.sensor_dirs(s.elev, s.azim)
    Q = synth.random_rotation(rng, 1)[0]
    T = rng.uniform(-50, 50, 3)
    v2 = (v.astype(np.float64) @ Q.T + T).astype(np.float32)
    P2 = P.astype(np.float64).copy()
    P2[:, :, :3] = np.einsum("ij,ejk->eik", Q, P[:, :, :3].astype(np.float64))
    P2[:, :, 3] = P[:, :, 3].astype(np.float64) @ Q.T + T
    o1, d1 = oracle.world_rays(dirs, P)
    o2, d2 = oracle.world_rays(dirs, P2.astype(np.float32))
    r1, i1, f1 = oracle.Scene(v, t).cast(o1, d1, 100.0)
    r2, i2, f2 = oracle.Scene(v2, t).cast(o2, d2, 100.0)
    ok = (f1 == 0) & (f2 == 0)
    assert ok.mean() > 0.99
    assert np.array_equal(i1[ok], i2[ok])
    assert np.all(np.abs(r1[ok] - r2[ok]) <= 1e-4 + 1e-6 * r1[ok])


# ---------------------------------------------------------------------------
# flags on hand-built ambiguous cases
# ---------------------------------------------------------------------------
QUAD_V = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], np.float32)
QUAD_T = np.array([[0, 1, 2], [0, 2, 3]], np.int32)


def _cast1(v, t, o, d, R=10.0, bvh=False):
    r, i, f = oracle.Scene(v, t, bvh).cast(np.array([o], np.float32), np.array([d], np.float32), R)
    return r[0], i[0], f[0]


@pytest.mark.parametrize("bvh", [False, True])
def test_flag_shared_edge(bvh):
    r, i, f = _cast1(QUAD_V, QUAD_T, [0.5, 0.5, 1.0], [0, 0, -1], bvh=bvh)
    assert r == 1.0 and i == 0                      # tie goes to the smaller id
    assert f & oracle.FLAG_EDGE and f & oracle.FLAG_TIE


@pytest.mark.parametrize("bvh", [False, True])
def test_flag_interior_hit_unflagged(bvh):
    r, i, f = _cast1(QUAD_V, QUAD_T, [0.7, 0.2, 1.0], [0, 0, -1], bvh=bvh)
    assert r == 1.0 and i == 0 and f == 0
    r, i, f = _cast1(QUAD_V, QUAD_T, [0.2, 0.7, 2.0], [0, 0, -1], bvh=bvh)
    assert r == 2.0 and i == 1 and f == 0


def test_flag_range_boundary():
    r, i, f = _cast1(QUAD_V, QUAD_T, [0.2, 0.7, 2.0], [0, 0, -1], R=2.0)
    assert r == 2.0 and i == 1 and f & oracle.FLAG_RANGE
    r, i, f = _cast1(QUAD_V, QUAD_T, [0.2, 0.7, 2.0], [0, 0, -1], R=1.99995)
    assert i == -1 and f & oracle.FLAG_RANGE
    r, i, f = _cast1(QUAD_V, QUAD_T, [0.2, 0.7, 2.0], [0, 0, -1], R=1.9)
    assert i == -1 and f == 0


def test_flag_coplanar_duplicate():
    t = np.array([[0, 1, 2], [0, 1, 2]], np.int32)
    r, i, f = _cast1(QUAD_V, t, [0.7, 0.2, 1.0], [0, 0, -1])
    assert r == 1.0 and i == 0 and f & oracle.FLAG_TIE and not f & oracle.FLAG_EDGE


def test_flag_near_edge_miss_and_vertex():
    # passes one float32 ulp outside triangle 0's side x=1
    x = float(np.nextafter(np.float32(1.0), np.float32(2.0)))
    r, i, f = _cast1(QUAD_V[:3], QUAD_T[:1], [x, 0.5, 1.0], [0, 0, -1])
    assert i == -1 and f & oracle.FLAG_EDGE
    r, i, f = _cast1(QUAD_V[:3], QUAD_T[:1], [1.01, 0.5, 1.0], [0, 0, -1])
    assert i == -1 and f == 0
    r, i, f = _cast1(QUAD_V, QUAD_T, [1.0, 1.0, 1.0], [0, 0, -1])
    assert i == 0 and f & oracle.FLAG_EDGE


def test_flag_grazing_ray_in_plane():
    # ray in the quad's plane crossing its interior: edges at distance 0
    r, i, f = _cast1(QUAD_V, QUAD_T, [-1.0, 0.3, 0.0], [1, 0, 0])
    assert f & oracle.FLAG_EDGE


# ---------------------------------------------------------------------------
# validator: accepts correct answers, rejects planted mistakes
# ---------------------------------------------------------------------------
def test_validate_accepts_oracle_and_rejects_mistakes():
    v, t, obs = synth.tiny_room_scene(3)
    P = synth.sample_free_pose(np.random.default_rng(4), obs, 2)
    s = synth.grid_sensor(16, -15, 15, 360)
    o, d = oracle.world_rays(oracle.sensor_dirs(s.elev, s.azim), P)
    sc = oracle.Scene(v, t)
    r, ids, fl = sc.cast(o, d, 100.0)
    assert sc.validate(o, d, 100.0, r.astype(np.float32), ids).all()
    # range off by 1 cm
    assert not sc.validate(o, d, 100.0, (r + 0.01).astype(np.float32), ids).any()
    # claiming a miss where a definite hit exists
    miss_r = np.full(len(r), 100.0, np.float32)
    assert not sc.validate(o, d, 100.0, miss_r, np.full(len(r), -1, np.int32)).any()
    # reporting the far wall behind a box: pick rays whose nearest hit is a box
    # triangle (ids >= 12) and claim the room wall behind it instead
    box = (ids >= 12) & (fl == 0)
    assert box.any()
    far_r, far_i, _ = oracle.Scene(v[:8], t[:12]).cast(o[box], d[box], 100.0)
    assert not sc.validate(o[box], d[box], 100.0, far_r.astype(np.float32), far_i).any()


# ---------------------------------------------------------------------------
# per-environment rigid instances
# ---------------------------------------------------------------------------
def _rot_z(deg):
    a = np.deg2rad(deg)
    return np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])


def test_instance_rays_identity_and_closed_form():
    rng = np.random.default_rng(21)
    o, d = random_rays(rng, 50)
    P = np.tile(np.hstack([np.eye(3), np.zeros((3, 1))]).reshape(1, 12), (50, 1)).astype(np.float32)
    lo, ld = oracle.instance_rays(o, d, P)
    assert np.array_equal(lo, o) and np.array_equal(ld, d)
    # a unit box turned 90 degrees about z and moved to (5, 2, 0): rays along +x at height 0.5
    v, t = synth.aabb_box((0, 0, 0), (1, 1, 1), 1)
    box = oracle.Scene(v, t, bvh=False)
    pose = np.hstack([np.round(_rot_z(90), 12), [[5.0], [2.0], [0.0]]]).astype(np.float32)
    # in the world the box occupies x in [4, 5], y in [2, 3]
    o = np.array([[0.0, 2.25, 0.5], [0.0, 2.75, 0.25], [0.0, 3.5, 0.5]], np.float32)
    d = np.tile(np.array([[1.0, 0.0, 0.0]], np.float32), (3, 1))
    lo, ld = oracle.instance_rays(o, d, np.tile(pose.reshape(1, 12), (3, 1)))
    r, ids, _ = box.cast(lo, ld, 100.0)
    assert r[0] == 4.0 and r[1] == 4.0 and ids[2] == -1


def test_instances_match_the_union_mesh_moved_in_fp64():
    """Casting each instance in its own frame agrees with casting one mesh
    made of the scene and the instances' vertices moved into the world."""
    rng = np.random.default_rng(22)
    vs, ts, obs = synth.tiny_room_scene(3)
    uv, ut = synth.icosphere_unit(2)
    sphere_v, sphere_t = (0.4 * uv).astype(np.float32), ut
    box_v, box_t = synth.aabb_box((-0.3, -0.2, -0.25), (0.3, 0.2, 0.25), 2)
    inst_mesh = [(sphere_v, sphere_t), (box_v, box_t)]
    n_env, R = 3, 100.0
    P = synth.sample_free_pose(rng, obs, n_env)
    tab = synth.grid_sensor(8, -10, 10, 90)
    dirs = oracle.sensor_dirs(tab.elev, tab.azim)
    o, d = oracle.world_rays(dirs, P)
    IP = np.zeros((n_env, 2, 3, 4), np.float32)
    for e in range(n_env):
        for k in range(2):
            IP[e, k, :, :3] = _rot_z(rng.uniform(0, 360))
            IP[e, k, :, 3] = P[e, :, 3] + rng.uniform(-2, 2, 3) * [1, 1, 0.3] + [0, 0, 0.2]
    r, ids, inst, fl = oracle.cast_with_instances(oracle.Scene(vs, ts), [oracle.Scene(*m) for m in inst_mesh],
                                                  o, d, IP, tab.n_rays, R)
    assert (inst >= 0).sum() > 20                           # the instances are seen
    for e in range(n_env):
        parts_v, parts_t, base, offs = [vs.astype(np.float64)], [ts], len(vs), [0]
        for k, (mv, mt) in enumerate(inst_mesh):
            wv = mv.astype(np.float64) @ IP[e, k, :, :3].astype(np.float64).T + IP[e, k, :, 3]
            parts_v.append(wv)
            parts_t.append(mt + base)
            offs.append(len(ts) + sum(len(x[1]) for x in inst_mesh[:k]))
            base += len(mv)
        U = oracle.Scene(np.concatenate(parts_v).astype(np.float32), np.concatenate(parts_t), bvh=False)
        sl = slice(e * tab.n_rays, (e + 1) * tab.n_rays)
        ru, iu, fu = U.cast(o[sl], d[sl], R)
        ok = (fl[sl] == 0) & (fu == 0)
        # world vertices rounded to float32 move surfaces by ~1e-7 m
        np.testing.assert_allclose(r[sl][ok], ru[ok], rtol=1e-5, atol=1e-5)
        gi = np.where(inst[sl] < 0, ids[sl], np.array(offs)[inst[sl] + 1] + ids[sl])
        gi = np.where(ids[sl] < 0, -1, gi)
        assert np.mean(gi[ok] == iu[ok]) > 0.999


@pytest.mark.parametrize("bvh", [False, True])
def test_edge_measure_is_the_continuous_edge_flag(bvh):
    """edge_measure (smallest ray-to-edge distance over L_k in the flag's
    window) is below 1e-6 exactly where the EDGE flag is set; a ray aimed at
    an edge's midpoint measures ~0, and nudging it sideways by a known angle
    raises the measure by that angle's chord over L (closed form)."""
    uv, ut = synth.icosphere_unit(3)
    v = (uv * 2.0).astype(np.float32)
    sc = oracle.Scene(v, ut, bvh=bvh)
    rng = np.random.default_rng(7)
    # rays from outside at the midpoints of 200 edges facing the origin (on a
    # convex mesh the first crossing), plus 2000 random rays
    eye = np.array([0.3, -0.2, 9.0])
    allmid = 0.5 * (v[ut[:, 0]].astype(np.float64) + v[ut[:, 1]])
    front = np.nonzero(np.einsum("ij,ij->i", allmid, eye - allmid) > 0.3 * np.linalg.norm(allmid, axis=1)
                       * np.linalg.norm(eye - allmid, axis=1))[0]
    k = rng.choice(front, 200, replace=False)
    mid = allmid[k]
    o = np.tile(eye[None], (200, 1))
    d = mid - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o2 = rng.uniform(-6, 6, (2000, 3))
    d2 = rng.standard_normal((2000, 3))
    d2 /= np.linalg.norm(d2, axis=1, keepdims=True)
    O = np.concatenate([o, o2]).astype(np.float32)
    D = np.concatenate([d, d2]).astype(np.float32)
    r, ids, fl = sc.cast(O, D, 50.0)
    m = sc.edge_measure(O, D, r, cap=1e-3)
    assert np.array_equal((fl & oracle.FLAG_EDGE) != 0, m < 1e-6)
    aimed = m[:200]
    assert np.all(aimed < 1e-6)                               # float32 rounding of the aim only
    # a sideways nudge by angle a (perpendicular to the edge) moves the line
    # a |p - o| from the edge point p: the measure is a |p - o| / L_k, L_k the
    # farthest vertex of the nearer triangle -- unless the nudged ray hits
    # before the edge's closest approach (the edge then lies beyond the hit,
    # outside the window, and the measure is the cap)
    a = 2e-4
    perp = np.cross(d, (v[ut[k, 1]] - v[ut[k, 0]]).astype(np.float64))
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    dn = d + a * perp
    dn /= np.linalg.norm(dn, axis=1, keepdims=True)
    rn, idn, fln = sc.cast(o.astype(np.float32), dn.astype(np.float32), 50.0)
    mn = sc.edge_measure(o.astype(np.float32), dn.astype(np.float32), rn, cap=1e-3)
    assert not np.any(fln & oracle.FLAG_EDGE)
    L = np.linalg.norm(v[ut[idn]].astype(np.float64) - eye, axis=2).max(axis=1)
    ratio = mn * L / (a * np.linalg.norm(mid - eye, axis=1))
    near = mn < 1e-3
    assert near.mean() > 0.3 and np.all(mn[~near] == 1e-3)
    assert np.all((ratio[near] > 0.95) & (ratio[near] < 1.01))
