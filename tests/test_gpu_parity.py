"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Contract (per ray): hit/miss and triangle id equal to the oracle's, range
within 1e-4 m + 1e-6 * range, except on rays the oracle flags as ambiguous
(edge-grazing, depth tie, range boundary); those must still pass the
oracle's plausibility check.  Results must be bitwise identical across every
launch variant (BVH width, stack split, postponing, block size, packet size,
refill threshold, graph capture, batched vs plain).
"""

import numpy as np
import pytest

import oracle
import synth
from synth import workloads
from tests.helpers import assert_parity, oracle_mesher, parity_report

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

fgl = pytest.importorskip("paper_2509_17390_gb300")


@pytest.fixture(scope="module")
def tiny():
    w = workloads.tiny_cast(1)
    P = np.concatenate([w.poses, synth.sample_free_pose(np.random.default_rng(9), w.obstacles, 7,
                                                        upright=False)])
    return w, P


@pytest.fixture(scope="module")
def indoor():
    w = workloads.indoor_scan(2)
    return w


@pytest.fixture(scope="module")
def indoor_scenes(indoor):
    return {W: fgl.Scene(indoor.verts, indoor.tris, width=W) for W in (8, 4)}


@pytest.fixture(scope="module")
def indoor_oracle(indoor):
    return oracle.Scene(indoor.verts, indoor.tris, bvh=True)


def run_plain(scene, sensor, P, max_range, opts=None):
    poses = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
    if opts is None:
        r, i = fgl.cast(scene, sensor, poses, max_range)
    else:
        r, i = fgl.cast_opts(scene, sensor, poses, max_range, opts)
    fgl.sync()
    return r.cpu().numpy(), i.cpu().numpy()


def run_batched(items_np, opts=None, stream=None):
    """items_np: (scene, sensor, poses np, max_range[, min_range])."""
    items, outs = [], []
    for it in items_np:
        sc, se, P, R = it[:4]
        poses = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
        n = P.shape[0] * se.n_rays
        r = torch.full((n,), -7.0, dtype=torch.float32, device="cuda")
        i = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        items.append((sc, se, poses, R, r, i) + tuple(it[4:]))
        outs.append((r, i))
    torch.cuda.synchronize()            # the fills above ran on the current stream
    fgl.cast_batched(items, opts, stream=stream)
    fgl.sync(stream)
    return [(r.cpu().numpy(), i.cpu().numpy()) for r, i in outs]


# ---------------------------------------------------------------------------
# ray generation (eq. r_j) is bit-identical to the oracle's
# ---------------------------------------------------------------------------
def test_sensor_dirs_bit_exact():
    for tab in (synth.grid_sensor(16, -15, 15, 360), synth.grid_sensor(32, -16, 15, 1800),
                synth.rosette_sensor(20000, 3)):
        se = fgl.Sensor.from_table(tab)
        assert np.array_equal(se.dirs(), oracle.sensor_dirs(tab.elev, tab.azim))


def test_world_rays_bit_exact(tiny):
    w, P = tiny
    for tab, tiles in ((w.sensor, (4, 8)), (synth.grid_sensor(7, -3, 20, 33), (3, 5)),
                       (synth.rosette_sensor(1000, 1), (1, 32))):
        se = fgl.Sensor.from_table(tab, *tiles)
        poses = torch.from_numpy(P).cuda()
        go, gd = fgl.world_rays(se, poses)
        fgl.sync()
        oo, od = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), P)
        assert np.array_equal(go.cpu().numpy(), oo)
        assert np.array_equal(gd.cpu().numpy(), od)


# ---------------------------------------------------------------------------
# parity against the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("width", [8, 4])
def test_tiny_cast_vs_brute_force(tiny, width):
    w, P = tiny
    sc = fgl.Scene(w.verts, w.tris, width=width)
    se = fgl.Sensor.from_table(w.sensor)
    gr, gi = run_plain(sc, se, P, w.max_range)
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), P)
    rep = parity_report(oracle.Scene(w.verts, w.tris, bvh=False), o, d, w.max_range, gr, gi)
    assert_parity(rep)
    assert rep["hits"] == rep["n"]          # closed room: every ray hits


@pytest.mark.parametrize("offset", [(0.0, 0.0, 0.0), (100.0, -60.0, 40.0)])
@pytest.mark.parametrize("width", [8, 4])
def test_translated_room_and_axis_aligned_beams(tiny, width, offset):
    """The child boxes' margin against the traversal's float32 plane
    arithmetic on the GPU: the tiny room moved away from the origin (the
    margin scales with the coordinates), seen through beams along the axes
    (direction components exactly 0, the reciprocal's clamp) and the grid
    sensor, from upright and tilted poses."""
    w, P = tiny
    off = np.asarray(offset, np.float64)
    v = (w.verts.astype(np.float64) + off).astype(np.float32)
    Pt = P.astype(np.float64).copy()
    Pt[:, :, 3] += off
    Pa = synth.pose_from_yaw(P[:3, :, 3].astype(np.float64) + off, [0.0, 0.0, 0.0])
    Pt = np.concatenate([Pt, Pa]).astype(np.float32)
    sc = fgl.Scene(v, w.tris, width=width)
    osc = oracle.Scene(v, w.tris, bvh=False)
    el = np.repeat([0.0, 0.4, -0.4], 4)
    az = np.tile([0.0, 0.5 * np.pi, np.pi, 1.5 * np.pi], 3)
    for tab_el, tab_az, se in ((w.sensor.elev, w.sensor.azim, fgl.Sensor.from_table(w.sensor)),
                               (el, az, fgl.Sensor(el, az, rows=3, cols=4))):
        gr, gi = run_plain(sc, se, Pt, w.max_range)
        o, d = oracle.world_rays(oracle.sensor_dirs(tab_el, tab_az), Pt)
        rep = parity_report(osc, o, d, w.max_range, gr, gi)
        assert_parity(rep)
        assert rep["hits"] == rep["n"]      # closed room: every ray hits


@pytest.mark.parametrize("width", [8, 4])
def test_indoor_scan_vs_bvh_oracle(indoor, indoor_scenes, indoor_oracle, width):
    w = indoor
    se = fgl.Sensor.from_table(w.sensor)
    gr, gi = run_plain(indoor_scenes[width], se, w.poses, w.max_range)
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), w.poses)
    rep = parity_report(indoor_oracle, o, d, w.max_range, gr, gi)
    assert_parity(rep)
    assert rep["flagged"] < 0.01 * rep["n"]


def test_indoor_random_poses_and_short_range(indoor, indoor_scenes, indoor_oracle):
    w = indoor
    P = synth.sample_free_pose(np.random.default_rng(31), w.obstacles, 6, upright=False)
    tab = synth.grid_sensor(16, -15, 15, 360)
    se = fgl.Sensor.from_table(tab)
    o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), P)
    for R in (120.0, 0.75):                 # short range: many misses
        gr, gi = run_plain(indoor_scenes[8], se, P, R)
        rep = parity_report(indoor_oracle, o, d, R, gr, gi)
        assert_parity(rep)
        if R < 1:
            assert rep["hits"] < rep["n"]


@pytest.mark.parametrize("width", [8, 4])
def test_min_range_vs_oracle(indoor, indoor_scenes, indoor_oracle, width):
    """t_min of eq. t_j*: nearer surfaces are passed through (the two-sided
    test then returns the back of a thin object or the next surface)."""
    w = indoor
    P = synth.sample_free_pose(np.random.default_rng(41), w.obstacles, 6, upright=False)
    tab = synth.grid_sensor(16, -15, 15, 360)
    se = fgl.Sensor.from_table(tab)
    o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), P)
    mins = (0.4, 1.5, 4.0)
    outs = run_batched([(indoor_scenes[width], se, P, 120.0, m) for m in mins])
    plain, _ = run_plain(indoor_scenes[width], se, P, 120.0)
    for m, (gr, gi) in zip(mins, outs):
        rep = parity_report(indoor_oracle, o, d, 120.0, gr, gi, min_range=m)
        assert_parity(rep)
        assert np.all(gr[gi >= 0] >= np.float32(m))
        assert np.any(gr > plain)                  # some nearer surfaces were skipped
    # one item alone gives the same bits as inside the mixed batch
    (gr1, gi1), = run_batched([(indoor_scenes[width], se, P, 120.0, mins[1])])
    assert np.array_equal(gr1, outs[1][0]) and np.array_equal(gi1, outs[1][1])


# ---------------------------------------------------------------------------
# variant invariance (bitwise)
# ---------------------------------------------------------------------------
def test_plain_variants_bitwise(indoor, indoor_scenes):
    w = indoor
    P = synth.sample_free_pose(np.random.default_rng(5), w.obstacles, 3, upright=False)
    tab = synth.grid_sensor(16, -15, 15, 360)
    base = None
    for tiles in ((4, 8), (1, 32), (16, 2)):
        se = fgl.Sensor.from_table(tab, *tiles)
        for W in (8, 4):
            for sdepth, tri_mode, postpone, block in ((12, 0, 0, 128), (12, 1, 20, 128), (8, 0, 0, 96),
                                                      (2, 1, 100, 64), (1, 1, -1, 256),
                                                      (30, 0, 0, 32), (0, 0, 0, 512)):
                opts = fgl.BatchOpts(block_threads=block, stack_smem=sdepth, postpone_pct=postpone,
                                     tri_mode=tri_mode)
                out = run_plain(indoor_scenes[W], se, P, w.max_range, opts)
                if base is None:
                    base = out
                else:
                    assert np.array_equal(out[0], base[0]) and np.array_equal(out[1], base[1]), \
                        (tiles, W, sdepth, tri_mode, postpone, block)


def test_batched_variants_bitwise_and_equal_plain(indoor, indoor_scenes, tiny):
    w = indoor
    tw, tP = tiny
    tscene = fgl.Scene(tw.verts, tw.tris)
    P1 = synth.sample_free_pose(np.random.default_rng(6), w.obstacles, 5, upright=False)
    P2 = synth.sample_free_pose(np.random.default_rng(7), w.obstacles, 3)
    s1 = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    s2 = fgl.Sensor.from_table(synth.grid_sensor(7, -3, 20, 33), 2, 4)     # ragged
    s3 = fgl.Sensor.from_table(synth.rosette_sensor(1000, 2))
    plain = [run_plain(indoor_scenes[8], s1, P1, 120.0),
             run_plain(indoor_scenes[4], s2, P2, 50.0),
             run_plain(tscene, s3, tP, 100.0),
             run_plain(indoor_scenes[8], s3, P2, 3.0)]
    items = [(indoor_scenes[8], s1, P1, 120.0), (indoor_scenes[4], s2, P2, 50.0),
             (tscene, s3, tP, 100.0), (indoor_scenes[8], s3, P2, 3.0)]
    stream = torch.cuda.Stream()
    for packet, block, sdepth, refill, tri_mode, postpone, graph in (
            (64, 128, 12, 8, 0, 0, 0), (32, 32, 0, 1, 1, -1, 0), (256, 256, 4, 32, 1, 100, 1),
            (96, 64, 2, 4, 0, 30, 1), (64, 128, 12, 8, 1, 20, 1), (64, 512, 8, 16, 0, 0, 1), (64, 128, 12, 32, 0, 0, 1)):
        opts = fgl.BatchOpts(packet_rays=packet, block_threads=block, stack_smem=sdepth,
                             refill_min=refill, postpone_pct=postpone, use_graph=graph,
                             tri_mode=tri_mode)
        for rep in range(2 if graph else 1):          # graph replay too
            outs = run_batched(items, opts, stream=stream if graph else None)
            for (pr, pi), (br, bi) in zip(plain, outs):
                assert np.array_equal(pr, br) and np.array_equal(pi, bi), (packet, block, sdepth)


def test_graph_replay_after_scene_rebuilt_at_other_width(indoor, indoor_scenes):
    """A captured graph is never replayed for a scene of another BVH width,
    even when the new scene's buffers land at the freed scene's addresses:
    the item records carry the width, so the graph's key changes."""
    w = indoor
    P = synth.sample_free_pose(np.random.default_rng(11), w.obstacles, 4)
    s = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    ref = run_plain(indoor_scenes[8], s, P, 120.0)
    assert all(np.array_equal(a, b) for a, b in zip(ref, run_plain(indoor_scenes[4], s, P, 120.0)))
    stream = torch.cuda.Stream()
    opts = fgl.BatchOpts(use_graph=1)
    for W in (8, 4, 8, 4):
        sc = fgl.Scene(w.verts, w.tris, width=W)
        for rep in range(2):
            (r, i), = run_batched([(sc, s, P, 120.0)], opts, stream=stream)
            assert np.array_equal(r, ref[0]) and np.array_equal(i, ref[1]), (W, rep)
        sc.close()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
def test_edge_cases(tiny):
    w, P = tiny
    sc = fgl.Scene(w.verts, w.tris)
    se = fgl.Sensor.from_table(w.sensor)
    # n_env = 0 is a no-op; an empty batch too
    poses = torch.zeros((0, 3, 4), dtype=torch.float32, device="cuda")
    r, i = fgl.cast(sc, se, poses, 10.0)
    assert r.numel() == 0
    fgl.cast_batched([])
    # tiny max_range: everything misses with (max_range, -1)
    gr, gi = run_plain(sc, se, P, 1e-3)
    assert np.all(gi == -1) and np.all(gr == np.float32(1e-3))
    # a sensor inside a closed box sees the box from inside (two-sided test)
    v, t = synth.aabb_box((0, 0, 0), (1, 1, 1), 3)
    bsc = fgl.Scene(v, t)
    Pin = synth.pose_from_yaw([[0.5, 0.5, 0.5]], [0.3])
    gr, gi = run_plain(bsc, se, Pin, 100.0)
    assert np.all(gi >= 0) and np.all(gr <= np.sqrt(3) / 2 + 1e-5)
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), Pin)
    assert_parity(parity_report(oracle.Scene(v, t, bvh=False), o, d, 100.0, gr, gi))
    # single-triangle scene
    v1 = np.array([[2, -50, -50], [2, 50, -50], [2, 0, 50]], np.float32)
    s1 = fgl.Scene(v1, np.array([[0, 1, 2]], np.int32))
    Pz = synth.pose_from_yaw([[0, 0, 0]], [0.0])
    gr, gi = run_plain(s1, se, Pz, 100.0)
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), Pz)
    assert_parity(parity_report(oracle.Scene(v1, np.array([[0, 1, 2]], np.int32), bvh=False),
                                o, d, 100.0, gr, gi))
    assert (gi == 0).any() and (gi == -1).any()


def test_argument_errors(tiny):
    w, P = tiny
    sc = fgl.Scene(w.verts, w.tris)
    se = fgl.Sensor.from_table(w.sensor)
    poses = torch.from_numpy(P).cuda()
    with pytest.raises(fgl.FglError):
        fgl.cast(sc, se, poses, float("nan"))
    with pytest.raises(fgl.FglError):
        fgl.cast(sc, se, poses, -1.0)
    with pytest.raises(fgl.FglError):
        fgl.cast_opts(sc, se, poses, 10.0, fgl.BatchOpts(block_threads=33))
    with pytest.raises(fgl.FglError):
        fgl.cast_batched([(sc, se, poses, 10.0, torch.empty(len(P) * se.n_rays, device="cuda"),
                           torch.empty(len(P) * se.n_rays, dtype=torch.int32, device="cuda"))],
                         fgl.BatchOpts(packet_rays=48))
    sc.evict()
    with pytest.raises(fgl.FglError):
        fgl.cast(sc, se, poses, 10.0)
    sc.upload()
    fgl.cast(sc, se, poses, 10.0)
    fgl.sync()


# ---------------------------------------------------------------------------
# the bench workload at full size, in the bench's launch configuration
# ---------------------------------------------------------------------------
def test_batched_walk_full_size_sampled(indoor_oracle):
    w = workloads.batched_walk(2, n_env=4096, n_steps=2)
    scene = fgl.Scene(w.verts, w.tris, width=8)
    sensor = fgl.Sensor.from_table(w.sensor)
    P = w.poses[1]
    n = P.shape[0] * sensor.n_rays
    poses = torch.from_numpy(P).cuda()
    r = torch.full((n,), -3.0, dtype=torch.float32, device="cuda")
    i = torch.full((n,), -3, dtype=torch.int32, device="cuda")
    stream = torch.cuda.Stream()
    opts = fgl.BatchOpts(use_graph=1)
    torch.cuda.synchronize()            # the fills above ran on the current stream
    for _ in range(2):
        fgl.cast_batched([(scene, sensor, poses, w.max_range, r, i)], opts, stream=stream)
    fgl.sync(stream)
    gr, gi = r.cpu().numpy(), i.cpu().numpy()
    # every output written, every range within [0, max_range], misses well formed
    assert np.all(gi >= -1) and np.all(gr > 0) and np.all(gr <= np.float32(w.max_range))
    assert np.all(gr[gi < 0] == np.float32(w.max_range))
    # sample: 24 whole environments + 20,000 random rays of the others
    rng = np.random.default_rng(77)
    envs = rng.choice(P.shape[0], 24, replace=False)
    idx = np.concatenate([(e * sensor.n_rays + np.arange(sensor.n_rays)) for e in envs] +
                         [rng.choice(n, 20000, replace=False)])
    idx = np.unique(idx)
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), P)
    rep = parity_report(indoor_oracle, o[idx], d[idx], w.max_range, gr[idx], gi[idx])
    assert_parity(rep)


# ---------------------------------------------------------------------------
# heterogeneous batch at its stated size: all 8 ladder meshes (86k - 5.05M
# triangles) from the oracle's 3DGS-to-mesh steps (an oracle input never comes
# from the CUDA path), the 256 environments and full sensor mix of the bench,
# one graph-captured launch per BVH width
# ---------------------------------------------------------------------------
def hetero_sample(rng, n_env, n_rays, whole_max=65536, env_rays=16384, extra=2000):
    """Indices into a group's rays (env-major): its first environment whole
    (or env_rays random rays of it when it has more than whole_max), plus
    `extra` random rays of the group's other environments."""
    first = np.arange(n_rays) if n_rays <= whole_max else rng.choice(n_rays, env_rays, replace=False)
    rest = np.empty(0, np.int64)
    if n_env > 1:
        rest = n_rays + rng.choice((n_env - 1) * n_rays, min(extra, (n_env - 1) * n_rays), replace=False)
    return np.unique(np.concatenate([first, rest]))


def test_hetero_batch_full_ladder_vs_oracle():
    meshes = workloads.hetero_meshes(oracle_mesher, 4)
    assert len(meshes) == 8 and len(meshes[-1].tris) > 4_000_000
    tables = workloads.hetero_sensors(4)
    envs = workloads.hetero_envs(4, meshes, n_env=256)
    scenes = [fgl.Scene(m.verts, m.tris, width=8 if k % 2 == 0 else 4) for k, m in enumerate(meshes)]
    groups = {}
    for m, s, P in envs:
        groups.setdefault((m, s), []).append(P)
    sensors = {s: fgl.Sensor.from_table(tables[s]) for (_, s) in groups}
    assert len({s for (_, s) in groups}) == len(tables)          # every sensor of the mix is cast
    items, keys = [], []
    for (m, s), Ps in sorted(groups.items()):
        P = np.stack(Ps)
        items.append((scenes[m], sensors[s], P, 30.0))
        keys.append((m, s, P))
    stream = torch.cuda.Stream()
    outs = run_batched(items, fgl.BatchOpts(use_graph=1), stream=stream)
    rng = np.random.default_rng(3)
    checked = np.zeros(len(meshes), np.int64)
    for m in range(len(meshes)):
        osc = oracle.Scene(meshes[m].verts, meshes[m].tris, bvh=True)
        for (mk, s, P), (gr, gi) in zip(keys, outs):
            if mk != m:
                continue
            assert np.all(gi >= -1) and np.all(gr <= np.float32(30.0))
            tab = tables[s]
            idx = hetero_sample(rng, P.shape[0], tab.n_rays)
            o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), P)
            rep = parity_report(osc, o[idx], d[idx], 30.0, gr[idx], gi[idx])
            assert_parity(rep)
            checked[m] += len(idx)
        del osc
    assert checked.min() >= 20000, checked


# ---------------------------------------------------------------------------
# end-to-end host entry (fgl_cast_batched_host): one launch for small batches,
# chunks whose copies overlap the next chunk's cast for large ones -- both
# bitwise equal to the device-buffer batched call
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n_big,n_small,pinned", [(3, 5, True), (200, 100, True), (3, 5, False),
                                                  (200, 100, False)])
def test_host_entry_equals_device_batched(n_big, n_small, pinned):
    """Page-locked outputs take the path where the kernel stores the returns
    straight into host memory; pageable ones the staged path (one launch for
    small batches, overlapped chunks for large ones).  Both equal the
    device-buffer call bit for bit."""
    v, t, obs = synth.tiny_room_scene(6)
    scene = fgl.Scene(v, t)
    big = fgl.Sensor.from_table(synth.grid_sensor(32, -16.0, 15.0, 1800))
    small = fgl.Sensor.from_table(synth.grid_sensor(16, -15.0, 15.0, 360))
    rng = np.random.default_rng(n_big)
    Pb = synth.sample_free_pose(rng, obs, n_big, upright=False)
    Ps = synth.sample_free_pose(rng, obs, n_small, upright=False)
    n_rays = n_big * big.n_rays + n_small * small.n_rays
    pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t)
    hb_r = pin(torch.empty(n_big * big.n_rays, dtype=torch.float32))
    hb_i = pin(torch.empty(n_big * big.n_rays, dtype=torch.int32))
    hs_r = pin(torch.empty(n_small * small.n_rays, dtype=torch.float32))
    hs_i = pin(torch.empty(n_small * small.n_rays, dtype=torch.int32))
    hb_r.fill_(-7.0)
    hs_i.fill_(-7)
    stream = torch.cuda.Stream()
    fgl.cast_batched_host([(scene, big, torch.from_numpy(Pb).pin_memory(), 60.0, hb_r, hb_i),
                           (scene, small, torch.from_numpy(Ps).pin_memory(), 60.0, hs_r, hs_i, 0.4)],
                          stream=stream)
    (db_r, db_i), (ds_r, ds_i) = run_batched([(scene, big, Pb, 60.0), (scene, small, Ps, 60.0, 0.4)])
    assert np.array_equal(hb_r.numpy(), db_r) and np.array_equal(hb_i.numpy(), db_i)
    assert np.array_equal(hs_r.numpy(), ds_r) and np.array_equal(hs_i.numpy(), ds_i)
    assert (n_rays >= 8 << 20) == (n_big == 200)            # the large case takes the chunked path


# ---------------------------------------------------------------------------
# evidence for the reading of "within 1e-6 (relative) of a triangle edge":
# GPU/oracle id mismatches against the oracle's edge measure (distance to the
# nearest edge over the triangle's distance scale L_k), swept over thresholds
# ---------------------------------------------------------------------------
SWEEP = (1e-8, 3e-8, 1e-7, 3e-7, 1e-6, 3e-6, 1e-5)


def sweep_counts(osc, o, d, max_range, gr, gi):
    r_o, i_o, fl = osc.cast(o, d, max_range)
    m = osc.edge_measure(o, d, r_o, cap=1e-4)
    bad = (gi != i_o) & ((fl & (oracle.FLAG_TIE | oracle.FLAG_RANGE)) == 0)
    return [int((bad & (m >= tau)).sum()) for tau in SWEEP], int(bad.sum()), len(o)


def test_edge_threshold_sweep():
    rows = []
    w = workloads.indoor_scan(2)
    scene = fgl.Scene(w.verts, w.tris)
    P = np.concatenate([w.poses, synth.sample_free_pose(np.random.default_rng(21), w.obstacles, 3)])
    se = fgl.Sensor.from_table(w.sensor)
    (gr, gi), = run_batched([(scene, se, P, w.max_range)])
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), P)
    rows.append(("indoor 1M tris", *sweep_counts(oracle.Scene(w.verts, w.tris), o, d, w.max_range, gr, gi)))
    meshes = workloads.hetero_meshes(oracle_mesher, 4, workloads.HETERO_LADDER[:4])
    mh = meshes[3]                                            # 3.5 cm marching-tetrahedra triangles
    tab = synth.grid_sensor(64, -25.0, 25.0, 2048)
    Ph = synth.sample_free_pose(np.random.default_rng(22), mh.obstacles, 3, margin=0.25)
    (gr, gi), = run_batched([(fgl.Scene(mh.verts, mh.tris), fgl.Sensor.from_table(tab), Ph, 30.0)])
    o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), Ph)
    rows.append((f"hetero mesh {len(mh.tris)} tris", *sweep_counts(oracle.Scene(mh.verts, mh.tris), o, d,
                                                                   30.0, gr, gi)))
    print("\nid mismatches (TIE/RANGE rays excluded) among rays whose edge measure is >= tau")
    print("case".ljust(28) + "".join(f"{t:>9.0e}" for t in SWEEP) + "   all  rays")
    for name, counts, total, n in rows:
        print(name.ljust(28) + "".join(f"{c:>9d}" for c in counts) + f"{total:>6d}{n:>8d}")
    for _, counts, _, _ in rows:
        assert counts[SWEEP.index(1e-6)] == 0
