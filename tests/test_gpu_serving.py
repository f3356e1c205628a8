"""GPU tests of the batching runtime: autotuner and serving loop.

The serving contract: every request's result is the same as casting it
alone (bitwise here; the parity contract only asks for the range tolerance),
under continuous batching with other requests of different sizes, with
eviction under a small HBM budget, with poses kept in the server's
device-resident environment slots and updated from host or device memory,
and with host-side faults (injected allocation failures, cancellations,
malformed requests) affecting only their own requests.  The served mix of the
heterogeneous scenes is also checked against the FP64 oracle.
"""

import os

import numpy as np
import pytest

import oracle
import synth
from synth import workloads
from tests.helpers import assert_parity, oracle_mesher, parity_report

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
fgl = pytest.importorskip("paper_2509_17390_gb300")
from paper_2509_17390_gb300 import tuning  # noqa: E402


@pytest.fixture(scope="module")
def world():
    tiny = workloads.tiny_cast(1)
    indoor = workloads.indoor_scan(2)
    scenes = [fgl.Scene(tiny.verts, tiny.tris), fgl.Scene(indoor.verts, indoor.tris, width=8),
              fgl.Scene(indoor.verts, indoor.tris, width=4)]
    tables = [synth.grid_sensor(16, -15, 15, 360), synth.grid_sensor(7, -3, 20, 33),
              synth.rosette_sensor(1000, 4)]
    sensors = [fgl.Sensor.from_table(t) for t in tables]
    obs = [tiny.obstacles, indoor.obstacles, indoor.obstacles]
    return scenes, sensors, obs


def alone(scene, sensor, P, R, min_range=0.0):
    scene.upload()          # a server may have evicted it (no-op when resident)
    poses = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
    if min_range == 0.0:
        r, i = fgl.cast(scene, sensor, poses, R)
    else:
        n = P.shape[0] * sensor.n_rays
        r = torch.empty(n, dtype=torch.float32, device="cuda")
        i = torch.empty(n, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        fgl.cast_batched([(scene, sensor, poses, R, r, i, min_range)])
    fgl.sync()
    return r.cpu().numpy(), i.cpu().numpy()


def make_requests(world, n, seed, max_env=40):
    scenes, sensors, obs = world
    rng = np.random.default_rng(seed)
    reqs = []
    for k in range(n):
        si = int(rng.integers(len(scenes)))
        ti = int(rng.integers(len(sensors)))
        n_env = int(np.exp(rng.uniform(0, np.log(max_env))))
        P = synth.sample_free_pose(rng, obs[si], n_env, upright=bool(k % 2))
        R = float(rng.choice([5.0, 50.0, 120.0]))
        reqs.append((si, ti, P, R))
    return reqs


def serve_and_check(world, srv, reqs):
    scenes, sensors, _ = world
    sid = [srv.add_scene(s) for s in scenes]
    tid = [srv.add_sensor(s) for s in sensors]
    outs, tickets = [], []
    for si, ti, P, R in reqs:
        n = P.shape[0] * sensors[ti].n_rays
        r = torch.empty(n, dtype=torch.float32).pin_memory()
        i = torch.empty(n, dtype=torch.int32).pin_memory()
        tickets.append(srv.submit(sid[si], tid[ti], P, R, r, i))
        outs.append((r, i))
    infos = [srv.wait(t, timeout_ms=120000) for t in tickets]
    for (si, ti, P, R), (r, i) in zip(reqs, outs):
        ar, ai = alone(scenes[si], sensors[ti], P, R)
        assert np.array_equal(ar, r.numpy()) and np.array_equal(ai, i.numpy())
    return infos


def test_serving_results_equal_alone(world):
    srv = fgl.Server(tick_rays=200_000)            # small ticks: requests span several ticks
    reqs = make_requests(world, 24, seed=1)
    infos = serve_and_check(world, srv, reqs)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["ticks"] > 1
    assert st["p99_ms"] >= st["p50_ms"] > 0 and st["rays_per_s"] > 0
    assert all(x["latency_ms"] >= x["queue_ms"] >= 0 for x in infos)
    srv.close()


def test_serving_per_env_mode_equal_alone(world):
    srv = fgl.Server(mode=1)
    serve_and_check(world, srv, make_requests(world, 6, seed=2, max_env=8))
    srv.close()


def test_serving_evicts_under_small_budget(world):
    scenes, _, _ = world
    st0 = scenes[1].stats()
    big = st0["node_bytes"] + st0["tri_bytes"]
    # room for one large scene plus requests, not two: forces evictions
    srv = fgl.Server(hbm_budget_bytes=int(big * 1.6), tick_rays=300_000)
    reqs = [r for r in make_requests(world, 16, seed=3, max_env=12)]
    serve_and_check(world, srv, reqs)
    st = srv.stats()
    assert st["evictions"] > 0 and st["uploads"] > 0
    srv.close()
    for s in scenes:       # leave every scene resident for the other tests
        s.upload()


def test_serving_budget_rejection_and_faults(world):
    scenes, sensors, obs = world
    srv = fgl.Server(hbm_budget_bytes=200 << 20)
    sid = srv.add_scene(scenes[0])
    tid = srv.add_sensor(sensors[0])
    P = synth.sample_free_pose(np.random.default_rng(5), obs[0], 8)
    huge = np.repeat(P, 8000, axis=0)        # 64k envs x 5760 rays x 8 B = 2.9 GB
    r = np.empty(huge.shape[0] * sensors[0].n_rays, np.float32)
    i = np.empty_like(r, dtype=np.int32)
    with pytest.raises(fgl.FglError) as e:
        srv.submit(sid, tid, huge, 10.0, r, i)
    assert e.value.status == fgl.FGL_ERR_BUDGET
    # malformed requests are rejected at submission
    ro = np.empty(8 * sensors[0].n_rays, np.float32)
    io = np.empty_like(ro, dtype=np.int32)
    bad = P.copy()
    bad[0, 0, 0] = np.nan
    for args in ((sid, tid, bad, 10.0), (sid + 7, tid, P, 10.0), (sid, tid, P, float("nan"))):
        with pytest.raises(fgl.FglError) as e:
            srv.submit(*args, ro, io)
        assert e.value.status == fgl.FGL_ERR_INVALID
    # output buffers must stay alive until the request completes
    bufs = [(np.empty_like(ro), np.empty_like(io)) for _ in range(10)]
    # injected allocation failures hit exactly the next two admissions
    srv.inject_alloc_failures(2)
    tk = [srv.submit(sid, tid, P, 10.0, *bufs[k]) for k in range(4)]
    st = [srv.wait(t, 60000, check=False)["status"] for t in tk]
    assert st == [fgl.FGL_ERR_OOM, fgl.FGL_ERR_OOM, fgl.FGL_OK, fgl.FGL_OK]
    # cancelling a request: it ends cancelled (or already done), others unaffected
    tk = [srv.submit(sid, tid, P, 10.0, *bufs[4 + k]) for k in range(6)]
    srv.cancel(tk[3])
    st = [srv.wait(t, 60000, check=False)["status"] for t in tk]
    assert st[3] in (fgl.FGL_ERR_CANCELLED, fgl.FGL_OK)
    assert all(s == fgl.FGL_OK for k, s in enumerate(st) if k != 3)
    srv.close()


def test_serving_contains_worker_exceptions(world):
    """A host exception in the worker thread (injected between packing a tick
    and launching it) fails exactly the requests with chunks in that tick,
    with FGL_ERR_INTERNAL: a request split over several ticks ends once, its
    later chunks unscheduled; concurrent and later requests complete bitwise
    equal to casting them alone; the server keeps serving and holds no
    request's buffers afterwards."""
    scenes, sensors, obs = world
    P = synth.sample_free_pose(np.random.default_rng(21), obs[1], 6)
    n = 6 * sensors[1].n_rays
    ar, ai = alone(scenes[1], sensors[1], P, 50.0)
    bufs = [(np.empty(n, np.float32), np.empty(n, np.int32)) for _ in range(12)]

    def exact(k):
        return np.array_equal(bufs[k][0], ar) and np.array_equal(bufs[k][1], ai)

    for tick_rays in (0, 2 * sensors[1].n_rays):       # one tick a request / three ticks
        srv = fgl.Server(tick_rays=tick_rays)
        sid, tid = srv.add_scene(scenes[1]), srv.add_sensor(sensors[1])
        b = 0 if tick_rays == 0 else 6
        srv.inject_worker_faults(1)
        t0 = srv.submit(sid, tid, P, 50.0, *bufs[b])
        assert srv.wait(t0, 60000, check=False)["status"] == fgl.FGL_ERR_INTERNAL
        t1 = srv.submit(sid, tid, P, 50.0, *bufs[b + 1])
        assert srv.wait(t1, 60000, check=False)["status"] == fgl.FGL_OK and exact(b + 1)
        srv.inject_worker_faults(1)
        tk = [srv.submit(sid, tid, P, 50.0, *bufs[b + 2 + k]) for k in range(4)]
        st = [srv.wait(t, 60000, check=False)["status"] for t in tk]
        assert fgl.FGL_ERR_INTERNAL in st
        assert all(s == fgl.FGL_ERR_INTERNAL or (s == fgl.FGL_OK and exact(b + 2 + k))
                   for k, s in enumerate(st))
        s2 = srv.stats()
        assert s2["rejected"] == 1 + st.count(fgl.FGL_ERR_INTERNAL) and s2["active"] == 0
        assert s2["pending"] == 0 and s2["completed"] == 1 + st.count(fgl.FGL_OK)
        srv.close()


def test_serving_env_slots_keep_poses_on_device(world):
    """Per-environment pose state resident on the device: requests scan slot
    ranges as they are, overwrite them from host or from device memory first,
    or carry their own poses, all submitted at once.  Each result equals,
    bitwise, casting alone the poses its slots held at its turn in
    submission order (earlier requests' updates applied, later ones not), and
    the slots read back as the last update left them."""
    scenes, sensors, obs = world
    rng = np.random.default_rng(31)
    srv = fgl.Server(tick_rays=150_000, env_capacity=100)
    sid = [srv.add_scene(s) for s in scenes]
    tid = [srv.add_sensor(s) for s in sensors]
    P0 = synth.sample_free_pose(rng, obs[1], 40, upright=False)
    first = srv.add_envs(P0)
    assert first == 0 and np.array_equal(srv.read_poses(0, 40), P0)
    Pa = synth.sample_free_pose(rng, obs[1], 20)
    Pb = synth.sample_free_pose(rng, obs[1], 20, upright=False)
    Pb_dev = torch.from_numpy(Pb).cuda()
    Q = synth.sample_free_pose(rng, obs[1], 7)
    state = P0.copy()
    # (scene, sensor, slot range or None, update (None / host / device), own poses, min_range)
    plan = [(1, 0, (0, 40), None, None, 0.0),
            (1, 1, (0, 20), "host", Pa, 0.0),
            (2, 0, (0, 40), None, None, 0.0),
            (1, 2, (10, 30), "device", Pb, 0.0),
            (1, 0, (5, 35), None, None, 0.5),
            (2, 1, None, None, Q, 0.0),
            (1, 0, (0, 40), None, None, 0.0),
            (2, 2, (30, 40), "host", Pa[:10], 0.0)]
    tickets, outs, expect = [], [], []
    for k, (si, ti, rg, upd, P, rmin) in enumerate(plan):
        if rg is None:
            used = P
        else:
            a, b = rg
            if upd is not None:
                state[a:b] = P
            used = state[a:b].copy()
        n = used.shape[0] * sensors[ti].n_rays
        if k % 2:
            r, i = np.empty(n, np.float32), np.empty(n, np.int32)             # pageable
        else:
            r = torch.empty(n, dtype=torch.float32).pin_memory()
            i = torch.empty(n, dtype=torch.int32).pin_memory()
        if rg is None:
            t = srv.submit(sid[si], tid[ti], P, 50.0, r, i, min_range=rmin)
        elif upd is None:
            t = srv.submit(sid[si], tid[ti], None, 50.0, r, i, min_range=rmin, env_first=rg[0],
                           n_env=rg[1] - rg[0])
        else:
            t = srv.submit(sid[si], tid[ti], Pb_dev if upd == "device" else P, 50.0, r, i,
                           min_range=rmin, env_first=rg[0])
        tickets.append(t)
        outs.append((r, i))
        expect.append((si, ti, used, rmin))
    for t in tickets:
        srv.wait(t, timeout_ms=120000)
    for (si, ti, used, rmin), (r, i) in zip(expect, outs):
        ar, ai = alone(scenes[si], sensors[ti], used, 50.0, rmin)
        assert np.array_equal(ar, np.asarray(r)) and np.array_equal(ai, np.asarray(i))
    assert np.array_equal(srv.read_poses(0, 40), state)
    # slot ranges are checked at submission, capacity at registration
    ro, io = np.empty(sensors[0].n_rays, np.float32), np.empty(sensors[0].n_rays, np.int32)
    with pytest.raises(fgl.FglError) as e:
        srv.submit(sid[0], tid[0], None, 10.0, ro, io, env_first=40, n_env=1)
    assert e.value.status == fgl.FGL_ERR_INVALID
    assert srv.add_envs(np.concatenate([P0, P0[:20]])) == 40      # fills the 100 slots
    with pytest.raises(fgl.FglError) as e:
        srv.add_envs(P0[:1])
    assert e.value.status == fgl.FGL_ERR_CAPACITY
    assert srv.stats()["active"] == 0
    srv.close()


def test_serving_hetero_mix_vs_oracle():
    """The served workload's scene and sensor mix -- the 8 heterogeneous
    meshes (86k - 5.05M triangles, from the oracle's own 3DGS-to-mesh steps),
    the 21 sensors, a minimum range on some requests, poses carried by the
    request or kept in resident slots and updated from host or device memory
    -- submitted at once under continuous batching.  Every request equals its
    cast alone bitwise and, on a sample of its rays, the FP64 oracle."""
    meshes = workloads.hetero_meshes(oracle_mesher, 4)
    tables = workloads.hetero_sensors(4)
    scenes = [fgl.Scene(m.verts, m.tris, width=8 if k % 2 == 0 else 4) for k, m in enumerate(meshes)]
    sensors = [fgl.Sensor.from_table(t) for t in tables]
    rng = np.random.default_rng(51)
    srv = fgl.Server(tick_rays=2 << 20, env_capacity=8 * 32)
    sid = [srv.add_scene(s) for s in scenes]
    tid = [srv.add_sensor(s) for s in sensors]
    pools = [synth.sample_free_pose(rng, m.obstacles, 32, margin=0.25) for m in meshes]
    firsts = [srv.add_envs(P) for P in pools]
    state = [P.copy() for P in pools]
    tickets, keep, expect = [], [], []
    for k in range(40):
        m = int(rng.integers(len(meshes)))
        ti = int(rng.integers(len(tables)))
        n_env = max(1, int(np.exp(rng.uniform(0, np.log(12)))))
        if sensors[ti].n_rays > 100_000:
            n_env = min(n_env, 3)
        rmin = 0.3 if k % 3 == 0 else 0.0
        src = int(rng.integers(4))
        n = n_env * sensors[ti].n_rays
        if k % 2:
            r, i = np.empty(n, np.float32), np.empty(n, np.int32)
        else:
            r = torch.empty(n, dtype=torch.float32).pin_memory()
            i = torch.empty(n, dtype=torch.int32).pin_memory()
        a = int(rng.integers(0, 32 - n_env + 1))
        if src == 0:
            used = synth.sample_free_pose(rng, meshes[m].obstacles, n_env, margin=0.25)
            t = srv.submit(sid[m], tid[ti], used, 30.0, r, i, min_range=rmin)
        elif src == 1:
            used = state[m][a:a + n_env].copy()
            t = srv.submit(sid[m], tid[ti], None, 30.0, r, i, min_range=rmin,
                           env_first=firsts[m] + a, n_env=n_env)
        else:
            used = synth.sample_free_pose(rng, meshes[m].obstacles, n_env, margin=0.25)
            state[m][a:a + n_env] = used
            src_p = torch.from_numpy(used).cuda() if src == 3 else used
            t = srv.submit(sid[m], tid[ti], src_p, 30.0, r, i, min_range=rmin,
                           env_first=firsts[m] + a)
            keep.append(src_p)                     # a device update must outlive the request
        tickets.append(t)
        expect.append((m, ti, used, rmin, r, i))
    infos = [srv.wait(t, timeout_ms=300000) for t in tickets]
    assert srv.stats()["completed"] == 40
    assert all(x["status"] == fgl.FGL_OK for x in infos)
    osc = {}
    for m, ti, used, rmin, r, i in expect:
        gr, gi = np.asarray(r), np.asarray(i)
        ar, ai = alone(scenes[m], sensors[ti], used, 30.0, rmin)
        assert np.array_equal(ar, gr) and np.array_equal(ai, gi)
        if m not in osc:
            osc[m] = oracle.Scene(meshes[m].verts, meshes[m].tris, bvh=True)
        tab = tables[ti]
        o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), used)
        idx = rng.choice(len(o), min(len(o), 3000), replace=False)
        rep = parity_report(osc[m], o[idx], d[idx], 30.0, gr[idx], gi[idx], min_range=rmin)
        assert_parity(rep)
    for m in range(len(meshes)):
        assert np.array_equal(srv.read_poses(firsts[m], 32), state[m])
    srv.close()


def test_autotune_keeps_results_and_caches(world, tmp_path):
    scenes, sensors, obs = world
    P = synth.sample_free_pose(np.random.default_rng(8), obs[1], 64, upright=False)
    poses = torch.from_numpy(P).cuda()
    n = 64 * sensors[0].n_rays
    r = torch.empty(n, device="cuda")
    i = torch.empty(n, dtype=torch.int32, device="cuda")
    items = [(scenes[1], sensors[0], poses, 120.0, r, i)]
    best, res = fgl.autotune(items, reps=2, passes=1)
    assert res["trials"] >= 5 and res["best_ms"] <= res["start_ms"] * 1.05
    fgl.cast_batched(items, best)
    fgl.sync()
    ar, ai = alone(scenes[1], sensors[0], P, 120.0)
    assert np.array_equal(ar, r.cpu().numpy()) and np.array_equal(ai, i.cpu().numpy())
    tab = synth.grid_sensor(16, -15, 15, 360)
    indoor = workloads.indoor_scan(2)
    path = str(tmp_path / "tune.json")
    t1 = tuning.tune_workload(indoor.verts, indoor.tris, tab, poses, 120.0, widths=(8, 4),
                              tiles=((4, 8), (1, 32)), cache_path=path, reps=2, passes=1,
                              scenes={8: scenes[1], 4: scenes[2]})
    assert t1["width"] in (8, 4) and not t1["cached"] and os.path.exists(path)
    t2 = tuning.tune_workload(indoor.verts, indoor.tris, tab, poses, 120.0, cache_path=path)
    assert t2["cached"] and t2["width"] == t1["width"] and t2["opts"] == t1["opts"]
