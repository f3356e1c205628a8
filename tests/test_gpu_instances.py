"""GPU parity of per-environment rigid instances and return points through
the C-ABI (fgl_cast_batched items with instances / out_points).

Contract: as for the scene alone (tests/test_gpu_parity.py), against the
oracle's scene-plus-instances cast (oracle.cast_with_instances): unflagged
rays match hit/miss, triangle id and instance exactly and the range within
1e-4 + 1e-6 t; TIE rays match the range.  Return points match o + t d within
the range tolerance times |d| plus the rounding of o + t d.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

fgl = pytest.importorskip("paper_2509_17390_gb300")


def rot_z(a):
    return np.array([[np.cos(a), -np.sin(a), 0], [np.sin(a), np.cos(a), 0], [0, 0, 1.0]])


def instance_setup(seed, n_env, n_inst):
    rng = np.random.default_rng(seed)
    vs, ts, obs = synth.tiny_room_scene(seed)
    uv, ut = synth.icosphere_unit(2)
    meshes = [((0.35 * uv).astype(np.float32), ut),
              synth.aabb_box((-0.3, -0.2, -0.25), (0.3, 0.2, 0.25), 2),
              synth.aabb_box((-0.1, -0.1, -0.6), (0.1, 0.1, 0.6), 1)][:n_inst]
    P = synth.sample_free_pose(rng, obs, n_env)
    IP = np.zeros((n_env, n_inst, 3, 4), np.float32)
    for e in range(n_env):
        for k in range(n_inst):
            IP[e, k, :, :3] = synth.random_rotation(rng, 1)[0] if k == 1 else rot_z(rng.uniform(0, 2 * np.pi))
            IP[e, k, :, 3] = P[e, :, 3] + rng.uniform(-2.5, 2.5, 3) * [1, 1, 0.3] + [0, 0, 0.1]
    return vs, ts, meshes, P, IP


def gpu_cast(scene, sensor, P, R, inst_scenes, IP, min_range=0.0, points=True, graph=False, stream=None):
    n = P.shape[0] * sensor.n_rays
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    r = torch.full((n,), -7.0, device="cuda")
    i = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    inst = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    pts = torch.full((n, 3), -7.0, device="cuda") if points else None
    ex = {"out_instance": inst}
    if points:
        ex["points"] = pts
    if inst_scenes:
        ex["instances"] = inst_scenes
        ex["instance_poses"] = cu(IP)
    opts = fgl.BatchOpts(use_graph=1) if graph else None
    fgl.cast_batched([(scene, sensor, cu(P), R, r, i, min_range, ex)], opts, stream=stream)
    fgl.sync(stream)
    return (r.cpu().numpy(), i.cpu().numpy(), inst.cpu().numpy(),
            pts.cpu().numpy() if points else None)


def check(gr, gi, ginst, r_o, i_o, inst_o, fl, R):
    hard = (fl & (oracle.FLAG_EDGE | oracle.FLAG_RANGE)) != 0
    tie = (fl & oracle.FLAG_TIE) != 0
    ok = ~hard
    tol = 1e-4 + 1e-6 * np.abs(r_o)
    bad = ok & ((gi >= 0) != (i_o >= 0))
    bad |= ok & ~tie & ((gi != i_o) | (ginst != inst_o))
    bad |= ok & (i_o >= 0) & (np.abs(gr - r_o) > tol)
    bad |= ok & (i_o < 0) & (gr != np.float32(R))
    assert not bad.any(), (int(bad.sum()), np.nonzero(bad)[0][:10])
    assert hard.mean() < 0.01
    assert np.all(gr <= np.float32(R))


@pytest.mark.parametrize("width", [8, 4])
def test_instances_vs_oracle(width):
    vs, ts, meshes, P, IP = instance_setup(5, 6, 3)
    tab = synth.grid_sensor(16, -15, 15, 360)
    se = fgl.Sensor.from_table(tab)
    scene = fgl.Scene(vs, ts, width=width)
    inst = [fgl.Scene(v, t, width=w) for (v, t), w in zip(meshes, (width, 12 - width, width))]
    gr, gi, ginst, pts = gpu_cast(scene, se, P, 100.0, inst, IP)
    o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), P)
    r_o, i_o, inst_o, fl = oracle.cast_with_instances(oracle.Scene(vs, ts), [oracle.Scene(v, t) for v, t in meshes],
                                                      o, d, IP, tab.n_rays, 100.0)
    check(gr, gi, ginst, r_o, i_o, inst_o, fl, 100.0)
    assert (ginst >= 0).sum() > 500 and set(np.unique(ginst)) >= {-1, 0, 1, 2}
    # return points: o + t d
    hit = gi >= 0
    ref = o.astype(np.float64) + gr.astype(np.float64)[:, None] * d.astype(np.float64)
    err = np.abs(pts[hit] - ref[hit]).max(axis=1)
    assert np.all(err <= 4e-7 * (np.abs(ref[hit]).max(axis=1) + 1)), float(err.max())
    assert np.all(np.isnan(pts[~hit]))


def test_instances_with_min_range_and_graph_replay():
    vs, ts, meshes, P, IP = instance_setup(7, 4, 2)
    tab = synth.grid_sensor(8, -10, 10, 180)
    se = fgl.Sensor.from_table(tab)
    scene = fgl.Scene(vs, ts)
    inst = [fgl.Scene(v, t) for v, t in meshes]
    o, d = oracle.world_rays(oracle.sensor_dirs(tab.elev, tab.azim), P)
    r_o, i_o, inst_o, fl = oracle.cast_with_instances(oracle.Scene(vs, ts), [oracle.Scene(v, t) for v, t in meshes],
                                                      o, d, IP, tab.n_rays, 60.0, min_range=1.2)
    stream = torch.cuda.Stream()
    outs = [gpu_cast(scene, se, P, 60.0, inst, IP, min_range=1.2, graph=True, stream=stream) for _ in range(2)]
    for gr, gi, ginst, _ in outs:
        check(gr, gi, ginst, r_o, i_o, inst_o, fl, 60.0)
    assert all(np.array_equal(a, b) for a, b in zip(outs[0][:3], outs[1][:3]))
    # moving the instances changes the graph's inputs only: replay sees the new poses
    IP2 = IP.copy()
    IP2[:, :, :, 3] += 0.5
    r2, i2, n2, f2 = oracle.cast_with_instances(oracle.Scene(vs, ts), [oracle.Scene(v, t) for v, t in meshes],
                                                o, d, IP2, tab.n_rays, 60.0, min_range=1.2)
    gr, gi, ginst, _ = gpu_cast(scene, se, P, 60.0, inst, IP2, min_range=1.2, graph=True, stream=stream)
    check(gr, gi, ginst, r2, i2, n2, f2, 60.0)


def test_no_instances_points_and_out_instance():
    vs, ts, meshes, P, IP = instance_setup(9, 3, 1)
    tab = synth.grid_sensor(8, -10, 10, 90)
    se = fgl.Sensor.from_table(tab)
    scene = fgl.Scene(vs, ts)
    gr, gi, ginst, pts = gpu_cast(scene, se, P, 100.0, [], None)
    assert np.all(ginst == -1)
    plain = fgl.cast(scene, se, torch.from_numpy(P).cuda(), 100.0)
    fgl.sync()
    assert np.array_equal(gr, plain[0].cpu().numpy()) and np.array_equal(gi, plain[1].cpu().numpy())
    assert np.all(np.isfinite(pts[gi >= 0])) and np.all(np.isnan(pts[gi < 0]))


def test_walk_instances_fullsize_sampled_vs_oracle():
    """The walk_instances bench configuration (4096 environments x 5,760
    rays on the 1,000,300-triangle scene, four moving rigid instances each,
    the return points) cast in one batched launch: 48 sampled environments,
    all their rays, against the oracle's scene-plus-instances cast."""
    from synth import workloads
    wi = workloads.walk_instances(2, 4096, 3)
    w, IP = wi.walk, wi.poses[2]
    scene = fgl.Scene(w.verts, w.tris)
    inst = [fgl.Scene(v, t) for v, t in wi.meshes]
    se = fgl.Sensor.from_table(w.sensor)
    P = w.poses[2]
    gr, gi, ginst, pts = gpu_cast(scene, se, P, w.max_range, inst, IP, graph=True, stream=torch.cuda.Stream())
    envs = np.sort(np.random.default_rng(5).choice(4096, 48, replace=False))
    n = se.n_rays
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), P[envs])
    r_o, i_o, inst_o, fl = oracle.cast_with_instances(oracle.Scene(w.verts, w.tris),
                                                      [oracle.Scene(v, t) for v, t in wi.meshes],
                                                      o, d, IP[envs], n, w.max_range)
    sel = (envs[:, None] * n + np.arange(n)[None, :]).ravel()
    check(gr[sel], gi[sel], ginst[sel], r_o, i_o, inst_o, fl, w.max_range)
    assert (ginst[sel] >= 0).mean() > 0.05                    # the instances are in view
    hit = gi[sel] >= 0
    ref = o.astype(np.float64) + gr[sel].astype(np.float64)[:, None] * d.astype(np.float64)
    err = np.abs(pts[sel][hit] - ref[hit]).max(axis=1)
    assert np.all(err <= 4e-7 * (np.abs(ref[hit]).max(axis=1) + 1))


@pytest.mark.parametrize("min_range", [0.0, 0.7])
def test_fused_instance_pass_equals_per_instance_passes(min_range):
    """Instances of one width go through one fused launch, mixed widths
    through one pass per instance; widths never change a result, so both
    give the same ranges, triangles, instances and points bit for bit."""
    vs, ts, meshes, P, IP = instance_setup(9, 8, 3)
    se = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    scene = fgl.Scene(vs, ts)
    fused = [fgl.Scene(v, t, width=8) for v, t in meshes]
    mixed = [fgl.Scene(v, t, width=w) for (v, t), w in zip(meshes, (8, 4, 8))]
    a = gpu_cast(scene, se, P, 100.0, fused, IP, min_range=min_range)
    b = gpu_cast(scene, se, P, 100.0, mixed, IP, min_range=min_range)
    for x, y in zip(a, b):
        assert np.array_equal(x, y, equal_nan=True)
    assert (a[2] >= 0).sum() > 300


@pytest.mark.parametrize("n_env", [6, 1500])
def test_host_entry_with_instances_equals_device_entry(n_env):
    """fgl_cast_batched_host with instances, instance indices and return
    points in host memory (one launch for 6 environments; 1,500 x 5,760 =
    8.6 M rays run as overlapped chunks) returns what fgl_cast_batched returns
    from device memory, bit for bit."""
    vs, ts, meshes, P, IP = instance_setup(11, n_env, 3)
    se = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    scene = fgl.Scene(vs, ts)
    inst = [fgl.Scene(v, t, width=8) for v, t in meshes]
    dev = gpu_cast(scene, se, P, 100.0, inst, IP, min_range=0.2)
    n = n_env * se.n_rays
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    hr = torch.full((n,), -7.0).pin_memory()
    hi = torch.full((n,), -7, dtype=torch.int32).pin_memory()
    hk = torch.full((n,), -7, dtype=torch.int32).pin_memory()
    hp = torch.full((n, 3), -7.0).pin_memory()
    fgl.cast_batched_host([(scene, se, pin(P), 100.0, hr, hi, 0.2,
                            {"instances": inst, "instance_poses": pin(IP), "out_instance": hk,
                             "points": hp})])
    for x, y in zip(dev, (hr.numpy(), hi.numpy(), hk.numpy(), hp.numpy())):
        assert np.array_equal(x, y, equal_nan=True)
    assert (dev[2] >= 0).sum() > 50
