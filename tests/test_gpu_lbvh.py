"""The GPU-built triangle LBVH (fgl_lbvh_*) and its one-thread-per-beam cast.

Structure: every triangle sits in exactly one leaf, every node but the root
has exactly one parent, child boxes nest in their parents' and each leaf box
holds its triangle grown by the margin.  Returns: bitwise equal to the wide
BVH's (same watertight test and (t, id) rule), and within the oracle's
contract; after a rebuild on moved vertices, equal to a fresh wide BVH of the
moved mesh.
"""

import numpy as np
import pytest

import oracle
import synth
from synth import workloads
from tests.helpers import assert_parity, parity_report

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

fgl = pytest.importorskip("paper_2509_17390_gb300")


def cu(a, dt=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dt)).cuda()


def check_structure(lb, verts, tris):
    st = lb.stats()
    nodes, trec = lb.export()
    nt = len(tris)
    ids = trec[:, 3].copy().view(np.int32)
    assert np.array_equal(np.sort(ids), np.arange(nt))                  # each triangle once
    tv = trec.reshape(-1, 3, 4)[:, :, :3]
    assert np.array_equal(tv, verts[tris[ids]])                         # its own vertices
    if nt == 1:
        return st
    rec = nodes.view(np.uint32).reshape(-1, 16)                         # 16 words per node
    fb = rec[:, :12].copy().view(np.float32)
    d = rec[:, 12:16].copy().view(np.int32)
    lbox = fb[:, 0:6]                                                   # lo xyz, hi xyz
    rbox = fb[:, 6:12]
    refs = d[:, :2].ravel()
    internal = refs[refs >= 0]
    leaves = ~refs[refs < 0]
    assert np.array_equal(np.sort(leaves), np.arange(nt))               # each leaf once
    assert np.array_equal(np.sort(internal), np.arange(1, nt - 1))      # each non-root node once
    assert np.all(d[1:, 2] >= 0) and d[0, 2] == -1
    m = np.float32(st["margin"])
    # leaf boxes hold their triangle grown by the margin; child boxes nest
    tlo, thi = tv.min(axis=1), tv.max(axis=1)
    for side, box in ((0, lbox), (1, rbox)):
        r = d[:, side]
        lf = r < 0
        k = ~r[lf]
        assert np.all(box[lf, :3] <= tlo[k] - m * 0.999) and np.all(box[lf, 3:] >= thi[k] + m * 0.999)
        it = ~lf
        child = r[it]
        cl = np.minimum(lbox[child, :3], rbox[child, :3])
        ch = np.maximum(lbox[child, 3:], rbox[child, 3:])
        assert np.all(box[it, :3] <= cl) and np.all(box[it, 3:] >= ch)
    assert st["depth"] >= int(np.ceil(np.log2(nt))) and st["overflow"] == 0
    # the reported depth is the tree's exact height (a leaf counts 1)
    order, stack = [], [0]
    while stack:
        q = stack.pop()
        order.append(q)
        stack.extend(int(c) for c in d[q, :2] if c >= 0)
    height = np.zeros(len(d), np.int64)
    for q in reversed(order):
        height[q] = 1 + max((height[c] if c >= 0 else 1) for c in d[q, :2])
    assert st["depth"] == height[0]
    return st


def test_structure_tiny_and_single_triangle():
    v, t, _ = synth.tiny_room_scene(2)
    lb = fgl.Lbvh(cu(v), cu(t, np.int32))
    check_structure(lb, v, t)
    one = fgl.Lbvh(cu(v), cu(t[:1], np.int32))
    check_structure(one, v, t[:1])


def test_indoor_bitwise_equal_to_wide_bvh_and_oracle():
    w = workloads.indoor_scan(2)
    lb = fgl.Lbvh(cu(w.verts), cu(w.tris, np.int32))
    st = check_structure(lb, w.verts, w.tris)
    assert st["build_ms"] > 0
    P = np.concatenate([w.poses, synth.sample_free_pose(np.random.default_rng(12), w.obstacles, 5)])
    se = fgl.Sensor.from_table(w.sensor)
    poses = cu(P)
    r1, i1 = lb.cast(se, poses, w.max_range)
    wide = fgl.Scene(w.verts, w.tris)
    r2, i2 = fgl.cast(wide, se, poses, w.max_range)
    fgl.sync()
    assert torch.equal(r1, r2) and torch.equal(i1, i2)
    # and against the oracle on the first pose
    o, d = oracle.world_rays(oracle.sensor_dirs(w.sensor.elev, w.sensor.azim), P[:1])
    n = len(o)
    rep = parity_report(oracle.Scene(w.verts, w.tris), o, d, w.max_range, r1[:n].cpu().numpy(),
                        i1[:n].cpu().numpy())
    assert_parity(rep)


def test_rebuild_after_moving_vertices_and_min_range():
    v, t, obs = synth.tiny_room_scene(4)
    rng = np.random.default_rng(4)
    P = synth.sample_free_pose(rng, obs, 4)
    se = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    vd = cu(v)
    td = cu(t, np.int32)
    lb = fgl.Lbvh(vd, td)
    poses = cu(P)
    for step in range(3):
        moved = (v + np.float32(0.05 * step) * np.array([1.0, -0.5, 0.0], np.float32)).astype(np.float32)
        vd.copy_(cu(moved))
        lb.rebuild(vd, td)
        check_structure(lb, moved, t)
        wide = fgl.Scene(moved, t)
        for rmin in (0.0, 1.3):
            r1, i1 = lb.cast(se, poses, 100.0, min_range=rmin)
            r2 = torch.empty_like(r1)
            i2 = torch.empty_like(i1)
            fgl.cast_batched([(wide, se, poses, 100.0, r2, i2, rmin)])
            fgl.sync()
            assert torch.equal(r1, r2) and torch.equal(i1, i2), (step, rmin)


def test_bad_input_is_rejected():
    v, t, _ = synth.tiny_room_scene(2)
    bad = t.copy()
    bad[5, 1] = len(v) + 3
    with pytest.raises(fgl.FglError):
        fgl.Lbvh(cu(v), cu(bad, np.int32))
