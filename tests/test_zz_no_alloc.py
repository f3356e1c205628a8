"""The allocation-free batched entry point (fgl_cast_batched_static).

Some callers cannot allocate device memory -- real-time loops that must not
trigger an allocator's device synchronisation, plugins inside an application
that owns every device allocation, processes whose device memory belongs to a
pool they do not own.  For them the library offers fgl_cast_batched_static, which keeps
its work queue in a fixed array inside the library instead of allocating it.
This file checks, through the C-ABI, that it returns exactly what the regular
fgl_cast_batched returns, on two calls in a row (the second reuses the array
the first one left behind), and that it rejects batches beyond its 256-item
limit.  It is collected last so a failure here cannot hide other results.
"""

import ctypes

import numpy as np
import pytest

import synth
from synth import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
fgl = pytest.importorskip("paper_2509_17390_gb300")


def _items(scenes, sensors, pose_sets, ranges, min_ranges=None):
    items, outs = [], []
    min_ranges = min_ranges or [0.0] * len(scenes)
    for sc, se, P, R, m in zip(scenes, sensors, pose_sets, ranges, min_ranges):
        poses = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
        n = P.shape[0] * se.n_rays
        r = torch.full((n,), -5.0, dtype=torch.float32, device="cuda")
        i = torch.full((n,), -5, dtype=torch.int32, device="cuda")
        items.append((sc, se, poses, R, r, i) + ((m,) if m else ()))
        outs.append((r, i))
    return items, outs


def _call(entry, items, opts=None):
    L = fgl.lib()
    arr = fgl.make_items(items)
    st = getattr(L, entry)(arr, len(items), ctypes.byref(opts) if opts else None, None)
    assert st == fgl.FGL_OK, L.fgl_last_error()
    assert L.fgl_sync(None) == fgl.FGL_OK, L.fgl_last_error()


def test_static_entry_matches_batched_on_two_calls():
    w = workloads.tiny_cast(1)
    indoor = workloads.indoor_scan(2)
    room = fgl.Scene(w.verts, w.tris, width=8)
    big8 = fgl.Scene(indoor.verts, indoor.tris, width=8)
    big4 = fgl.Scene(indoor.verts, indoor.tris, width=4)
    s1 = fgl.Sensor.from_table(w.sensor)
    s2 = fgl.Sensor.from_table(synth.grid_sensor(7, -3, 20, 33), 2, 4)
    s3 = fgl.Sensor.from_table(synth.rosette_sensor(1000, 5))
    rng = np.random.default_rng(40)
    calls = [
        ([room, big8, big4], [s1, s2, s3],
         [synth.sample_free_pose(rng, w.obstacles, 3, upright=False),
          synth.sample_free_pose(rng, indoor.obstacles, 5),
          synth.sample_free_pose(rng, indoor.obstacles, 2, upright=False)],
         [100.0, 50.0, 120.0]),
        ([big4, room], [s1, s2],
         [synth.sample_free_pose(rng, indoor.obstacles, 4, upright=False),
          synth.sample_free_pose(rng, w.obstacles, 6)],
         [7.0, 100.0]),
    ]
    for scenes, sensors, pose_sets, ranges in calls:        # two calls in a row
        ref_items, ref = _items(scenes, sensors, pose_sets, ranges)
        _call("fgl_cast_batched", ref_items)
        st_items, got = _items(scenes, sensors, pose_sets, ranges)
        _call("fgl_cast_batched_static", st_items)
        for (rr, ri), (gr, gi) in zip(ref, got):
            # the variant tolerance of this suite: bitwise equal results
            assert torch.equal(rr, gr) and torch.equal(ri, gi)
            assert (gi >= -1).all()


def test_static_entry_rejects_batches_beyond_its_limit():
    w = workloads.tiny_cast(1)
    sc = fgl.Scene(w.verts, w.tris)
    se = fgl.Sensor.from_table(w.sensor)
    P = np.repeat(w.poses, 1, axis=0)
    items, _ = _items([sc] * 257, [se] * 257, [P] * 257, [10.0] * 257)
    L = fgl.lib()
    arr = fgl.make_items(items)
    st = L.fgl_cast_batched_static(arr, 257, None, None)
    assert st == fgl.FGL_ERR_INVALID
    assert b"256" in L.fgl_last_error()
    assert L.fgl_cast_batched_static(arr, 256, None, None) == fgl.FGL_OK
    assert L.fgl_sync(None) == fgl.FGL_OK


def test_static_entry_matches_with_min_range_and_launch_options():
    """A minimum range (the t_min kernel variant) and non-default launch
    options (packet size, blocks per SM, lane-serial leaf tests) take other
    grid and grouping code in the allocation-free entry; results stay equal
    to fgl_cast_batched's."""
    w = workloads.tiny_cast(1)
    indoor = workloads.indoor_scan(2)
    room = fgl.Scene(w.verts, w.tris, width=4)
    big = fgl.Scene(indoor.verts, indoor.tris, width=8)
    s1 = fgl.Sensor.from_table(w.sensor)
    s2 = fgl.Sensor.from_table(synth.grid_sensor(32, -16, 15, 180))
    rng = np.random.default_rng(41)
    pose_sets = [synth.sample_free_pose(rng, w.obstacles, 3, upright=False),
                 synth.sample_free_pose(rng, indoor.obstacles, 6)]
    for opts in (None, fgl.BatchOpts(packet_rays=64, blocks_per_sm=2, tri_mode=1),
                 fgl.BatchOpts(packet_rays=96, block_threads=256, stack_smem=2)):
        ref_items, ref = _items([room, big], [s1, s2], pose_sets, [100.0, 60.0], [0.0, 0.8])
        _call("fgl_cast_batched", ref_items, opts)
        st_items, got = _items([room, big], [s1, s2], pose_sets, [100.0, 60.0], [0.0, 0.8])
        _call("fgl_cast_batched_static", st_items, opts)
        for (rr, ri), (gr, gi) in zip(ref, got):
            assert torch.equal(rr, gr) and torch.equal(ri, gi)
        assert (got[1][0][got[1][1] >= 0] >= 0.8).all()        # the minimum range held


def test_static_entry_leaves_free_device_memory_unchanged():
    """After a first call (which may load the kernels' code on the device),
    further calls take no device memory: the device's free bytes stay the
    same across them."""
    w = workloads.tiny_cast(1)
    sc = fgl.Scene(w.verts, w.tris)
    se = fgl.Sensor.from_table(w.sensor)
    rng = np.random.default_rng(42)
    P = synth.sample_free_pose(rng, w.obstacles, 4, upright=False)
    items, _ = _items([sc, sc], [se, se], [P, P[:2]], [100.0, 20.0])
    _call("fgl_cast_batched_static", items)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        _call("fgl_cast_batched_static", items)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
