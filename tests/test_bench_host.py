"""Host-side logic of bench.py that needs no GPU: the clock sampler's summary
keeps only the samples taken inside the timed region (nvidia-smi's own
timestamps), reports the median SM clock, the maximum and every throttle
reason seen there, and falls back to all samples, flagged, when none fell
inside; the serve workload's trace is scaled to its offered load."""

import datetime
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import pytest  # noqa: E402

import bench  # noqa: E402


def _sampler(tmp_path, rows, t0_ms, t1_ms):
    c = bench.ClockSampler(0)
    c.path = str(tmp_path / "clocks.csv")
    now = datetime.datetime(2026, 1, 2, 3, 4, 5, 0)
    c.t0 = now + datetime.timedelta(milliseconds=t0_ms)
    c.t1 = now + datetime.timedelta(milliseconds=t1_ms)
    lines = []
    for ms, mhz, reasons in rows:
        ts = (now + datetime.timedelta(milliseconds=ms)).strftime(bench.ClockSampler.TS)[:-3]
        flags = ["Active" if r in reasons else "Not Active"
                 for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")]
        lines.append(", ".join([ts, "0", str(mhz), "2070", "950.25", "0x0"] + flags))
    lines.append("garbage line")
    open(c.path, "w").write("\n".join(lines) + "\n")
    return c


def test_clock_summary_keeps_the_timed_region(tmp_path):
    rows = [(-50, 345, ()), (0, 2070, ()), (50, 2040, ("sw_power_cap",)), (100, 2070, ()),
            (150, 2055, ()), (200, 600, ("hw_slowdown",))]
    s = _sampler(tmp_path, rows, 0, 160).summary()
    assert s["samples"] == 4 and s["samples_in_timed_region"] == 4
    assert s["sm_mhz"] == 2062.5 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]                      # the hw_slowdown came after
    assert not os.path.exists(str(tmp_path / "clocks.csv"))


def test_clock_summary_falls_back_to_all_samples(tmp_path):
    rows = [(-100, 2070, ()), (300, 1980, ("hw_thermal_slowdown",))]
    s = _sampler(tmp_path, rows, 0, 40).summary()
    assert s["samples"] == 2 and s["samples_in_timed_region"] == 0
    assert s["reasons"] == ["hw_thermal_slowdown"] and s["sm_mhz"] == 2025.0


class _FakeServer:
    """Stands in for fgl.Server in the slot-plan tests (no GPU)."""

    def __init__(self):
        self.n = 0
        self.added = []

    def add_envs(self, poses):
        first = self.n
        self.n += len(poses)
        self.added.append(poses)
        return first


def test_slot_plan_rings_and_sources():
    """Each scene owns a ring of slots; a request takes the next n_env slots
    of its scene's ring (wrapping to the start when it would run past the
    end) and a contiguous slice of that scene's pose source."""
    torch = __import__("pytest").importorskip("torch")
    import numpy as np
    src = [torch.arange(10 * 12, dtype=torch.float32).reshape(10, 3, 4),
           torch.zeros(6, 3, 4)]
    srv = _FakeServer()
    plan = bench.SlotPlan(srv, src, 8, seed=1)
    assert srv.n == 16 and plan.first == [0, 8]
    assert np.array_equal(srv.added[0][:8], src[0][:8].numpy())          # initial poses from the source
    assert np.array_equal(srv.added[1][6:], src[1][:2].numpy())          # a short source repeats
    f, v = plan.take(0, 5)
    assert f == 0 and v.shape == (5, 3, 4)
    f, v = plan.take(0, 3)
    assert f == 5
    f, v = plan.take(0, 2)                                               # 8 + 2 > 8: back to the start
    assert f == 0
    f, v = plan.take(1, 4)
    assert f == 8
    with __import__("pytest").raises(ValueError):
        plan.take(1, 7)                                                  # more than its source holds
    trace = [(0.1, 0, 0, np.zeros((3, 3, 4), np.float32)), (0.2, 1, 0, np.zeros((2, 3, 4), np.float32))]
    st = bench.slot_trace(trace, bench.SlotPlan(_FakeServer(), src, 8, seed=2))
    assert [e[3] for e in st] == [None, None] and [e[4][1].shape[0] for e in st] == [3, 2]


def test_serve_trace_scaled_to_the_offered_load():
    """The serve workload's trace keeps its requests and order; its arrival
    times stretch so that the rays it offers over the stretched window equal
    the target (here a request of 3 environments on a 1,000-ray sensor and
    one of 5 on a 10-ray sensor: 3,050 rays over 2 s offered as 500 rays/s
    need a 6.1 s window)."""
    import numpy as np
    P3, P5 = np.zeros((3, 3, 4), np.float32), np.zeros((5, 3, 4), np.float32)
    trace = [(0.5, 0, 0, P3), (1.5, 1, 1, P5)]
    out, window = bench.scale_to_load(trace, 2.0, [1000, 10], 500.0)
    assert window == pytest.approx(6.1)
    assert [e[0] for e in out] == pytest.approx([0.5 * 3.05, 1.5 * 3.05])
    assert [e[1:3] for e in out] == [(0, 0), (1, 1)] and out[0][3] is P3
    offered = sum(e[3].shape[0] * [1000, 10][e[2]] for e in out) / window
    assert offered == pytest.approx(500.0)


def test_mesh_group_roofline_on_the_largest_set():
    """The mesh line's largest-set figure takes the set with the most voxels
    and divides its algorithmic bytes by its three Sec. IV-B stages only."""
    voxels = [1000, 8000, 27]
    caps = [(10, 20), (100, 200), (1, 1)]
    stages = [[9.0, 1.0, 1.0, 1.0], [50.0, 0.5, 1.0, 0.5], [1.0, 1.0, 1.0, 1.0]]
    r = bench.mesh_group_roofline(voxels, caps, stages, peak_gbs=1.0)
    nbytes = 11 * 8000 + 12 * 300
    assert r["voxels"] == 8000 and r["bytes"] == nbytes and r["ms"] == pytest.approx(2.0)
    assert r["achieved"] == pytest.approx(nbytes / 2e-3 / 1e9, abs=0.05)
    assert r["frac"] == pytest.approx(nbytes / 2e-3 / 1e9, rel=1e-3)
