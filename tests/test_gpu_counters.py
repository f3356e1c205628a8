"""GPU tests of the measurement entry points: the count_work phase counters
(fgl_work_phase_counters) and the L2 bandwidth probe (fgl_probe_l2_read).

The counters feed the roofline (eq. cost(r_j): node visits and triangle
tests per ray) and the per-phase budget of the batched kernel; here they are
checked against what they must satisfy whatever the scene: one count per ray
cast, lanes and pairs bounded by the warp width, one packet per packet_rays
rays of an environment, and a count_work launch returning the same results
as the uncounted one.
"""

import numpy as np
import pytest

import synth
from synth import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
fgl = pytest.importorskip("paper_2509_17390_gb300")


def _cast(scene, sensor, P, opts):
    poses = torch.from_numpy(np.ascontiguousarray(P, np.float32)).cuda()
    n = P.shape[0] * sensor.n_rays
    r = torch.empty(n, dtype=torch.float32, device="cuda")
    i = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    fgl.cast_batched([(scene, sensor, poses, 60.0, r, i)], opts)
    fgl.sync()
    return r, i


@pytest.mark.parametrize("packet", [32, 96])
def test_phase_counters_are_consistent(packet):
    w = workloads.indoor_scan(2)
    scene = fgl.Scene(w.verts, w.tris)
    sensor = fgl.Sensor.from_table(synth.grid_sensor(16, -15, 15, 360))
    P = synth.sample_free_pose(np.random.default_rng(5), w.obstacles, 6, upright=False)
    ref = _cast(scene, sensor, P, fgl.BatchOpts(packet_rays=packet))
    fgl.work_phase_counters()                                   # reset
    got = _cast(scene, sensor, P, fgl.BatchOpts(packet_rays=packet, count_work=1))
    c = fgl.work_phase_counters()
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])
    n = P.shape[0] * sensor.n_rays
    assert c["rays"] == n
    assert c["node_visits"] >= n                                # every ray visits the root
    assert 0 < c["active_lane_iterations"] <= 32 * c["warp_iterations"]
    assert c["node_visits"] <= c["active_lane_iterations"]      # at most one visit a lane a step
    assert c["tri_tests"] <= 32 * c["tri_rounds"]
    assert c["tri_rounds"] <= c["warp_iterations"] * max(1, (24 * 32 + 31) // 32)
    assert c["packets"] == P.shape[0] * -(-sensor.n_rays // packet)
    assert fgl.work_phase_counters()["rays"] == 0               # read and reset


def test_l2_probe_runs_and_checks_arguments():
    buf = torch.ones(1 << 20, dtype=torch.float32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    fgl.probe_l2_read(buf, 3, sink)
    torch.cuda.synchronize()
    assert int(sink.item()) == 0                                # the sink is written only in a corner case
    L = fgl.lib()
    for args in ((buf.data_ptr() + 4, 1 << 16, 1), (buf.data_ptr(), 100, 1), (buf.data_ptr(), 1 << 16, 0),
                 (None, 1 << 16, 1)):
        assert L.fgl_probe_l2_read(args[0], args[1], args[2], sink.data_ptr(), None) == fgl.FGL_ERR_INVALID
