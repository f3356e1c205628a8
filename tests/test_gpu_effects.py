"""GPU parity of the optional sensor effects (seeded dropout and range noise
applied to cast returns, fgl_apply_sensor_effects) against the FP64 oracle.

Contract: the random decisions are exact -- which returns are dropped, hit or
miss, and every triangle id, bit for bit; noisy ranges agree within the
float32 rounding of t + (sigma0 + sigma1 t) n: 6e-7 of the range (a few ulp)
plus 5e-6 of the noise scale (n carries a few ulp of logf, sqrtf and cospif
and is at most sqrt(2 ln 2^24) = 5.8 in size).
"""

import numpy as np
import pytest

import oracle
import synth
from synth import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
fgl = pytest.importorskip("paper_2509_17390_gb300")


def cast_walk(n_env, seed=2):
    w = workloads.batched_walk(seed, n_env=n_env, n_steps=2)
    scene = fgl.Scene(w.verts, w.tris)
    sensor = fgl.Sensor.from_table(w.sensor)
    poses = torch.from_numpy(w.poses[1]).cuda()
    n = n_env * sensor.n_rays
    r = torch.empty(n, dtype=torch.float32, device="cuda")
    i = torch.empty(n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    fgl.cast_batched([(scene, sensor, poses, w.max_range, r, i)])
    fgl.sync()
    return r, i, w.max_range


def check(r0, i0, n_env, max_range, **fx):
    r, i = r0.clone(), i0.clone()
    fgl.apply_sensor_effects(r, i, n_env, max_range=max_range, **fx)
    fgl.sync()
    ro, io, dro = oracle.sensor_effects(r0.cpu().numpy(), i0.cpu().numpy(), n_env, max_range=max_range, **fx)
    gr, gi = r.cpu().numpy(), i.cpu().numpy()
    assert np.array_equal(gi, io)                                     # dropout and misses: exact
    miss = io < 0
    assert np.all(gr[miss] == np.float32(max_range))
    t_in = r0.cpu().numpy().astype(np.float64)
    sig = fx.get("sigma0", 0.0) + fx.get("sigma1", 0.0) * t_in
    tol = 6e-7 * np.maximum(np.abs(ro.astype(np.float64)), 1.0) + 5e-6 * sig
    assert np.all(np.abs(gr.astype(np.float64) - ro)[~miss] <= tol[~miss])
    return dro


@pytest.mark.parametrize("fx", [dict(seed=1, drop_prob=0.3),
                                dict(seed=2, step=7, sigma0=0.02, sigma1=0.002),
                                dict(seed=(3 << 40) | 5, step=1, env_offset=100, drop_prob=0.05,
                                     sigma0=0.05, sigma1=0.01),
                                dict(seed=4, drop_prob=1.0), dict(seed=4)])
def test_effects_match_oracle(fx):
    r0, i0, R = cast_walk(64)
    dro = check(r0, i0, 64, R, **fx)
    hits = (i0 >= 0).cpu().numpy()
    if fx.get("drop_prob", 0) == 1.0:
        assert np.array_equal(dro == 1, hits)


def test_effects_per_chunk_equal_whole_and_full_size():
    """The bench-size batch (4096 environments x 5760 rays) against the
    oracle, and the same effects applied in two chunks (env_offset) equal to
    applying them once."""
    r0, i0, R = cast_walk(4096)
    fx = dict(seed=77, step=3, drop_prob=0.1, sigma0=0.01, sigma1=0.001)
    check(r0, i0, 4096, R, **fx)
    n_rays = r0.numel() // 4096
    whole_r, whole_i = r0.clone(), i0.clone()
    fgl.apply_sensor_effects(whole_r, whole_i, 4096, max_range=R, **fx)
    a_r, a_i = r0[:1000 * n_rays].clone(), i0[:1000 * n_rays].clone()
    b_r, b_i = r0[1000 * n_rays:].clone(), i0[1000 * n_rays:].clone()
    fgl.apply_sensor_effects(a_r, a_i, 1000, max_range=R, **fx)
    fgl.apply_sensor_effects(b_r, b_i, 3096, max_range=R, env_offset=1000, **fx)
    fgl.sync()
    assert torch.equal(torch.cat([a_r, b_r]), whole_r) and torch.equal(torch.cat([a_i, b_i]), whole_i)


def test_effects_argument_errors():
    r = torch.zeros(10, device="cuda")
    i = torch.zeros(10, dtype=torch.int32, device="cuda")
    for bad in (dict(drop_prob=1.5), dict(drop_prob=-0.1), dict(sigma0=-1.0), dict(sigma1=float("nan")),
                dict(max_range=0.0), dict(env_offset=-1)):
        kw = dict(seed=1, max_range=10.0)
        kw.update(bad)
        with pytest.raises(fgl.FglError) as e:
            fgl.apply_sensor_effects(r, i, 2, **kw)
        assert e.value.status == fgl.FGL_ERR_INVALID
