"""Pins of the oracle's optional sensor effects (seeded return dropout and
range noise on top of eq. t_j*; the paper leaves sensor physics to future
work, Sec. VI).  The generator is pinned to Philox-4x32-10's published
known-answer vectors; dropout and noise to their distributions (binomial
and normal laws, checked against their sampling error); the rest to
invariants (misses untouched, identity without effects, clamping,
determinism per (seed, step, environment, ray))."""

import json
import os

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_known_answer_vectors():
    kat = json.load(open(os.path.join(HERE, "golden", "philox4x32_10_kat.json")))
    for v in kat["vectors"]:
        ctr = [int(x, 16) for x in v["ctr"]]
        key = [int(x, 16) for x in v["key"]]
        out = [int(x, 16) for x in v["out"]]
        assert oracle.philox4x32(ctr, key, kat["rounds"]).tolist() == out


def _returns(n_env, n_rays, rng, hit_frac=0.8, max_range=50.0):
    r = rng.uniform(0.5, 40.0, n_env * n_rays).astype(np.float32)
    t = rng.integers(0, 10 ** 6, n_env * n_rays).astype(np.int32)
    miss = rng.random(n_env * n_rays) > hit_frac
    r[miss] = np.float32(max_range)
    t[miss] = -1
    return r, t


def test_dropout_is_binomial_and_only_on_hits():
    rng = np.random.default_rng(0)
    r, t = _returns(64, 4000, rng)
    for p in (0.05, 0.3, 0.9):
        rr, tt, dr = oracle.sensor_effects(r, t, 64, seed=11, drop_prob=p, max_range=50.0)
        hits = t >= 0
        k = int(dr[hits].sum())
        n = int(hits.sum())
        assert abs(k - p * n) <= 5 * np.sqrt(n * p * (1 - p))          # 5 sigma of the binomial law
        assert not dr[~hits].any()
        assert np.all(tt[dr == 1] == -1) and np.all(rr[dr == 1] == np.float32(50.0))
        assert np.array_equal(rr[hits & (dr == 0)], r[hits & (dr == 0)])  # no noise asked
    # p = 0 keeps everything, p = 1 drops every hit
    assert not oracle.sensor_effects(r, t, 64, seed=11, drop_prob=0.0)[2].any()
    assert np.array_equal(oracle.sensor_effects(r, t, 64, seed=11, drop_prob=1.0)[2] == 1, t >= 0)


def test_noise_is_normal_with_the_stated_sigma():
    from scipy import stats
    rng = np.random.default_rng(1)
    r, t = _returns(50, 4000, rng, hit_frac=1.0, max_range=1e4)
    sig0, sig1 = 0.02, 0.001
    rr, tt, _ = oracle.sensor_effects(r, t, 50, seed=5, step=3, sigma0=sig0, sigma1=sig1, max_range=1e4)
    z = (rr.astype(np.float64) - r) / (sig0 + sig1 * r.astype(np.float64))
    n = len(z)
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.std() - 1.0) < 5 * np.sqrt(0.5 / n) + 1e-4
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert np.array_equal(tt, t)


def test_noise_clamps_and_leaves_misses():
    r = np.array([0.001, 49.999, 50.0, 10.0], np.float32)
    t = np.array([3, 4, -1, 5], np.int32)
    rr, tt, dr = oracle.sensor_effects(r, t, 1, seed=2, sigma0=5.0, max_range=50.0)
    assert np.all((rr >= 0) & (rr <= np.float32(50.0)))
    assert rr[2] == np.float32(50.0) and tt[2] == -1 and not dr.any()
    big = oracle.sensor_effects(np.full(4000, 1.0, np.float32), np.zeros(4000, np.int32), 1, seed=2,
                                sigma0=5.0, max_range=3.0)[0]
    assert (big == 0).any() and (big == np.float32(3.0)).any()      # both clamps reached


def test_effects_are_deterministic_per_counter():
    rng = np.random.default_rng(3)
    r, t = _returns(8, 500, rng)
    kw = dict(drop_prob=0.4, sigma0=0.05, max_range=50.0)
    a = oracle.sensor_effects(r, t, 8, seed=9, step=1, **kw)
    b = oracle.sensor_effects(r, t, 8, seed=9, step=1, **kw)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    for other in (dict(seed=10, step=1), dict(seed=9, step=2)):
        c = oracle.sensor_effects(r, t, 8, **other, **kw)
        assert not np.array_equal(a[2], c[2])
    # environment e of a batch starting at env_offset o draws what environment
    # o + e draws alone
    full = oracle.sensor_effects(r, t, 8, seed=9, step=1, **kw)
    part = oracle.sensor_effects(r[3 * 500:], t[3 * 500:], 5, seed=9, step=1, env_offset=3, **kw)
    assert all(np.array_equal(x[3 * 500:], y) for x, y in zip(full, part))
    # no effects: identity
    ident = oracle.sensor_effects(r, t, 8, seed=9)
    assert np.array_equal(ident[0], r) and np.array_equal(ident[1], t)
