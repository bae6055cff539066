"""Pins for the oracle's Gaussian stream (oracle.rng) -- CPU only.

What fixes each part, independently of the oracle's own code:
* Philox words: the published Random123 known-answer vectors.
* log / cos / sin: float64 libm on the same FP32 arguments (error bounds in ulp).
* Box-Muller: float64 Box-Muller on the same uniforms; distribution moments and a
  Kolmogorov-Smirnov test against the standard normal CDF.
"""

import math
import os

import numpy as np
import pytest
import scipy.stats

from oracle import rng


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            rows.append([int(t, 16) for t in line.split()])
    return rows


def test_philox_known_answers(golden_dir):
    rows = _kat(golden_dir)
    assert len(rows) == 3
    for r in rows:
        c, k, o = r[0:4], r[4:6], r[6:10]
        out = rng.philox4x32_10(*[np.array([x], dtype=np.uint64) for x in c], k[0], k[1])
        assert [int(w[0]) for w in out] == o


def test_philox_vectorised_matches_scalar_calls():
    c0 = np.arange(5, dtype=np.uint64)
    outs = rng.philox4x32_10(c0, c0 * 7, c0 * 11, c0 * 13, 0x12345678, 0x9ABCDEF0)
    for i in range(5):
        one = rng.philox4x32_10(*[np.array([int(c0[i]) * m], dtype=np.uint64) for m in (1, 7, 11, 13)],
                                0x12345678, 0x9ABCDEF0)
        assert all(int(outs[t][i]) == int(one[t][0]) for t in range(4))


def test_uniforms_are_odd_multiples_in_open_interval():
    w = np.array([0, 1, 255, 256, 0x7FFFFFFF, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = rng.uniform24(w)
    k = (u.astype(np.float64) * 2.0 ** 24)
    assert np.all(k == np.round(k)) and np.all(k.astype(np.int64) % 2 == 1)
    assert np.all(u > 0) and np.all(u < 1)
    assert float(u[0]) == 2.0 ** -24 and float(u[5]) == 1.0 - 2.0 ** -24


def _ulp32(x):
    x = np.abs(np.asarray(x, dtype=np.float64))
    e = np.floor(np.log2(np.maximum(x, 2.0 ** -126)))
    return 2.0 ** (e - 23)


def test_log_f32_within_two_ulp_of_libm():
    k = np.unique(np.concatenate([np.arange(1, 1 << 14, 2), np.arange((1 << 24) - (1 << 14) + 1, 1 << 24, 2),
                                  np.random.default_rng(0).integers(0, 1 << 23, 200000) * 2 + 1]))
    u = (k.astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    got = rng.log_f32(u).astype(np.float64)
    ref = np.log(u.astype(np.float64))
    err = np.abs(got - ref) / _ulp32(ref)
    assert err.max() <= 2.0, err.max()


def test_cossin_within_two_ulp_absolute():
    k = np.random.default_rng(1).integers(0, 1 << 23, 400000) * 2 + 1
    k = np.concatenate([k, [1, (1 << 24) - 1, 1 << 22, (1 << 22) + 1, 3 << 22]])
    u = (k.astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)
    c, s = rng.cossin_2pi_f32(u)
    th = 2.0 * math.pi * u.astype(np.float64)
    # absolute error in units of 2^-24 (the ulp of values near 1)
    assert np.abs(c - np.cos(th)).max() <= 2.0 * 2.0 ** -24
    assert np.abs(s - np.sin(th)).max() <= 2.0 * 2.0 ** -24


def test_box_muller_matches_double_precision_transform():
    rs = np.random.default_rng(2)
    wa = rs.integers(0, 1 << 32, 300000, dtype=np.uint64).astype(np.uint32)
    wb = rs.integers(0, 1 << 32, 300000, dtype=np.uint64).astype(np.uint32)
    n0, n1 = rng.box_muller_f32(wa, wb)
    ua = rng.uniform24(wa).astype(np.float64)
    ub = rng.uniform24(wb).astype(np.float64)
    rho = np.sqrt(-2.0 * np.log(ua))
    r0 = rho * np.cos(2 * np.pi * ub)
    r1 = rho * np.sin(2 * np.pi * ub)
    # a few ulp of rho: errors of log (2 ulp), sqrt (0.5), cos/sin (2^-23 abs), product (0.5)
    tol = 4.0 * _ulp32(rho) + rho * 2.0 ** -22
    assert np.all(np.abs(n0 - r0) <= tol)
    assert np.all(np.abs(n1 - r1) <= tol)


def test_omega_distribution():
    om = rng.omega(12345, 3, 1, np.arange(200000, dtype=np.int64), 8).astype(np.float64)
    flat = om.ravel()
    n = flat.size
    assert abs(flat.mean()) < 5.0 / math.sqrt(n)
    assert abs(flat.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(scipy.stats.kurtosis(flat, fisher=False) - 3.0) < 0.05
    assert scipy.stats.kstest(flat, "norm").pvalue > 1e-4
    c = np.corrcoef(om.T)
    assert np.abs(c - np.eye(8)).max() < 6.0 / math.sqrt(om.shape[0])


def test_omega_keys_separate_streams_and_rows_are_independent_of_batch():
    rows = np.array([0, 1, 2, 1 << 33, (1 << 40) + 5], dtype=np.int64)
    full = rng.omega(7, 0, 2, rows, 13)
    for i, r in enumerate(rows):
        one = rng.omega(7, 0, 2, np.array([r]), 13)
        assert np.array_equal(one[0], full[i])
    # a different mode, tensor or seed gives a different stream
    assert not np.array_equal(full, rng.omega(7, 0, 3, rows, 13))
    assert not np.array_equal(full, rng.omega(7, 1, 2, rows, 13))
    assert not np.array_equal(full, rng.omega(8, 0, 2, rows, 13))
    # columns are prefixes: fewer columns give the leading block
    assert np.array_equal(rng.omega(7, 0, 2, rows, 5), full[:, :5])


def test_round_bf16_ties_to_even():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5 - 2 ** -9, 3.0e-3], dtype=np.float32)
    got = rng.round_bf16(vals)
    assert got[0] == 1.0
    assert got[1] == 1.0                       # tie -> even mantissa
    assert got[2] == 1.0 + 4 * 2 ** -8         # tie -> even mantissa (rounds up)
    assert np.all(np.abs(got - vals) <= np.abs(vals) * 2.0 ** -8)


@pytest.mark.parametrize("mode", [0, 15])
def test_stream_id_limits(mode):
    assert rng.stream_id(5, mode) == (5 << 4) | mode
    with pytest.raises(ValueError):
        rng.stream_id(0, 16)


def test_omega_columns_equal_the_full_draw():
    from oracle import rng as r

    rows = np.arange((1 << 32) - 50, (1 << 32) + 50, dtype=np.int64)
    full = r.omega(11, 7, 2, rows, 64)
    cols = [63, 0, 17, 18, 19, 20, 5]
    sub = r.omega_columns(11, 7, 2, rows, cols)
    assert np.array_equal(full[:, cols].view(np.uint32), sub.view(np.uint32))
