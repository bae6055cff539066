"""Pins of the oracle's reading of the low-precision storage forms (CPU).

* E4M3 decoding: anchor values fixed by the format definition (smallest subnormal 2^-9, largest
  subnormal 7 * 2^-9, smallest normal 2^-6, one, the largest finite 448, the NaN codes), monotone
  codes, sign symmetry, and code-for-code agreement with torch's float8_e4m3fn (a separate
  implementation of the same format).
* The block-scaled layout: the element-to-byte and element-to-scale maps, checked on a buffer
  built by hand, with and without fibre padding.
* The quantizer used to build test inputs: nearest representable value (error at most half a
  code step), saturation, all-zero blocks.
"""

import numpy as np
import pytest

from oracle.storage import e4m3_values, fp8_dequantize, fp8_layout
from workloads import fp8_quantize_np


def test_e4m3_anchor_values():
    v = e4m3_values()
    assert v[0x00] == 0.0 and np.signbit(v[0x80]) and v[0x80] == 0.0
    assert v[0x01] == 2.0 ** -9
    assert v[0x07] == 7 * 2.0 ** -9
    assert v[0x08] == 2.0 ** -6
    assert v[0x38] == 1.0
    assert v[0x7E] == 448.0 and v[0xFE] == -448.0
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF])
    pos = v[:0x7F]
    assert np.all(np.diff(pos) > 0)
    assert np.array_equal(v[0x80:0xFF], -pos)


def test_e4m3_matches_torch_float8():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8_e4m3fn")
    t = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    v = e4m3_values()
    fin = ~np.isnan(v)
    assert np.array_equal(np.isnan(t), ~fin)
    assert np.array_equal(v[fin], t[fin])


@pytest.mark.parametrize("dims", [(16, 3, 2), (20, 7), (8, 5, 3), (128, 2)])
def test_fp8_layout_and_dequantize_by_hand(dims):
    ld, off, nscales, total = fp8_layout(dims)
    I0 = dims[0]
    m = int(np.prod(dims[1:]))
    assert ld % 16 == 0 and ld - I0 < 16 and ld >= I0
    assert off % 16 == 0 and off >= ld * m and nscales == -(-(ld * m) // 128)
    rs = np.random.default_rng(1)
    buf = np.zeros(total, dtype=np.uint8)
    codes = rs.integers(0, 0x7F, size=ld * m).astype(np.uint8) | (rs.integers(0, 2, size=ld * m) << 7).astype(np.uint8)
    buf[:ld * m] = codes
    scales = (2.0 ** rs.integers(-3, 4, size=nscales) * rs.uniform(1, 2, size=nscales)).astype(np.float32)
    buf[off:off + 4 * nscales] = scales.view(np.uint8)
    X = fp8_dequantize(buf, dims)
    v = e4m3_values()
    for idx in [(0,) * len(dims), tuple(d - 1 for d in dims), tuple(d // 2 for d in dims)]:
        i = idx[0]
        p = 0
        stride = 1
        for n in range(1, len(dims)):
            p += idx[n] * stride
            stride *= dims[n]
        e = i + ld * p
        want = np.float32(np.float32(v[codes[e]]) * scales[e // 128])
        assert X[idx] == float(want), (idx, X[idx], want)


def test_quantizer_is_nearest_and_saturates():
    rs = np.random.default_rng(2)
    X = (rs.standard_normal((24, 9, 5)) * np.exp(rs.uniform(-6, 6, (24, 9, 5)))).astype(np.float32)
    X[:, 0, 0] = 0.0                                   # a zero fibre
    buf = fp8_quantize_np(X)
    Xd = fp8_dequantize(buf, X.shape)
    ld, off, nscales, _ = fp8_layout(X.shape)
    scales = buf[off:off + 4 * nscales].view(np.float32)
    m = int(np.prod(X.shape[1:]))
    e = (np.arange(X.shape[0])[:, None] + ld * np.arange(m)[None, :]).ravel(order="F")
    s = scales[e // 128].reshape(X.shape, order="F").astype(np.float64)
    # every block reaches +-448 (up to the FP32 rounding of the scale) and no element exceeds it
    y = np.abs(X.astype(np.float64)) / s
    assert np.all(y <= 448.0 * (1 + 2.0 ** -22))
    # nearest code: the error is at most half a step of the E4M3 grid at that magnitude
    step = np.where(y < 2.0 ** -6, 2.0 ** -9, 2.0 ** (np.floor(np.log2(np.maximum(y, 2.0 ** -6))) - 3))
    err = np.abs(Xd / s - np.clip(X / s, -448, 448)) - 0.5 * step
    assert np.all(err <= 1e-6 * step)
    assert np.all(Xd[:, 0, 0] == 0.0)


def test_fp8_rows_equal_the_full_dequantization():
    from oracle.storage import fp8_dequantize_rows
    from oracle.tensor import unfold

    rs = np.random.default_rng(3)
    X = rs.standard_normal((20, 7, 5)).astype(np.float32)
    buf = fp8_quantize_np(X)
    full = unfold(fp8_dequantize(buf, X.shape), 0)
    rows = [0, 7, 19]
    assert np.array_equal(fp8_dequantize_rows(buf, X.shape, rows), full[rows])
