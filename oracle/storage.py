"""Low-precision storage forms of the input tensor -- oracle side (test infrastructure only).

The method itself computes on real numbers; a tensor stored in a low-precision form is read as
the real tensor its bytes denote.  This module writes that reading out from the format
definitions, independently of the CUDA library:

* E4M3 (OCP 8-bit floating point, "FP8 E4M3"): 1 sign bit, 4 exponent bits with bias 7, 3
  mantissa bits; exponent field 0 holds the subnormals m 2^-9; there are no infinities and the
  codes S.1111.111 are NaN, so the largest finite magnitude is 1.75 * 2^8 = 448.
* Block-scaled E4M3 tensor (``RH_FP8_E4M3``): the codes column-major with the mode-1 fibres at a
  stride of ld = I_1 rounded up to a multiple of 16 bytes, then, from the next 16-byte boundary,
  one FP32 scale per 128 consecutive bytes of that code array.  Element (i, p) of X_(1) is the
  FP32 product fl32(value(code[i + ld p]) * scale[(i + ld p) // 128]).

Parity of the GPU's FP8 path is stated against the tensor this module returns.
"""

import numpy as np

E4M3_MAX = 448.0


def e4m3_values():
    """Real values of the 256 E4M3 codes (float64; NaN for the two NaN codes)."""
    out = np.empty(256, dtype=np.float64)
    for code in range(256):
        sign = -1.0 if code & 0x80 else 1.0
        e = (code >> 3) & 0xF
        m = code & 0x7
        if e == 0xF and m == 0x7:
            out[code] = np.nan
        elif e == 0:
            out[code] = sign * m * 2.0 ** -9            # subnormal: 2^(1 - 7) * m / 8
        else:
            out[code] = sign * (1.0 + m / 8.0) * 2.0 ** (e - 7)
    return out


def fp8_layout(dims):
    """(ld, scale_offset, nscales, total_bytes) of a block-scaled E4M3 tensor with sizes dims."""
    dims = [int(v) for v in dims]
    m = int(np.prod(dims[1:], dtype=np.int64)) if len(dims) > 1 else 1
    ld = -(-dims[0] // 16) * 16
    data = ld * m
    off = -(-data // 16) * 16
    nscales = -(-data // 128)
    return ld, off, nscales, off + 4 * nscales


def fp8_dequantize(buf, dims):
    """The real tensor (float64 ndarray of shape dims) denoted by a block-scaled E4M3 buffer."""
    buf = np.asarray(buf, dtype=np.uint8).ravel()
    dims = [int(v) for v in dims]
    ld, off, nscales, total = fp8_layout(dims)
    if buf.size != total:
        raise ValueError(f"buffer has {buf.size} bytes, the layout needs {total}")
    mcols = int(np.prod(dims[1:], dtype=np.int64)) if len(dims) > 1 else 1
    codes = buf[:ld * mcols]
    scales = buf[off:off + 4 * nscales].view(np.float32)
    vals = e4m3_values()[codes].astype(np.float32)                     # exact in FP32
    s = scales[np.arange(ld * mcols) // 128]
    x = (vals * s).astype(np.float32)                                  # FP32 product, ties to even
    X1 = np.reshape(x, (ld, mcols), order="F")[:dims[0], :]
    return np.reshape(X1.astype(np.float64), dims, order="F")


def fp8_dequantize_rows(buf, dims, rows):
    """Rows ``rows`` of the mode-1 unfolding of the tensor a block-scaled E4M3 buffer denotes
    (float64 array len(rows) x prod(dims[1:])), read without expanding the rest of the tensor."""
    buf = np.asarray(buf, dtype=np.uint8).ravel()
    ld, off, nscales, total = fp8_layout(dims)
    if buf.size != total:
        raise ValueError(f"buffer has {buf.size} bytes, the layout needs {total}")
    mcols = int(np.prod([int(v) for v in dims[1:]], dtype=np.int64)) if len(dims) > 1 else 1
    scales = buf[off:off + 4 * nscales].view(np.float32)
    table = e4m3_values().astype(np.float32)
    out = np.empty((len(rows), mcols), dtype=np.float64)
    p = np.arange(mcols, dtype=np.int64)
    for j, i in enumerate(rows):
        e = int(i) + ld * p
        out[j] = (table[buf[e]] * scales[e // 128]).astype(np.float32)
    return out
