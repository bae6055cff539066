"""Gaussian test matrices Omega_j for the randomized range finder -- oracle side.

Test infrastructure only (see ``oracle/__init__``).

The paper draws Omega_j with i.i.d. N(0,1) entries (Sec. 2.4) and notes that the
entries need not be stored but can be generated on the fly (Sec. 3.1, after
Alg. 2).  It fixes nothing else, so this library specifies the stream; both the
CUDA path and this file implement the specification independently:

* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), published round multipliers
  0xD2511F53 / 0xCD9E8D57 and Weyl key increments 0x9E3779B9 / 0xBB67AE85.
* key     = (lo32(seed), hi32(seed))
* counter = (col // 4, lo32(row), hi32(row), (tensor_id << 4) | mode)
  where ``row`` is the Kolda column index of the mode-``mode`` unfolding of the
  tensor being sketched and ``col`` is the column of Omega.
* uniform from a 32-bit word w:  u = float32((w >> 8) | 1) * 2^-24, an odd
  multiple of 2^-24 in (0, 1), exact in FP32.
* Box-Muller on the word pairs (w0, w1) and (w2, w3):
      rho = sqrt(-2 log u_a),  n_even = rho cos(2 pi u_b),  n_odd = rho sin(2 pi u_b)
  evaluated in FP32 with one rounding per elementary operation (no fused
  multiply-add), correctly rounded division and square root, and this module's
  own log and sin/cos:
    - log: u = m 2^e with m in (sqrt(1/2), sqrt(2)], log m = 2 atanh(s),
      s = (m-1)/(m+1), atanh by its Taylor series to s^9; e ln2 with ln2 split
      into a 15-bit head and a tail (Cody-Waite).
    - cos/sin(2 pi u): quadrant q = round(4u), r = u - q/4 in [-1/8, 1/8] (exact),
      Taylor series of sin(2 pi r) to r^9 and cos(2 pi r) to r^10, then the
      quadrant rotation.
  Ω entry (row, 4k + t) is n_t of the Philox call with counter word 0 = k.
"""

import math

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

F32 = np.float32


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 block function, vectorised over equal-shape uint32 arrays.

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 (64-bit products),
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is bumped by the
    Weyl constants.  Ten rounds.  Returns four uint32 arrays.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0)), lo1, (hi0 ^ c3 ^ np.uint64(k1)), lo0
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def uniform24(w):
    """u = ((w >> 8) | 1) * 2^-24 as FP32 (exact)."""
    w = np.asarray(w, dtype=np.uint32)
    return ((w >> np.uint32(8)) | np.uint32(1)).astype(F32) * F32(2.0 ** -24)


# ---- FP32 log by argument reduction + atanh series ---------------------------------
_SQRT2 = F32(math.sqrt(2.0))
_LN2_HI = F32(0.693145751953125)                 # 0x3F317200: 15 significant bits
_LN2_LO = F32(math.log(2.0) - 0.693145751953125)
_L3 = F32(2.0 / 3.0)
_L5 = F32(2.0 / 5.0)
_L7 = F32(2.0 / 7.0)
_L9 = F32(2.0 / 9.0)
_L11 = F32(2.0 / 11.0)


def log_f32(u):
    """Natural log of positive normal FP32 values, one rounding per operation."""
    u = np.asarray(u, dtype=F32)
    bits = u.view(np.uint32)
    e = (bits >> np.uint32(23)).astype(np.int32) - 127
    m = ((bits & np.uint32(0x7FFFFF)) | np.uint32(0x3F800000)).view(F32)
    big = m > _SQRT2
    m = np.where(big, m * F32(0.5), m).astype(F32)
    e = e + big.astype(np.int32)
    f = m - F32(1.0)
    s = f / (m + F32(1.0))
    z = s * s
    p = _L11
    p = p * z + _L9
    p = p * z + _L7
    p = p * z + _L5
    p = p * z + _L3
    t = s * z
    t = t * p
    logm = (s + s) + t
    ef = e.astype(F32)
    return (ef * _LN2_HI + (ef * _LN2_LO + logm)).astype(F32)


# ---- FP32 cos / sin of 2*pi*u by quadrant reduction + Taylor series -----------------
_TAU = 2.0 * math.pi
_S1 = F32(_TAU)
_S3 = F32(-(_TAU ** 3) / 6.0)
_S5 = F32((_TAU ** 5) / 120.0)
_S7 = F32(-(_TAU ** 7) / 5040.0)
_S9 = F32((_TAU ** 9) / 362880.0)
_C2 = F32(-(_TAU ** 2) / 2.0)
_C4 = F32((_TAU ** 4) / 24.0)
_C6 = F32(-(_TAU ** 6) / 720.0)
_C8 = F32((_TAU ** 8) / 40320.0)
_C10 = F32(-(_TAU ** 10) / 3628800.0)


def cossin_2pi_f32(u):
    """(cos 2 pi u, sin 2 pi u) for FP32 u in (0, 1), one rounding per operation."""
    u = np.asarray(u, dtype=F32)
    q = np.rint(u * F32(4.0)).astype(F32)          # no ties: 4u is never a half-integer
    r = u - q * F32(0.25)                            # exact, |r| <= 1/8
    z = r * r
    ps = _S9
    ps = ps * z + _S7
    ps = ps * z + _S5
    ps = ps * z + _S3
    ps = ps * z + _S1
    s = r * ps
    pc = _C10
    pc = pc * z + _C8
    pc = pc * z + _C6
    pc = pc * z + _C4
    pc = pc * z + _C2
    c = pc * z + F32(1.0)
    qi = q.astype(np.int64) & 3
    cos_t = np.select([qi == 0, qi == 1, qi == 2], [c, -s, -c], s).astype(F32)
    sin_t = np.select([qi == 0, qi == 1, qi == 2], [s, c, -s], -c).astype(F32)
    return cos_t, sin_t


def box_muller_f32(wa, wb):
    """Two FP32 normals from two Philox words: (rho cos 2 pi u_b, rho sin 2 pi u_b)."""
    ua = uniform24(wa)
    ub = uniform24(wb)
    rho = np.sqrt(log_f32(ua) * F32(-2.0)).astype(F32)
    cs, sn = cossin_2pi_f32(ub)
    return (rho * cs).astype(F32), (rho * sn).astype(F32)


def stream_id(tensor_id, mode):
    if not (0 <= mode < 16):
        raise ValueError("mode must be in [0, 16)")
    if not (0 <= tensor_id < (1 << 28)):
        raise ValueError("tensor_id must be in [0, 2^28)")
    return (int(tensor_id) << 4) | int(mode)


def omega(seed, tensor_id, mode, rows, ell):
    """Omega[rows, 0:ell] as an FP32 array of shape (len(rows), ell).

    ``rows`` are Kolda column indices of the unfolding being sketched.
    """
    rows = np.asarray(rows, dtype=np.int64).ravel()
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    lo = (rows & 0xFFFFFFFF).astype(np.uint64)
    hi = (rows >> 32).astype(np.uint64)
    sid = np.full(rows.shape, stream_id(tensor_id, mode), dtype=np.uint64)
    nq = (ell + 3) // 4
    out = np.empty((rows.size, 4 * nq), dtype=F32)
    for q in range(nq):
        w0, w1, w2, w3 = philox4x32_10(np.full(rows.shape, q, dtype=np.uint64), lo, hi, sid, k0, k1)
        n0, n1 = box_muller_f32(w0, w1)
        n2, n3 = box_muller_f32(w2, w3)
        out[:, 4 * q + 0] = n0
        out[:, 4 * q + 1] = n1
        out[:, 4 * q + 2] = n2
        out[:, 4 * q + 3] = n3
    return out[:, :ell]


def omega_columns(seed, tensor_id, mode, rows, cols):
    """Omega[rows, cols] for a list of column indices; only the Philox counters of those columns
    (col // 4) are evaluated, so single columns of a very long Omega stay cheap."""
    rows = np.asarray(rows, dtype=np.int64).ravel()
    cols = [int(c) for c in cols]
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    lo = (rows & 0xFFFFFFFF).astype(np.uint64)
    hi = (rows >> 32).astype(np.uint64)
    sid = np.full(rows.shape, stream_id(tensor_id, mode), dtype=np.uint64)
    out = np.empty((rows.size, len(cols)), dtype=F32)
    groups = {}
    for j, c in enumerate(cols):
        q = c // 4
        if q not in groups:
            w0, w1, w2, w3 = philox4x32_10(np.full(rows.shape, q, dtype=np.uint64), lo, hi, sid, k0, k1)
            n0, n1 = box_muller_f32(w0, w1)
            n2, n3 = box_muller_f32(w2, w3)
            groups[q] = (n0, n1, n2, n3)
        out[:, j] = groups[q][c % 4]
    return out


def round_bf16(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP32."""
    b = np.asarray(x, dtype=F32).view(np.uint32).astype(np.uint64)
    b = (b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(F32)
