"""Seeded synthetic input tensors shared by the tests, the bench and the oracle runs.

This module holds no step of the compression method: it only builds input
tensors (and their documented shapes).  Both the CUDA path and the oracle consume
the bytes it produces, so the two sides always see identical inputs.

Workloads (sizes follow the paper's experiments and the library's benchmark set):

* ``hilbert(dims, offset)``: X(i_1..i_d) = 1 / (i_1 + ... + i_d + offset) with
  0-based indices.  offset = d gives the paper's 1-based Hilbert tensor (Sec. 6.1,
  Eq. hilbert); offset = 1 gives the 200^3 tensor 1/(i+j+k+1).
* ``lowrank_plus_noise``: core of N(0,1) entries scaled by decay^(i_1+...+i_d)
  (0-based), factors U_n = orthonormal Q of an N(0,1) I_n x r_n matrix, plus
  N(0,1) noise rescaled to ``noise_rel`` times the Frobenius norm of the signal.
* ``zipf_coo``: sparse count tensor with per-mode Zipf(s) coordinates,
  deduplicated, values log(1 + Poisson(lam) + 1).

Tensors are returned column-major (index 1 fastest) as numpy arrays of shape
(I_1, ..., I_d) with Fortran order, or as torch tensors holding that flat buffer.
"""

import numpy as np


def hilbert(dims, offset, dtype=np.float64):
    """Hilbert-type tensor 1/(sum of 0-based indices + offset), Fortran order."""
    dims = [int(x) for x in dims]
    s = np.zeros(dims, dtype=np.float64, order="F")
    for n, I in enumerate(dims):
        shape = [1] * len(dims)
        shape[n] = I
        s = s + np.arange(I, dtype=np.float64).reshape(shape)
    return np.asfortranarray((1.0 / (s + float(offset))).astype(dtype))


def lowrank_plus_noise_np(dims, core_dims, decay, noise_rel, seed, dtype=np.float64):
    """Small-size numpy version of the low-rank + noise workload (CPU tests)."""
    rs = np.random.default_rng(seed)
    d = len(dims)
    core = rs.standard_normal(core_dims)
    for n, r in enumerate(core_dims):
        shape = [1] * d
        shape[n] = r
        core = core * (float(decay) ** np.arange(r, dtype=np.float64)).reshape(shape)
    U = [np.linalg.qr(rs.standard_normal((int(dims[n]), int(core_dims[n]))))[0] for n in range(d)]
    X = core
    for n in range(d):
        X = np.moveaxis(np.tensordot(U[n], X, axes=([1], [n])), 0, n)
    if noise_rel > 0:
        E = rs.standard_normal(dims)
        E *= noise_rel * np.linalg.norm(X) / np.linalg.norm(E)
        X = X + E
    return np.asfortranarray(X.astype(dtype))


def lowrank_plus_noise_torch(dims, core_dims, decay, noise_rel, seed, dtype, device):
    """Large-size version built with torch on ``device``; returns a flat column-major tensor.

    Steps: factors and core from a CPU generator seeded with ``seed``; the signal
    G x_1 U_1 ... x_d U_d by successive mode products in float64 on the device
    (float32 when the tensor exceeds 2^28 elements); noise from a generator on
    ``device`` seeded with ``seed + 1``.  The flat buffer is X(i_1, ..., i_d) at
    i_1 + I_1 (i_2 + I_2 (...)).
    """
    import torch

    g = torch.Generator(device="cpu").manual_seed(int(seed))
    d = len(dims)
    core = torch.randn(*core_dims, generator=g, dtype=torch.float64)
    for n, r in enumerate(core_dims):
        shape = [1] * d
        shape[n] = r
        core = core * (float(decay) ** torch.arange(r, dtype=torch.float64)).reshape(shape)
    U = [torch.linalg.qr(torch.randn(int(dims[n]), int(core_dims[n]), generator=g, dtype=torch.float64))[0]
         for n in range(d)]
    N = int(np.prod(dims))
    wdt = torch.float64 if N <= (1 << 28) else torch.float32
    # torch tensors here use C order with reversed axes: T[i_d, ..., i_1] so that the
    # flat buffer is column-major in (i_1..i_d).
    T = core.permute(*reversed(range(d))).contiguous().to(device=device, dtype=wdt)
    for n in range(d):
        ax = d - 1 - n
        Un = U[n].to(device=device, dtype=wdt)
        T = torch.movedim(torch.tensordot(Un, T, dims=([1], [ax])), 0, ax).contiguous()
    X = T.reshape(-1).to(dtype)
    del T
    if noise_rel > 0:
        gd = torch.Generator(device=device).manual_seed(int(seed) + 1)
        E = torch.randn(N, generator=gd, device=device, dtype=torch.float32)
        sig = torch.linalg.vector_norm(X.to(torch.float64))
        en = torch.linalg.vector_norm(E.to(torch.float64))
        X = (X.to(torch.float64 if dtype == torch.float64 else torch.float32)
             + (E * float(noise_rel * sig / en)).to(X.dtype)).to(dtype)
        del E
    return X


def zipf_coo(dims, nnz, s, lam, seed, batch=None):
    """Sparse count tensor: coordinates Zipf(s) per mode (rank k -> index k-1), deduplicated.

    Draws batches of coordinate tuples until ``nnz`` distinct ones exist, keeps
    the first ``nnz`` distinct in draw order, sorts them lexicographically (mode 1
    slowest), values log(1 + Poisson(lam) + 1) in float64 stored as float32.
    Returns (idx int32 array nnz x d, vals float32 array).
    """
    rs = np.random.default_rng(seed)
    dims = [int(x) for x in dims]
    d = len(dims)
    cdfs = []
    for I in dims:
        w = np.arange(1, I + 1, dtype=np.float64) ** (-float(s))
        c = np.cumsum(w)
        cdfs.append(c / c[-1])
    batch = batch or max(1024, nnz // 2)
    keys = np.zeros(0, dtype=np.int64)
    mult = [1] * d
    for n in range(d - 2, -1, -1):
        mult[n] = mult[n + 1] * dims[n + 1]
    while True:
        cols = [np.minimum(np.searchsorted(cdfs[n], rs.random(batch)), dims[n] - 1).astype(np.int64)
                for n in range(d)]
        k = np.zeros(batch, dtype=np.int64)
        for n in range(d):
            k += cols[n] * mult[n]
        keys = np.concatenate([keys, k])
        _, first = np.unique(keys, return_index=True)
        if first.size >= nnz:
            keep = np.sort(first)[:nnz]
            keys = np.sort(keys[keep])
            break
    idx = np.zeros((nnz, d), dtype=np.int32)
    rem = keys.copy()
    for n in range(d):
        idx[:, n] = (rem // mult[n]).astype(np.int32)
        rem = rem % mult[n]
    vals = np.log(1.0 + rs.poisson(lam, nnz).astype(np.float64) + 1.0).astype(np.float32)
    return idx, vals


def batch_recipe(count=512, seed=4, orders=(3, 4, 5), size_range=(16, 96), rank_range=(4, 16)):
    """Shapes and ranks of the batched workload: ``count`` tensors, order uniform in ``orders``, every
    mode size uniform in ``size_range``, every rank uniform in ``rank_range`` capped at the mode size
    (and at the size rule r + p <= prod of the other sizes is left to the caller's clamp).  Each
    tensor i is then ``lowrank_plus_noise`` with core sizes = its ranks, decay 0.9, noise 1e-3 and
    seed ``seed * 100003 + i``.  Returns a list of (dims, ranks, data_seed)."""
    rs = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = int(rs.choice(orders))
        dims = [int(v) for v in rs.integers(size_range[0], size_range[1] + 1, size=d)]
        ranks = [int(min(r, I)) for r, I in zip(rs.integers(rank_range[0], rank_range[1] + 1, size=d), dims)]
        out.append((dims, ranks, int(seed) * 100003 + i))
    return out


# ---- low-precision storage of an input tensor (the form the caller hands over) ---------------
# E4M3 with one FP32 scale per 128 bytes: codes column-major with the mode-1 fibres padded to a
# multiple of 16 bytes, then the scales from the next 16-byte boundary.  Block scale = amax / 448
# in FP32 (1 for an all-zero block), codes = nearest E4M3 value of x / scale (ties to the even
# code), saturated at +-448.

def _e4m3_finite_magnitudes():
    v = []
    for code in range(127):   # 0x00 .. 0x7E; 0x7F is NaN
        e, m = code >> 3, code & 7
        v.append(m * 2.0 ** -9 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7))
    return np.array(v)


def fp8_storage_layout(dims):
    dims = [int(v) for v in dims]
    m = int(np.prod(dims[1:], dtype=np.int64)) if len(dims) > 1 else 1
    ld = -(-dims[0] // 16) * 16
    off = -(-(ld * m) // 16) * 16
    nscales = -(-(ld * m) // 128)
    return ld, m, off, nscales, off + 4 * nscales


def fp8_quantize_np(X):
    """Block-scaled E4M3 buffer (uint8 ndarray) of the numpy tensor X (shape = its sizes)."""
    X = np.asarray(X, dtype=np.float32)
    ld, m, off, nscales, total = fp8_storage_layout(X.shape)
    P = np.zeros((ld, m), dtype=np.float32)
    P[:X.shape[0], :] = np.reshape(X, (X.shape[0], m), order="F")
    flat = np.zeros(nscales * 128, dtype=np.float32)
    flat[:ld * m] = P.ravel(order="F")
    blocks = flat.reshape(nscales, 128)
    amax = np.abs(blocks).max(axis=1)
    scale = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    y = (blocks / scale[:, None]).astype(np.float32).astype(np.float64)
    mag = np.minimum(np.abs(y), 448.0)
    tab = _e4m3_finite_magnitudes()
    hi = np.clip(np.searchsorted(tab, mag), 0, 126)
    lo = np.clip(hi - 1, 0, 126)
    dlo, dhi = mag - tab[lo], tab[hi] - mag
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(pick_hi, hi, lo).astype(np.uint8)
    code = code | np.where(y < 0, 0x80, 0).astype(np.uint8)
    buf = np.zeros(total, dtype=np.uint8)
    buf[:ld * m] = code.ravel()[:ld * m]
    buf[off:] = scale.view(np.uint8)
    return buf


def fp8_quantize_torch(X, dims):
    """Block-scaled E4M3 buffer (uint8 torch tensor on X's device) of the flat column-major
    FP32 torch tensor X with sizes dims (torch's float8_e4m3fn rounding, ties to even)."""
    import torch

    ld, m, off, nscales, total = fp8_storage_layout(dims)
    I0 = int(dims[0])
    buf = torch.zeros(total, dtype=torch.uint8, device=X.device)
    codes = buf[:ld * m].view(m, ld)
    scales = torch.empty(nscales, dtype=torch.float32, device=X.device)
    Xv = X.view(m, I0)
    # columns in slabs so the FP32 temporaries stay small; a slab covers whole 128-byte blocks
    step = max(1, (1 << 26) // ld)
    step = max(128, step // 128 * 128)
    for c0 in range(0, m, step):
        c1 = min(m, c0 + step)
        P = torch.zeros((c1 - c0, ld), dtype=torch.float32, device=X.device)
        P[:, :I0] = Xv[c0:c1]
        flat = P.reshape(-1)
        b0 = c0 * ld // 128
        nb = -(-flat.numel() // 128)
        fpad = torch.zeros(nb * 128, dtype=torch.float32, device=X.device)
        fpad[:flat.numel()] = flat
        blk = fpad.view(nb, 128)
        amax = blk.abs().amax(dim=1)
        sc = torch.where(amax > 0, amax / 448.0, torch.ones_like(amax))
        q = (blk / sc[:, None]).clamp_(-448.0, 448.0).to(torch.float8_e4m3fn).view(torch.uint8).reshape(-1)
        codes.view(-1)[c0 * ld:c1 * ld] = q[:flat.numel()]
        scales[b0:b0 + nb] = sc
    buf[off:] = scales.view(torch.uint8)
    return buf


def bf16_bits_np(X):
    """BF16 bit patterns (uint16, ties to even) of the numpy tensor X in column-major order."""
    x = np.asarray(X, dtype=np.float32).ravel(order="F").view(np.uint32).astype(np.uint64)
    r = (x + 0x7FFF + ((x >> 16) & 1)) >> 16
    return r.astype(np.uint16)


def zipf_coo_torch(dims, nnz, s, lam, seed, device):
    """The ``zipf_coo`` recipe drawn with torch generators on ``device`` (for full-size inputs):
    coordinates Zipf(s) per mode, the first ``nnz`` distinct tuples in draw order, sorted
    lexicographically (mode 1 slowest), values log(1 + Poisson(lam) + 1) in FP64 stored as FP32.
    Returns ([int32 index tensor per mode], FP32 values), all on ``device``."""
    import torch

    dims = [int(x) for x in dims]
    d = len(dims)
    g = torch.Generator(device=device).manual_seed(int(seed))
    cdfs = []
    for I in dims:
        w = torch.arange(1, I + 1, dtype=torch.float64, device=device) ** (-float(s))
        c = torch.cumsum(w, 0)
        cdfs.append(c / c[-1])
    mult = [1] * d
    for n in range(d - 2, -1, -1):
        mult[n] = mult[n + 1] * dims[n + 1]
    batch = max(1 << 20, nnz // 2)
    keys = torch.empty(0, dtype=torch.int64, device=device)
    while True:
        k = torch.zeros(batch, dtype=torch.int64, device=device)
        for n in range(d):
            u = torch.rand(batch, generator=g, dtype=torch.float64, device=device)
            col = torch.clamp(torch.searchsorted(cdfs[n], u), max=dims[n] - 1)
            k += col * mult[n]
        keys = torch.cat([keys, k])
        uniq, inv = torch.unique(keys, return_inverse=True)
        if uniq.numel() >= nnz:
            pos = torch.arange(keys.numel(), device=device)
            first = torch.full((uniq.numel(),), keys.numel(), dtype=torch.int64, device=device)
            first.scatter_reduce_(0, inv, pos, reduce="amin")
            order = torch.argsort(first)[:nnz]
            keys = torch.sort(uniq[order]).values
            break
    idx = []
    rem = keys.clone()
    for n in range(d):
        idx.append((rem // mult[n]).to(torch.int32))
        rem = rem % mult[n]
    lamt = torch.full((nnz,), float(lam), dtype=torch.float64, device=device)
    vals = torch.log(1.0 + torch.poisson(lamt, generator=g) + 1.0).to(torch.float32)
    return idx, vals
