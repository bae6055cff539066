"""Randomized Tucker compression on GB300 (sm_103a).

Python names mirror the C ABI of include/rhosvd.h: ``omega``, ``rhosvd_sketch``,
``orthonormalize``, ``rsthosvd``.  Tensors are torch CUDA tensors holding the flat
column-major buffer of the tensor (index 1 fastest) together with its ``dims``.
Outputs and the workspace are allocated with torch on the tensor's device; every
call runs on the current torch CUDA stream.
"""

import ctypes

from . import _lib
from ._lib import RH_F32, RH_F64, RhError, check, i32_array, i64_array, lib, make_options

__all__ = ["fp8_layout", "omega", "rhosvd_sketch", "orthonormalize", "mode_product", "left_svd", "core_ttm", "tucker_residual",
           "rsthosvd", "rhosvd", "rsthosvd_batched", "RsthosvdBatchedCall", "subset_select", "sp_sthosvd_coo",
           "rhosvd_sketch_coo", "RhError", "version"]


def _torch():
    import torch

    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float64:
        return RH_F64
    if t.dtype == torch.float32:
        return RH_F32
    raise TypeError(f"unsupported dtype {t.dtype}: use float64 or float32")


def _stream(device):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _check_input(X, dims, factor=1):
    torch = _torch()
    if not X.is_cuda:
        raise ValueError("X must be a CUDA tensor")
    if not X.is_contiguous():
        raise ValueError("X must be contiguous (flat column-major buffer)")
    n = 1
    for v in dims:
        n *= int(v)
    if X.numel() != factor * n:
        raise ValueError(f"X has {X.numel()} elements but dims multiply to {n} (x{factor})")
    return torch


_FORMS = {"bf16": 2, "bf16x2": 3, "f32_bf16x2": 4, "fp8_e4m3": 5, "f32_bf16x3": 6}


def _piece_form(pieces):
    """dtype code of a tensor-core input: pieces=2 (split_bf16x2 output), 1 (BF16 bits), "f32"
    (a plain FP32 tensor split on the fly, RH_F32_BF16X2), "f32x3" (split exactly into three pieces,
    RH_F32_BF16X3) or "fp8" (an RH_FP8_E4M3 buffer)."""
    if pieces == "f32":
        return _lib.RH_F32_BF16X2
    if pieces == "f32x3":
        return _lib.RH_F32_BF16X3
    if pieces == "fp8":
        return _lib.RH_FP8_E4M3
    return _lib.RH_BF16X2 if pieces == 2 else _lib.RH_BF16


def version():
    return lib().rh_version().decode()


def fp8_layout(dims):
    """Storage of an RH_FP8_E4M3 tensor with sizes ``dims``: dict with ``ld`` (stride of the mode-1
    fibres in bytes), ``scale_offset`` (byte offset of the FP32 scales), ``nscales`` and ``bytes``."""
    ld = ctypes.c_int64()
    off, ns, nb = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
    check(lib().rh_fp8_layout(len(dims), i64_array(dims), ctypes.byref(ld), ctypes.byref(off), ctypes.byref(ns),
                              ctypes.byref(nb)))
    return {"ld": ld.value, "scale_offset": off.value, "nscales": ns.value, "bytes": nb.value}


def omega(seed, tensor_id, mode, row0, nrows, ell, device="cuda"):
    """Omega_mode(row0 + i, c) for i < nrows, c < ell as an (ell, nrows) FP32 tensor (column c = row c)."""
    torch = _torch()
    out = torch.empty((ell, nrows), dtype=torch.float32, device=device)
    check(lib().rh_omega(int(seed) & 0xFFFFFFFFFFFFFFFF, int(tensor_id), int(mode), int(row0), int(nrows), int(ell),
                         _ptr(out), _stream(out.device)))
    return out


def rhosvd_sketch(X, dims, mode, ell, seed=0, tensor_id=0, with_norm=False):
    """Y = X_(mode) Omega_mode as an (ell, I_mode) FP64 tensor holding the column-major I x ell matrix."""
    torch = _check_input(X, dims)
    d = len(dims)
    dt = _dtype_code(X)
    da = i64_array(dims)
    ws_bytes = lib().rhosvd_sketch_workspace_size(d, da, dt, int(mode), int(ell))
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=X.device)
    Y = torch.empty((ell, int(dims[mode])), dtype=torch.float64, device=X.device)
    nrm = torch.empty(1, dtype=torch.float64, device=X.device) if with_norm else None
    check(lib().rhosvd_sketch(d, da, dt, _ptr(X), int(mode), int(ell), int(seed) & 0xFFFFFFFFFFFFFFFF,
                              int(tensor_id), _ptr(Y), _ptr(nrm), _ptr(ws), ws_bytes, _stream(X.device)))
    return (Y, nrm) if with_norm else Y


def rhosvd_sketch_offset(X, dims, mode, ell, row0, seed=0, tensor_id=0, with_norm=False, form=None, Y=None,
                         norm=None):
    """rhosvd_sketch with Omega rows row0, row0 + 1, ... (a slab of a larger tensor; see the C ABI).
    ``form="f32_bf16x2"`` runs a first-mode sketch of an FP32 tensor on the tensor cores.  Given
    ``Y`` (and ``norm``), the sketch (and ||X||^2) is added to them on the device."""
    torch = _torch()
    d = len(dims)
    dt = _FORMS[form] if form is not None else _dtype_code(X)
    da = i64_array(dims)
    ws_bytes = lib().rhosvd_sketch_workspace_size(d, da, dt, int(mode), int(ell))
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=X.device)
    acc = Y is not None
    if Y is None:
        Y = torch.empty((ell, int(dims[mode])), dtype=torch.float64, device=X.device)
    if with_norm and norm is None:
        norm = torch.zeros(1, dtype=torch.float64, device=X.device)
    check(lib().rhosvd_sketch_offset(d, da, dt, _ptr(X), int(mode), int(ell), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                     int(tensor_id), int(row0), int(acc), _ptr(Y), _ptr(norm if with_norm else None),
                                     _ptr(ws), ws_bytes, _stream(X.device)))
    return (Y, norm) if with_norm else Y


def tall_skinny_r(B, dims, mode):
    """R (I_mode x I_mode FP64, upper) of the tall-skinny QR of B_(mode)^T, as an (n, n) tensor holding
    the column-major matrix (row c of the tensor = column c of R)."""
    torch = _check_input(B, dims)
    d = len(dims)
    dt = _dtype_code(B)
    da = i64_array(dims)
    n = int(dims[mode])
    ws_bytes = lib().rh_tall_skinny_r_workspace_size(d, da, dt, int(mode))
    if ws_bytes == 0:
        raise ValueError("invalid tall-skinny QR request (I_mode must be <= 64)")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=B.device)
    R = torch.empty((n, n), dtype=torch.float64, device=B.device)
    check(lib().rh_tall_skinny_r(d, da, dt, _ptr(B), int(mode), _ptr(R), _ptr(ws), ws_bytes, _stream(B.device)))
    return R


def tucker_factor(Q, Ub, r):
    """A = Q Ub(:, 1:r) with the column-sign convention and Ur = Ub(:, 1:r) flipped alike; Q is the
    (ell, I) tensor of the I x ell matrix, Ub the (ell, ell) tensor of the ell x ell matrix.  Returns
    (A as (r, I), Ur as (r, ell))."""
    torch = _torch()
    ell, I = (int(v) for v in Q.shape)
    A = torch.empty((r, I), dtype=torch.float64, device=Q.device)
    Ur = torch.empty((r, ell), dtype=torch.float64, device=Q.device)
    check(lib().rh_tucker_factor(I, ell, int(r), _ptr(Q), _ptr(Ub.contiguous()), _ptr(A), _ptr(Ur),
                                 _stream(Q.device)))
    return A, Ur


def cast_f64(A, dtype):
    """An FP64 CUDA tensor converted by the library to ``dtype`` (torch.float32 or torch.float64)."""
    torch = _torch()
    out = torch.empty(A.shape, dtype=dtype, device=A.device)
    src = A.contiguous()
    check(lib().rh_cast_f64(_ptr(src), src.numel(), RH_F64 if dtype == torch.float64 else RH_F32, _ptr(out),
                            _stream(A.device)))
    return out


def split_bf16x2(X):
    """RH_BF16X2 representation of a flat FP32 CUDA tensor: an int16 tensor of 2 N BF16 bit patterns."""
    torch = _torch()
    n = X.numel()
    out = torch.empty(2 * n, dtype=torch.int16, device=X.device)
    check(lib().rh_split_bf16x2(_ptr(X), n, _ptr(out), _stream(X.device)))
    return out


def rhosvd_sketch_bf16(Xb, dims, ell, seed=0, tensor_id=0, pieces=2, with_norm=False):
    """Tensor-core sketch of mode 0 for a BF16 (pieces=1, int16 bit patterns of N values),
    BF16X2 (pieces=2, 2 N values) or FP32 (pieces="f32", split on the fly) tensor; returns the
    (ell, I_0) FP64 tensor of the I_0 x ell Y (and ||X||^2 when with_norm, FP32 input only)."""
    torch = _torch()
    d = len(dims)
    da = i64_array(dims)
    dt = _piece_form(pieces)
    ws_bytes = lib().rhosvd_sketch_workspace_size(d, da, dt, 0, int(ell))
    if ws_bytes == 0:
        raise ValueError("unsupported BF16 sketch request")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=Xb.device)
    Y = torch.empty((ell, int(dims[0])), dtype=torch.float64, device=Xb.device)
    nrm = torch.empty(1, dtype=torch.float64, device=Xb.device) if with_norm else None
    check(lib().rhosvd_sketch(d, da, dt, _ptr(Xb), 0, int(ell), int(seed) & 0xFFFFFFFFFFFFFFFF, int(tensor_id),
                              _ptr(Y), _ptr(nrm), _ptr(ws), ws_bytes, _stream(Xb.device)))
    return (Y, nrm) if with_norm else Y


def orthonormalize(Y):
    """Thin QR of the column-major m x n matrix held in the (n, m) FP64 tensor Y; returns (Q, info)."""
    torch = _torch()
    n, m = Y.shape
    ws_bytes = lib().rh_orthonormalize_workspace_size(m, n)
    if ws_bytes == 0:
        raise ValueError("need 1 <= n <= min(m, 64)")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=Y.device)
    Q = torch.empty_like(Y)
    info = torch.zeros(1, dtype=torch.int32, device=Y.device)
    check(lib().rh_orthonormalize(m, n, _ptr(Y.contiguous()), _ptr(Q), _ptr(info), _ptr(ws), ws_bytes,
                                  _stream(Y.device)))
    return Q, info


def mode_product(X, dims, mode, A, out_dtype=None, transpose=True):
    """Y = X x_mode A^T (A: tensor (k, I_mode) holding the column-major I_mode x k matrix), or with
    ``transpose=False`` Y = X x_mode A (A: tensor (I_mode, k) holding the column-major k x I_mode matrix)."""
    torch = _check_input(X, dims)
    k = int(A.shape[0]) if transpose else int(A.shape[1])
    dt = _dtype_code(X)
    odt = dt if out_dtype is None else (_lib.RH_F64 if out_dtype == torch.float64 else _lib.RH_F32)
    out_dims = list(dims)
    out_dims[mode] = k
    n = 1
    for v in out_dims:
        n *= int(v)
    Y = torch.empty(n, dtype=torch.float64 if odt == _lib.RH_F64 else torch.float32, device=X.device)
    check(lib().rh_mode_product(len(dims), i64_array(dims), dt, _ptr(X), int(mode), k, _ptr(A.contiguous()),
                                int(bool(transpose)), odt, _ptr(Y), _stream(X.device)))
    return Y, out_dims


def mode_product_bf16(Xb, dims, A, pieces=2):
    """First-mode product Y = X x_0 A^T on the tensor cores; Xb from split_bf16x2 (pieces=2), BF16
    bits (pieces=1) or a plain FP32 tensor (pieces="f32"); A a (k, I_0) FP64 tensor holding the
    column-major I_0 x k matrix.  Returns (Y flat FP32 of k x N/I_0, layout c + k p)."""
    torch = _torch()
    d = len(dims)
    da = i64_array(dims)
    dt = _piece_form(pieces)
    k = int(A.shape[0])
    ws_bytes = lib().rh_mode_product_workspace_size(d, da, dt, 0, k)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=Xb.device)
    n = 1
    for v in dims[1:]:
        n *= int(v)
    Y = torch.empty(k * n, dtype=torch.float32, device=Xb.device)
    check(lib().rh_mode_product_bf16(d, da, dt, _ptr(Xb), k, _ptr(A.contiguous()), _ptr(Y), _ptr(ws), ws_bytes,
                                     _stream(Xb.device)))
    return Y


def mode_product_split(X, dims, mode, A):
    """Y = X x_mode A^T on the tensor cores for a flat FP32 tensor X read as RH_F32_BF16X2; A the
    (k, I_mode) FP64 tensor of the I_mode x k matrix.  Returns (Y flat FP32, out dims)."""
    torch = _torch()
    d = len(dims)
    da = i64_array(dims)
    k = int(A.shape[0])
    ws_bytes = lib().rh_mode_product_split_workspace_size(d, da, int(mode), k)
    if ws_bytes == 0:
        raise ValueError("invalid split mode product request")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=X.device)
    out = [int(v) for v in dims]
    out[mode] = k
    n = 1
    for v in out:
        n *= v
    Y = torch.empty(n, dtype=torch.float32, device=X.device)
    check(lib().rh_mode_product_split(d, da, _ptr(X), int(mode), k, _ptr(A.contiguous()), _ptr(Y), _ptr(ws), ws_bytes,
                                      _stream(X.device)))
    return Y, out


def left_svd(B, dims, mode):
    """(U, sv) of the mode-``mode`` unfolding of B (I_mode <= 64); U as (I, I) holding column-major U."""
    torch = _check_input(B, dims)
    dt = _dtype_code(B)
    I = int(dims[mode])
    da = i64_array(dims)
    ws_bytes = lib().rh_left_svd_workspace_size(len(dims), da, dt, int(mode))
    if ws_bytes == 0:
        raise ValueError("left_svd needs I_mode <= 64")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=B.device)
    U = torch.empty((I, I), dtype=torch.float64, device=B.device)
    sv = torch.empty(I, dtype=torch.float64, device=B.device)
    check(lib().rh_left_svd(len(dims), da, dt, _ptr(B), int(mode), _ptr(U), _ptr(sv), _ptr(ws), ws_bytes,
                            _stream(B.device)))
    return U, sv


def _fptrs(factors):
    return (ctypes.c_void_p * len(factors))(*[f.data_ptr() for f in factors])


def core_ttm(X, dims, factors):
    """G = X x_1 A_1^T ... with factors given as (k_n, I_n) FP64 tensors (column-major I_n x k_n)."""
    torch = _check_input(X, dims)
    d = len(dims)
    dt = _dtype_code(X)
    ks = [int(f.shape[0]) for f in factors]
    da, ka = i64_array(dims), i32_array(ks)
    ws_bytes = lib().core_ttm_workspace_size(d, da, dt, ka)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=X.device)
    n = 1
    for k in ks:
        n *= k
    G = torch.empty(n, dtype=torch.float64, device=X.device)
    fs = [f.contiguous() for f in factors]
    check(lib().core_ttm(d, da, dt, _ptr(X), _fptrs(fs), ka, _ptr(G), _ptr(ws), ws_bytes, _stream(X.device)))
    return G, ks


def orthonormalize_tucker(factors, core, dims):
    """The orthonormalising post-processing of Sec. 5 in place: factors (list of (k_n, I_n) FP64 CUDA
    tensors holding column-major I_n x k_n matrices) become Q_n of A_n = Q_n R_n and the flat FP64 core
    G x_1 R_1 ... x_d R_d (k_1 x ... x k_d)."""
    torch = _torch()
    d = len(dims)
    ks = [int(f.shape[0]) for f in factors]
    da, ka = i64_array(dims), i32_array(ks)
    ws_bytes = lib().rh_orthonormalize_tucker_workspace_size(d, da, ka)
    if ws_bytes == 0:
        raise ValueError("invalid Tucker sizes (need 1 <= k_n <= min(I_n, 64))")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=core.device)
    check(lib().rh_orthonormalize_tucker(d, da, ka, _fptrs(factors), _ptr(core), _ptr(ws), ws_bytes,
                                         _stream(core.device)))
    return factors, core


def tucker_residual(X, dims, factors, core):
    """Device tensor [||X - X_hat||^2, ||X||^2] for a Tucker tensor (FP64 core and factors)."""
    torch = _check_input(X, dims)
    d = len(dims)
    dt = _dtype_code(X)
    ks = [int(f.shape[0]) for f in factors]
    da, ka = i64_array(dims), i32_array(ks)
    ws_bytes = lib().rh_tucker_residual_workspace_size(d, da, dt, ka)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=X.device)
    out = torch.empty(2, dtype=torch.float64, device=X.device)
    fs = [f.contiguous() for f in factors]
    check(lib().rh_tucker_residual(d, da, dt, _ptr(X), _fptrs(fs), ka, _ptr(core.contiguous()), _ptr(out), _ptr(ws),
                                   ws_bytes, _stream(X.device)))
    return out


class Tucker:
    """Tucker factors (list of (k_n, I_n) FP64 tensors holding column-major I_n x k_n matrices),
    the FP64 core (flat, column-major, sizes ``core_dims``), the norms ||X||^2, ||G||^2 and the
    per-mode flag of the Householder QR branch."""

    def __init__(self, factors, core, core_dims, norms, info):
        self.factors = factors
        self.core = core
        self.core_dims = core_dims
        self.norms = norms
        self.info = info


class RsthosvdCall:
    """A prepared R-STHOSVD call: outputs and workspace allocated once, ``run()`` enqueues it.

    Reusing the prepared buffers keeps allocation out of repeated calls (benchmarks).
    """

    ALG = "rsthosvd"

    def __init__(self, dims, dtype, ranks, p=5, seed=0, rho=None, tensor_id=0, clamp=False, truncate=True,
                 device="cuda", svd_route=0, power_iters=0):
        torch = _torch()
        self.dims = [int(x) for x in dims]
        d = len(self.dims)
        if isinstance(dtype, str):
            self.dt = _FORMS[dtype]
            self.factor = 2 if dtype == "bf16x2" else 1
        else:
            self.dt = RH_F64 if dtype == torch.float64 else RH_F32
            self.factor = 1
        self.opts = make_options(seed=seed, p=p, tensor_id=tensor_id, rho=rho, clamp=clamp, truncate=truncate,
                                 svd_route=svd_route, power_iters=power_iters)
        self.da = i64_array(self.dims)
        self.ra = i32_array(ranks)
        self._fn = getattr(lib(), self.ALG)
        self.ws_bytes = getattr(lib(), self.ALG + "_workspace_size")(d, self.da, self.dt, self.ra,
                                                                      ctypes.byref(self.opts))
        if self.ws_bytes == 0:
            # re-run the validation through the call itself to get the message
            check(self._fn(d, self.da, self.dt, None, self.ra, ctypes.byref(self.opts), None, None, None,
                           None, None, 0, None))
            raise ValueError("invalid request")
        ko = self._out_ranks(ranks, p, clamp, truncate, None if self.ALG == "rhosvd" else rho)
        self.core_dims = ko
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.factors = [torch.empty((ko[n], self.dims[n]), dtype=torch.float64, device=device) for n in range(d)]
        ncore = 1
        for k in ko:
            ncore *= k
        self.core = torch.empty(ncore, dtype=torch.float64, device=device)
        self.norms = torch.empty(2, dtype=torch.float64, device=device)
        self.info = torch.zeros(d, dtype=torch.int32, device=device)
        self.fptrs = (ctypes.c_void_p * d)(*[f.data_ptr() for f in self.factors])

    def _out_ranks(self, ranks, p, clamp, truncate, rho):
        d = len(self.dims)
        cur = list(self.dims)
        independent = self.ALG == "rhosvd"
        order = list(rho) if rho is not None else sorted(range(d), key=lambda n: (-cur[n], n))
        out = [0] * d
        for n in order:
            M = 1
            for k in range(d):
                if k != n:
                    M *= cur[k]
            ell = int(ranks[n]) + int(p)
            if clamp:
                ell = min(ell, cur[n], M)
            k = min(int(ranks[n]), ell) if truncate else ell
            out[n] = k
            if not independent:
                cur[n] = k
        return out

    def run(self, X, norms=True):
        if self.dt == _lib.RH_FP8_E4M3:
            nb = fp8_layout(self.dims)["bytes"]
            if not X.is_cuda or not X.is_contiguous() or X.numel() * X.element_size() != nb:
                raise ValueError(f"an RH_FP8_E4M3 tensor of sizes {self.dims} is a contiguous CUDA buffer of {nb} bytes")
        else:
            _check_input(X, self.dims, self.factor)
        check(self._fn(len(self.dims), self.da, self.dt, _ptr(X), self.ra, ctypes.byref(self.opts), self.fptrs,
                       _ptr(self.core), _ptr(self.norms) if norms else None, _ptr(self.info), _ptr(self.ws),
                       self.ws_bytes, _stream(X.device)))
        return Tucker(self.factors, self.core, self.core_dims, self.norms, self.info)


class RhosvdCall(RsthosvdCall):
    """A prepared R-HOSVD (Alg. 2) call."""

    ALG = "rhosvd"


def rhosvd(X, dims, ranks, p=5, seed=0, tensor_id=0, clamp=False, truncate=True, svd_route=0, power_iters=0,
           form=None):
    """R-HOSVD (Alg. 2) of the flat column-major tensor X with sizes ``dims``; ``power_iters`` steps of
    randomized subspace iteration in every range finder (rh_options.power_iters); ``form="f32_bf16x2"``
    runs every mode the tensor-core kernels cover there (FP32 X split on the fly)."""
    call = RhosvdCall(dims, form or X.dtype, ranks, p=p, seed=seed, tensor_id=tensor_id, clamp=clamp,
                      truncate=truncate, device=X.device, svd_route=svd_route, power_iters=power_iters)
    return call.run(X)


def adaptive(X, dims, eps, variant="sthosvd", block=8, max_ranks=None, p=10, seed=0, rho=None, tensor_id=0,
             form=None, svd_route=0):
    """Adaptive-rank R-HOSVD (``variant="hosvd"``, Alg. 4) or R-STHOSVD (``"sthosvd"``, Alg. 5) of the
    flat column-major tensor X to relative error ``eps`` (tolerance eps ||X|| / sqrt(d) per mode).
    ``max_ranks`` caps the range finder per mode (default min(I_n, 64 - p)).  ``form`` selects a
    low-precision storage form of X as in rsthosvd (Alg. 5 only; its first mode runs on the tensor
    cores).  Synchronous; returns a Tucker whose factors are (r_n, I_n) views and whose ``ranks``
    attribute lists the chosen ranks."""
    torch = _torch()
    if form is None:
        _check_input(X, dims)
    elif not X.is_cuda or not X.is_contiguous():
        raise ValueError("X must be a contiguous CUDA tensor")
    d = len(dims)
    dims = [int(v) for v in dims]
    if max_ranks is None:
        max_ranks = [max(1, min(v, 64 - int(p))) for v in dims]
    vcode = {"hosvd": 0, "sthosvd": 1}[variant]
    dt = _FORMS[form] if form is not None else _dtype_code(X)
    da, ma = i64_array(dims), i32_array(max_ranks)
    opts = make_options(seed=seed, p=p, tensor_id=tensor_id, rho=rho, svd_route=svd_route)
    ws_bytes = lib().adaptive_rank_workspace_size(d, da, dt, vcode, ma, ctypes.byref(opts))
    if ws_bytes == 0:
        raise ValueError("invalid adaptive request (check dtype, max_ranks + p <= 64)")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=X.device)
    ntot = 1
    for v in dims:
        ntot *= v
    ells = [min(int(max_ranks[n]) + int(p), dims[n], ntot // dims[n]) for n in range(d)]
    full = [torch.zeros((ells[n], dims[n]), dtype=torch.float64, device=X.device) for n in range(d)]
    ncore = 1
    for k in ells:
        ncore *= k
    core = torch.zeros(ncore, dtype=torch.float64, device=X.device)
    norms = torch.zeros(2, dtype=torch.float64, device=X.device)
    ranks = (ctypes.c_int32 * d)()
    fptrs = (ctypes.c_void_p * d)(*[f.data_ptr() for f in full])
    check(lib().adaptive_rank(d, da, dt, _ptr(X), float(eps), vcode, int(block), ma, ctypes.byref(opts), fptrs,
                              _ptr(core), ranks, _ptr(norms), _ptr(ws), ws_bytes, _stream(X.device)))
    rk = [int(ranks[n]) for n in range(d)]
    # factor n occupies the first r_n columns of its I_n x max_ranks[n] column-major buffer
    factors = [full[n].reshape(-1)[: rk[n] * dims[n]].reshape(rk[n], dims[n]) for n in range(d)]
    nc = 1
    for r in rk:
        nc *= r
    T = Tucker(factors, core[:nc], rk, norms, torch.zeros(d, dtype=torch.int32, device=X.device))
    T.ranks = rk
    return T


def _coo_args(idx, vals):
    torch = _torch()
    cols = [c.contiguous() for c in idx]
    for c in cols:
        if c.dtype != torch.int32 or not c.is_cuda:
            raise ValueError("COO indices must be int32 CUDA tensors")
    if vals.dtype != torch.float32 or not vals.is_cuda:
        raise ValueError("COO values must be a float32 CUDA tensor")
    return cols, (ctypes.c_void_p * len(cols))(*[c.data_ptr() for c in cols]), vals.contiguous()


def rhosvd_sketch_coo(idx, vals, dims, mode, ell, seed=0, tensor_id=0, omega="f32"):
    """Y = X_(mode) Omega_mode of the COO tensor (``idx``: list of d int32 CUDA index tensors, ``vals``
    FP32); returns the (ell, I_mode) FP64 tensor holding the column-major I_mode x ell Y.
    ``omega="bf16"``: Omega rounded to BF16 (the BF16-Omega form)."""
    torch = _torch()
    cols, iptr, vals = _coo_args(idx, vals)
    d = len(dims)
    da = i64_array(dims)
    nnz = int(vals.numel())
    ws_bytes = lib().rhosvd_sketch_coo_workspace_size(d, da, nnz, int(mode), int(ell))
    if ws_bytes == 0:
        raise ValueError("invalid COO sketch request")
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=vals.device)
    Y = torch.empty((int(ell), int(dims[mode])), dtype=torch.float64, device=vals.device)
    check(lib().rhosvd_sketch_coo(d, da, nnz, iptr, _ptr(vals), int(mode), int(ell), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                  int(tensor_id), {"f32": RH_F32, "bf16": _lib.RH_BF16}[omega], _ptr(Y), _ptr(ws),
                                  ws_bytes, _stream(vals.device)))
    return Y


SELECT_METHODS = {"srrqr": 0, "cpqr": 1, "deim": 2, "uniform": 3, "leverage": 4}


def subset_select(Q, method="srrqr", eta=2.0, seed=0, stream=0):
    """Row selection and A = Q (P^T Q)^{-1} of Alg. 6 steps 6-7 for a host FP64 tensor Q (I x ell),
    computed by the library's host step (no device call).  ``method``: "srrqr" (strong RRQR with
    bound ``eta``, the one SP-STHOSVD uses), "cpqr" (column-pivoted QR alone), "deim", or the
    sampling selections "uniform" and "leverage" (drawn from ``seed`` and ``stream``).  Returns
    (selected int32 tensor, increasing; A as an (ell, I) FP64 tensor holding the column-major I x ell A)."""
    torch = _torch()
    if Q.device.type != "cpu" or Q.dtype != torch.float64 or Q.dim() != 2:
        raise ValueError("Q must be a 2-D float64 host tensor")
    if method not in SELECT_METHODS:
        raise ValueError(f"method must be one of {sorted(SELECT_METHODS)}")
    I, ell = (int(v) for v in Q.shape)
    Qf = Q.t().contiguous()            # (ell, I) row-major = I x ell column-major
    sel = torch.empty(ell, dtype=torch.int32)
    A = torch.empty((ell, I), dtype=torch.float64)
    check(lib().rh_subset_select(I, ell, _ptr(Qf), SELECT_METHODS[method], float(eta),
                                 int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream) & 0xFFFFFFFF, _ptr(sel), _ptr(A)))
    return sel, A


class SpTucker(Tucker):
    """SP-STHOSVD result: factors (ell_n, I_n), selected row indices per mode, dense core."""


def sp_sthosvd_coo(idx, vals, dims, ranks, p=5, seed=0, rho=None, tensor_id=0, clamp=False, select="srrqr",
                   omega="f32", variant="sthosvd"):
    """Alg. 6 (SP-STHOSVD) of a COO tensor, or SP-HOSVD (``variant="hosvd"``: every mode on the input,
    Sec. 5); returns an SpTucker with ``selected``.  ``select``: the row selection (see subset_select);
    ``omega="bf16"``: the BF16-Omega sketch."""
    torch = _torch()
    cols, iptr, vals = _coo_args(idx, vals)
    d = len(dims)
    dims = [int(v) for v in dims]
    da, ra = i64_array(dims), i32_array(ranks)
    nnz = int(vals.numel())
    opts = make_options(seed=seed, p=p, tensor_id=tensor_id, rho=rho, clamp=clamp, select=select, omega_prec=omega)
    fn = {"sthosvd": "sp_sthosvd_coo", "hosvd": "sp_hosvd_coo"}[variant]
    ws_bytes = getattr(lib(), fn + "_workspace_size")(d, da, nnz, ra, ctypes.byref(opts))
    if ws_bytes == 0:
        check(getattr(lib(), fn)(d, da, nnz, iptr, _ptr(vals), ra, ctypes.byref(opts), None, None, None, None, None,
                                 0, None))
        raise ValueError("invalid structure-preserving request")
    # ell_n as the library computes it (same order and size rule)
    independent = variant == "hosvd"
    if independent:
        order = list(range(d))
    else:
        order = list(rho) if rho is not None else sorted(range(d), key=lambda n: (-dims[n], n))
    cur = list(dims)
    ells = [0] * d
    for n in order:
        M = 1
        for k in range(d):
            if k != n:
                M *= cur[k]
        ell = int(ranks[n]) + int(p)
        lim = min(cur[n], M)
        if ell >= lim:
            ell = lim - 1
        ells[n] = ell
        if not independent:
            cur[n] = ell
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=vals.device)
    factors = [torch.empty((ells[n], dims[n]), dtype=torch.float64, device=vals.device) for n in range(d)]
    selected = [torch.empty(ells[n], dtype=torch.int32, device=vals.device) for n in range(d)]
    ncore = 1
    for e in ells:
        ncore *= e
    core = torch.empty(ncore, dtype=torch.float64, device=vals.device)
    norms = torch.empty(2, dtype=torch.float64, device=vals.device)
    fptrs = (ctypes.c_void_p * d)(*[f.data_ptr() for f in factors])
    sptrs = (ctypes.c_void_p * d)(*[s_.data_ptr() for s_ in selected])
    check(getattr(lib(), fn)(d, da, nnz, iptr, _ptr(vals), ra, ctypes.byref(opts), fptrs, sptrs, _ptr(core),
                             _ptr(norms), _ptr(ws), ws_bytes, _stream(vals.device)))
    T = SpTucker(factors, core, ells, norms, torch.zeros(d, dtype=torch.int32, device=vals.device))
    T.selected = selected
    return T


def sp_hosvd_coo(idx, vals, dims, ranks, p=5, seed=0, tensor_id=0, clamp=False, select="srrqr", omega="f32"):
    """SP-HOSVD (Sec. 5: Alg. 6 with every mode taken on the input) of a COO tensor."""
    return sp_sthosvd_coo(idx, vals, dims, ranks, p=p, seed=seed, tensor_id=tensor_id, clamp=clamp, select=select,
                          omega=omega, variant="hosvd")


def rsthosvd(X, dims, ranks, p=5, seed=0, rho=None, tensor_id=0, clamp=False, truncate=True, form=None,
             svd_route=0, power_iters=0):
    """R-STHOSVD (Alg. 3) of the flat column-major tensor X with sizes ``dims``.

    ``form="bf16x2"`` (X from split_bf16x2), ``form="bf16"`` (X holding BF16 bit patterns),
    ``form="f32_bf16x2"`` (a plain FP32 X, split on the fly), ``form="f32_bf16x3"`` (a plain FP32 X
    split exactly into three pieces in every tensor-core kernel) or ``form="fp8_e4m3"`` (X a uint8
    buffer in the layout of fp8_layout) selects the tensor-core forms for the first mode.
    ``svd_route=1`` keeps the SVD of B on the tall-skinny QR (see rh_options.svd_route).
    ``power_iters`` adds that many randomized subspace-iteration steps to every range finder."""
    call = RsthosvdCall(dims, form or X.dtype, ranks, p=p, seed=seed, rho=rho, tensor_id=tensor_id, clamp=clamp,
                        truncate=truncate, device=X.device, svd_route=svd_route, power_iters=power_iters)
    return call.run(X)


class RsthosvdBatchedCall:
    """A prepared ``rsthosvd_batched`` call over tensors of shapes ``dims_list`` (one list of sizes
    per tensor) and ``ranks_list``; all tensors share ``dtype`` and the options, tensor i draws its
    Omega with tensor_id + i.  ``run(Xs)`` enqueues the whole batch on the current stream and
    returns one Tucker per tensor (views of buffers allocated once here)."""

    def __init__(self, dims_list, ranks_list, dtype, p=5, seed=0, tensor_id=0, clamp=False, truncate=True,
                 streams=0, device="cuda", svd_route=0, power_iters=0, rho=None):
        torch = _torch()
        if len(dims_list) != len(ranks_list) or not dims_list:
            raise ValueError("dims_list and ranks_list must be non-empty and of equal length")
        self.count = len(dims_list)
        self.dims_list = [[int(x) for x in d] for d in dims_list]
        if isinstance(dtype, str):
            self.dt = _FORMS[dtype]
            if dtype == "bf16x2":
                raise ValueError("batched calls take float32/float64 or the f32_bf16x2 and bf16 forms")
        else:
            self.dt = RH_F64 if dtype == torch.float64 else RH_F32
        if rho == "natural":
            rho = list(range(max(len(d) for d in self.dims_list)))
        self.opts = make_options(seed=seed, p=p, tensor_id=tensor_id, clamp=clamp, truncate=truncate,
                                 svd_route=svd_route, power_iters=power_iters, rho=rho)
        self.orders = i32_array([len(d) for d in self.dims_list])
        self.da = i64_array([x for d in self.dims_list for x in d])
        self.ra = i32_array([int(r) for rk in ranks_list for r in rk])
        self.streams = int(streams)
        self.ws_bytes = lib().rsthosvd_batched_workspace_size(self.count, self.orders, self.da, self.dt, self.ra,
                                                              ctypes.byref(self.opts), self.streams)
        if self.ws_bytes == 0:
            check(lib().rsthosvd_batched(self.count, self.orders, self.da, self.dt, None, self.ra,
                                         ctypes.byref(self.opts), None, None, None, None, self.streams, None, 0,
                                         None))
            raise ValueError("invalid batched request")
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.core_dims, self.factors, self.cores = [], [], []
        probe = RsthosvdCall.__new__(RsthosvdCall)
        for dims, ranks in zip(self.dims_list, ranks_list):
            probe.dims = dims
            ko = RsthosvdCall._out_ranks(probe, ranks, p, clamp, truncate, None)
            self.core_dims.append(ko)
            self.factors.append([torch.empty((ko[n], dims[n]), dtype=torch.float64, device=device)
                                 for n in range(len(dims))])
            ncore = 1
            for k in ko:
                ncore *= k
            self.cores.append(torch.empty(ncore, dtype=torch.float64, device=device))
        nf = sum(len(d) for d in self.dims_list)
        self.norms = torch.empty(2 * self.count, dtype=torch.float64, device=device)
        self.info = torch.zeros(nf, dtype=torch.int32, device=device)
        self.fptrs = (ctypes.c_void_p * nf)(*[f.data_ptr() for fs in self.factors for f in fs])
        self.cptrs = (ctypes.c_void_p * self.count)(*[c.data_ptr() for c in self.cores])
        self.device = torch.device(device)

    def run(self, Xs, norms=True):
        if len(Xs) != self.count:
            raise ValueError(f"expected {self.count} tensors, got {len(Xs)}")
        factor = 1
        for X, dims in zip(Xs, self.dims_list):
            _check_input(X, dims, factor)
        xptrs = (ctypes.c_void_p * self.count)(*[X.data_ptr() for X in Xs])
        check(lib().rsthosvd_batched(self.count, self.orders, self.da, self.dt, xptrs, self.ra, ctypes.byref(self.opts),
                                     self.fptrs, self.cptrs, _ptr(self.norms) if norms else None, _ptr(self.info),
                                     self.streams, _ptr(self.ws), self.ws_bytes, _stream(self.device)))
        return self._results()

    def _results(self):
        out, off = [], 0
        for i, dims in enumerate(self.dims_list):
            d = len(dims)
            out.append(Tucker(self.factors[i], self.cores[i], self.core_dims[i], self.norms[2 * i:2 * i + 2],
                              self.info[off:off + d]))
            off += d
        return out

    def plan(self, Xs, norms=True):
        """A recorded grouped run over these tensors (``rsthosvd_batched_plan_*``): ``plan.run()``
        enqueues it on the current stream and returns the Tucker results (the call's buffers)."""
        return BatchedPlan(self, Xs, norms)


class BatchedPlan:
    """``rsthosvd_batched_plan``: the grouped engine recorded once for fixed tensors and outputs."""

    def __init__(self, call, Xs, norms=True):
        if len(Xs) != call.count:
            raise ValueError(f"expected {call.count} tensors, got {len(Xs)}")
        for X, dims in zip(Xs, call.dims_list):
            _check_input(X, dims, 1)
        self.call = call
        self.Xs = list(Xs)   # the plan reads these buffers on every run
        xptrs = (ctypes.c_void_p * call.count)(*[X.data_ptr() for X in Xs])
        h = ctypes.c_void_p()
        check(lib().rsthosvd_batched_plan_create(call.count, call.orders, call.da, call.dt, xptrs, call.ra,
                                                 ctypes.byref(call.opts), call.fptrs, call.cptrs,
                                                 _ptr(call.norms) if norms else None, _ptr(call.info), _ptr(call.ws),
                                                 call.ws_bytes, ctypes.byref(h)))
        self.h = h
        self.launches = int(lib().rsthosvd_batched_plan_launches(h))

    def run(self):
        check(lib().rsthosvd_batched_plan_run(self.h, _stream(self.call.device)))
        return self.call._results()

    def close(self):
        if self.h:
            lib().rsthosvd_batched_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=0, tensor_id=0, clamp=False, truncate=True, form=None,
                     streams=0, svd_route=0, power_iters=0):
    """R-STHOSVD (Alg. 3) of every tensor in ``Xs`` (flat column-major, sizes ``dims_list[i]``) in
    one batched call; returns a list of Tucker results.  ``streams=0`` runs FP32 / FP64 truncated
    requests on the grouped engine (one launch per stage for the whole batch)."""
    call = RsthosvdBatchedCall(dims_list, ranks_list, form or Xs[0].dtype, p=p, seed=seed, tensor_id=tensor_id,
                               clamp=clamp, truncate=truncate, streams=streams, device=Xs[0].device,
                               svd_route=svd_route, power_iters=power_iters)
    return call.run(Xs)


class RsthosvdHostCall:
    """R-STHOSVD through ``rsthosvd_host``: X and the outputs live in (pinned) host memory.

    ``run(X_host)`` enqueues H2D copy, decomposition and D2H copies on the current stream;
    after the stream is synchronised the numpy views ``factors`` / ``core`` / ``norms``
    hold the result.  ``h2d_bytes`` / ``d2h_bytes`` are the bytes copied per call.
    """

    def __init__(self, dims, dtype, ranks, p=5, seed=0, rho=None, tensor_id=0, clamp=False, truncate=True,
                 device="cuda"):
        torch = _torch()
        dev_call = RsthosvdCall.__new__(RsthosvdCall)
        dev_call.dims = [int(x) for x in dims]
        ko = RsthosvdCall._out_ranks(dev_call, ranks, p, clamp, truncate, rho)
        self.dims = dev_call.dims
        d = len(self.dims)
        if isinstance(dtype, str):
            self.dt = _FORMS[dtype]
        else:
            self.dt = RH_F64 if dtype == torch.float64 else RH_F32
        self.opts = make_options(seed=seed, p=p, tensor_id=tensor_id, rho=rho, clamp=clamp, truncate=truncate)
        self.da = i64_array(self.dims)
        self.ra = i32_array(ranks)
        self.ws_bytes = lib().rsthosvd_host_workspace_size(d, self.da, self.dt, self.ra, ctypes.byref(self.opts))
        if self.ws_bytes == 0:
            raise ValueError("invalid R-STHOSVD request")
        self.core_dims = ko
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=device)
        self.factors = [torch.empty((ko[n], self.dims[n]), dtype=torch.float64).pin_memory() for n in range(d)]
        ncore = 1
        for k in ko:
            ncore *= k
        self.core = torch.empty(ncore, dtype=torch.float64).pin_memory()
        self.norms = torch.empty(2, dtype=torch.float64).pin_memory()
        self.info = torch.zeros(d, dtype=torch.int32).pin_memory()
        self.fptrs = (ctypes.c_void_p * d)(*[f.data_ptr() for f in self.factors])
        n = 1
        for v in self.dims:
            n *= v
        if self.dt == _lib.RH_FP8_E4M3:
            self.h2d_bytes = fp8_layout(self.dims)["bytes"]
        else:
            self.h2d_bytes = n * {RH_F64: 8, _lib.RH_BF16: 2}.get(self.dt, 4)
        self.d2h_bytes = 8 * (sum(self.dims[k] * ko[k] for k in range(d)) + ncore + 2) + 4 * d
        self.device = torch.device(device)

    def run(self, X_host):
        if X_host.is_cuda:
            raise ValueError("X_host must be a host tensor")
        check(lib().rsthosvd_host(len(self.dims), self.da, self.dt, _ptr(X_host), self.ra, ctypes.byref(self.opts),
                                  self.fptrs, _ptr(self.core), _ptr(self.norms), _ptr(self.info), _ptr(self.ws),
                                  self.ws_bytes, _stream(self.device)))
