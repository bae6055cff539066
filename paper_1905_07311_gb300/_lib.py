"""ctypes binding of ``librhosvd.so`` (the C ABI declared in include/rhosvd.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  PyTorch supplies device memory (outputs and workspace) and the current
stream.  There is no fallback: if the shared library is missing the import fails.
"""

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "librhosvd.so")

RH_MAX_ORDER = 8
RH_MAX_ELL = 64
RH_F64, RH_F32, RH_BF16, RH_BF16X2, RH_F32_BF16X2, RH_FP8_E4M3, RH_F32_BF16X3 = 0, 1, 2, 3, 4, 5, 6
STATUS = {0: "RH_OK", 1: "RH_EINVAL", 2: "RH_ENOMEM", 3: "RH_ECUDA", 4: "RH_ENUMERIC", 5: "RH_ETIMEOUT",
          6: "RH_EUNSUPPORTED"}


class RhOptions(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("tensor_id", ctypes.c_int32), ("p", ctypes.c_int32),
                ("rho", ctypes.c_int32 * RH_MAX_ORDER), ("clamp", ctypes.c_int32), ("truncate", ctypes.c_int32),
                ("svd_route", ctypes.c_int32), ("power_iters", ctypes.c_int32), ("select", ctypes.c_int32),
                ("omega_prec", ctypes.c_int32)]


class RhError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_SZ = ctypes.c_size_t

SIGNATURES = {
    "rh_version": (ctypes.c_char_p, []),
    "rh_last_error": (ctypes.c_char_p, []),
    "rh_kernel_launches": (ctypes.c_uint64, []),
    "rh_tuning_count": (_I32, []),
    "rh_tuning_name": (ctypes.c_char_p, [_I32]),
    "rh_tuning_get": (_I32, [ctypes.c_char_p]),
    "rh_tuning_set": (_I32, [ctypes.c_char_p, _I32]),
    "rh_profile_enable": (None, [_I32]),
    "rh_profile_collect": (_I32, [_P, _P, _P, _I32]),
    "rh_options_default": (None, [ctypes.POINTER(RhOptions)]),
    "rh_omega": (_I32, [_U64, _I32, _I32, _I64, _I64, _I32, _P, _P]),
    "rhosvd_sketch_workspace_size": (_SZ, [_I32, _P, _I32, _I32, _I32]),
    "rhosvd_sketch": (_I32, [_I32, _P, _I32, _P, _I32, _I32, _U64, _I32, _P, _P, _P, _SZ, _P]),
    "rhosvd_sketch_static": (_I32, [_I32, _P, _I32, _P, _I32, _I32, _U64, _I32, _P, _P, _P]),
    "rhosvd_sketch_offset": (_I32, [_I32, _P, _I32, _P, _I32, _I32, _U64, _I32, _I64, _I32, _P, _P, _P, _SZ, _P]),
    "rh_tall_skinny_r_workspace_size": (_SZ, [_I32, _P, _I32, _I32]),
    "rh_tall_skinny_r": (_I32, [_I32, _P, _I32, _P, _I32, _P, _P, _SZ, _P]),
    "rh_tucker_factor": (_I32, [_I64, _I32, _I32, _P, _P, _P, _P, _P]),
    "rh_cast_f64": (_I32, [_P, _I64, _I32, _P, _P]),
    "rh_mode_product": (_I32, [_I32, _P, _I32, _P, _I32, _I32, _P, _I32, _I32, _P, _P]),
    "rh_mode_product_workspace_size": (_SZ, [_I32, _P, _I32, _I32, _I32]),
    "rh_mode_product_bf16": (_I32, [_I32, _P, _I32, _P, _I32, _P, _P, _P, _SZ, _P]),
    "rh_mode_product_split_workspace_size": (_SZ, [_I32, _P, _I32, _I32]),
    "rh_mode_product_split": (_I32, [_I32, _P, _P, _I32, _I32, _P, _P, _P, _SZ, _P]),
    "rh_left_svd_workspace_size": (_SZ, [_I32, _P, _I32, _I32]),
    "rh_left_svd": (_I32, [_I32, _P, _I32, _P, _I32, _P, _P, _P, _SZ, _P]),
    "rh_split_bf16x2": (_I32, [_P, _I64, _P, _P]),
    "rh_orthonormalize_workspace_size": (_SZ, [_I64, _I32]),
    "rh_orthonormalize": (_I32, [_I64, _I32, _P, _P, _P, _P, _SZ, _P]),
    "rsthosvd_workspace_size": (_SZ, [_I32, _P, _I32, _P, ctypes.POINTER(RhOptions)]),
    "rsthosvd": (_I32, [_I32, _P, _I32, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P, _P, _SZ, _P]),
    "rhosvd_workspace_size": (_SZ, [_I32, _P, _I32, _P, ctypes.POINTER(RhOptions)]),
    "rhosvd": (_I32, [_I32, _P, _I32, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P, _P, _SZ, _P]),
    "core_ttm_workspace_size": (_SZ, [_I32, _P, _I32, _P]),
    "core_ttm": (_I32, [_I32, _P, _I32, _P, _P, _P, _P, _P, _SZ, _P]),
    "adaptive_rank_workspace_size": (_SZ, [_I32, _P, _I32, _I32, _P, ctypes.POINTER(RhOptions)]),
    "adaptive_rank": (_I32, [_I32, _P, _I32, _P, ctypes.c_double, _I32, _I32, _P, ctypes.POINTER(RhOptions), _P, _P,
                             _P, _P, _P, _SZ, _P]),
    "rhosvd_sketch_coo_workspace_size": (_SZ, [_I32, _P, _I64, _I32, _I32]),
    "rhosvd_sketch_coo": (_I32, [_I32, _P, _I64, _P, _P, _I32, _I32, ctypes.c_uint64, _I32, _I32, _P, _P, _SZ, _P]),
    "sp_hosvd_coo_workspace_size": (_SZ, [_I32, _P, _I64, _P, ctypes.POINTER(RhOptions)]),
    "sp_hosvd_coo": (_I32, [_I32, _P, _I64, _P, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P, _P, _SZ, _P]),
    "sp_sthosvd_coo_workspace_size": (_SZ, [_I32, _P, _I64, _P, ctypes.POINTER(RhOptions)]),
    "sp_sthosvd_coo": (_I32, [_I32, _P, _I64, _P, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P, _P, _SZ, _P]),
    "rh_orthonormalize_tucker_workspace_size": (_SZ, [_I32, _P, _P]),
    "rh_orthonormalize_tucker": (_I32, [_I32, _P, _P, _P, _P, _P, _SZ, _P]),
    "rh_tucker_residual_workspace_size": (_SZ, [_I32, _P, _I32, _P]),
    "rh_tucker_residual": (_I32, [_I32, _P, _I32, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "rh_fp8_layout": (_I32, [_I32, _P, _P, _P, _P, _P]),
    "rsthosvd_batched_workspace_size": (_SZ, [_I32, _P, _P, _I32, _P, ctypes.POINTER(RhOptions), _I32]),
    "rsthosvd_batched": (_I32, [_I32, _P, _P, _I32, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P, _I32, _P,
                                _SZ, _P]),
    "rsthosvd_batched_plan_create": (_I32, [_I32, _P, _P, _I32, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P,
                                            _P, _SZ, ctypes.POINTER(_P)]),
    "rsthosvd_batched_plan_run": (_I32, [_P, _P]),
    "rsthosvd_batched_plan_launches": (_I64, [_P]),
    "rsthosvd_batched_plan_destroy": (None, [_P]),
    "rh_subset_select": (_I32, [_I64, _I32, _P, _I32, ctypes.c_double, _U64, ctypes.c_uint32, _P, _P]),
    "rsthosvd_host_workspace_size": (_SZ, [_I32, _P, _I32, _P, ctypes.POINTER(RhOptions)]),
    "rsthosvd_host": (_I32, [_I32, _P, _I32, _P, _P, ctypes.POINTER(RhOptions), _P, _P, _P, _P, _P, _SZ, _P]),
    "rh_test_wait_probe": (None, [_I64]),
}


def lib():
    """Load the shared library once; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run `python -m paper_1905_07311_gb300.build` "
                              "(the CUDA library is required; there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != 0:
        raise RhError(code, lib().rh_last_error().decode())


def i64_array(vals):
    arr = (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])
    return arr


def i32_array(vals):
    return (ctypes.c_int32 * len(vals))(*[int(v) for v in vals])


SELECT = {"srrqr": 0, "cpqr": 1, "deim": 2, "uniform": 3, "leverage": 4}


def make_options(seed=0, p=5, tensor_id=0, rho=None, clamp=False, truncate=True, svd_route=0, power_iters=0,
                 select="srrqr", omega_prec="f32"):
    o = RhOptions()
    lib().rh_options_default(ctypes.byref(o))
    o.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    o.p = int(p)
    o.tensor_id = int(tensor_id)
    if rho is not None:
        for k, m in enumerate(rho):
            o.rho[k] = int(m)
    o.clamp = int(bool(clamp))
    o.truncate = int(bool(truncate))
    o.svd_route = int(svd_route)
    o.power_iters = int(power_iters)
    o.select = SELECT[select] if isinstance(select, str) else int(select)
    o.omega_prec = {"f32": RH_F32, "bf16": RH_BF16}[omega_prec] if isinstance(omega_prec, str) else int(omega_prec)
    return o
