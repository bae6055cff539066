"""The C-ABI library on a machine without a GPU: it builds, loads, exports every symbol
that include/rhosvd.h declares, and rejects invalid arguments before touching the device.
No compute call is made here.
"""

import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1905_07311_gb300 import build as b

    b.build()
    from paper_1905_07311_gb300 import _lib

    return _lib.lib()


def _declared():
    text = open(os.path.join(ROOT, "include", "rhosvd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:rh_status|size_t|const char\s*\*|void|uint64_t|int64_t|int32_t|double)\s+\**\s*(\w+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ["rh_omega", "rhosvd_sketch", "rh_orthonormalize", "rsthosvd", "rh_last_error", "rh_version"]:
        assert n in names


def test_binding_signatures_match_the_header():
    # every entry point has its argument and return types in the binding's table (a size_t or int64_t
    # result read through ctypes' default int would be truncated), and the table names nothing else
    from paper_1905_07311_gb300 import _lib

    declared = set(_declared())
    assert len(declared) > 50
    assert set(_lib.SIGNATURES) == declared


def test_every_declared_symbol_is_exported(L):
    from paper_1905_07311_gb300 import _lib

    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(\w+)$", out, flags=re.M))
    for n in _declared():
        assert n in exported, n
        assert hasattr(L, n)


def test_version_and_defaults(L):
    from paper_1905_07311_gb300 import _lib

    assert b"sm_103a" in L.rh_version()
    o = _lib.make_options()
    assert o.p == 5 and o.rho[0] == -1 and o.truncate == 1 and o.clamp == 0


def _tuning_table():
    text = open(os.path.join(ROOT, "paper_1905_07311_gb300", "csrc", "tuning_table.inc")).read()
    return {n: int(v) for n, v in re.findall(r'RH_TUNE\(\w+,\s*"([\w.]+)",\s*(\d+)\)', text)}


def test_tuning_knobs_round_trip(L):
    table = _tuning_table()
    n = L.rh_tuning_count()
    assert n == len(table) and n > 0
    names = [L.rh_tuning_name(i).decode() for i in range(n)]
    assert sorted(names) == sorted(table)
    assert L.rh_tuning_name(-1) is None and L.rh_tuning_name(n) is None
    for name in names:
        assert L.rh_tuning_get(name.encode()) == table[name]
    k = names[0].encode()
    try:
        assert L.rh_tuning_set(k, 3) == 0 and L.rh_tuning_get(k) == 3
        for bad in (-1, 4097):
            assert L.rh_tuning_set(k, bad) != 0
            assert "tuning value" in L.rh_last_error().decode()
            assert L.rh_tuning_get(k) == 3
    finally:
        assert L.rh_tuning_set(k, 0) == 0
    assert L.rh_tuning_get(k) == table[names[0]]
    assert L.rh_tuning_get(b"no.such.knob") == -1
    assert L.rh_tuning_set(b"no.such.knob", 2) != 0
    assert "unknown tuning key" in L.rh_last_error().decode()


def _ws(L, dims, ranks, dtype=0, **kw):
    from paper_1905_07311_gb300 import _lib

    o = _lib.make_options(**kw)
    return L.rsthosvd_workspace_size(len(dims), _lib.i64_array(dims), dtype, _lib.i32_array(ranks), ctypes.byref(o))


def _call_invalid(L, dims, ranks, dtype=0, **kw):
    from paper_1905_07311_gb300 import _lib

    o = _lib.make_options(**kw)
    fp = (ctypes.c_void_p * len(dims))(*([1] * len(dims)))
    code = L.rsthosvd(len(dims), _lib.i64_array(dims), dtype, ctypes.c_void_p(1), _lib.i32_array(ranks),
                      ctypes.byref(o), fp, ctypes.c_void_p(1), None, None, None, 0, None)
    return code, L.rh_last_error().decode()


def test_size_rule_is_enforced_before_launch(L):
    # r + p > I_n violates the REQUIRE line of Alg. 3
    code, msg = _call_invalid(L, [10, 40, 40], [8, 4, 4], p=5)
    assert code == 1 and "exceeds" in msg
    assert _ws(L, [10, 40, 40], [8, 4, 4], p=5) == 0
    # the same request is accepted with clamping
    assert _ws(L, [10, 40, 40], [8, 4, 4], p=5, clamp=True) > 0
    # the rule is checked on the current core: after mode 0 is truncated to 2, mode 1 sees M = 2 * 3
    code, msg = _call_invalid(L, [50, 50, 3], [2, 5, 3], p=2, rho=[0, 1, 2])
    assert code == 1


@pytest.mark.parametrize("bad", [dict(dims=[0, 4]), dict(dims=[4] * 9), dict(ranks=[0, 2])])
def test_invalid_shapes(L, bad):
    dims = bad.get("dims", [8, 8])
    ranks = bad.get("ranks", [2] * len(dims))
    code, _ = _call_invalid(L, dims, ranks, p=1)
    assert code == 1


def test_bad_dtype_and_order(L):
    code, msg = _call_invalid(L, [8, 8], [2, 2], dtype=7, p=1)
    assert code == 1 and "dtype" in msg
    code, msg = _call_invalid(L, [8, 8], [2, 2], p=1, rho=[0, 0])
    assert code == 1 and "permutation" in msg


def test_ell_beyond_64_is_unsupported(L):
    code, msg = _call_invalid(L, [200, 200, 200], [60, 20, 20], p=10)
    assert code == 6 and "64" in msg


def test_workspace_query_is_positive_and_monotone(L):
    a = _ws(L, [100, 100, 100], [10, 10, 10], p=5)
    b = _ws(L, [200, 200, 200], [10, 10, 10], p=5)
    assert 0 < a < b


def test_omega_and_sketch_argument_checks(L):
    assert L.rh_omega(0, 0, 16, 0, 4, 4, ctypes.c_void_p(1), None) == 1
    assert L.rh_omega(0, -1, 0, 0, 4, 4, ctypes.c_void_p(1), None) == 1
    from paper_1905_07311_gb300 import _lib

    dims = _lib.i64_array([5, 6])
    assert L.rhosvd_sketch(2, dims, 0, ctypes.c_void_p(1), 2, 4, 0, 0, ctypes.c_void_p(1), None, None, 0, None) == 1
    assert L.rhosvd_sketch(2, dims, 0, ctypes.c_void_p(1), 0, 65, 0, 0, ctypes.c_void_p(1), None, None, 0, None) == 1
    assert L.rhosvd_sketch(2, dims, 0, ctypes.c_void_p(1), 0, 4, 0, 0, ctypes.c_void_p(1), None, None, 0, None) == 2


def _batched_ws(L, dims_list, ranks_list, streams=0, dtype=0, **kw):
    from paper_1905_07311_gb300 import _lib

    o = _lib.make_options(**kw)
    return L.rsthosvd_batched_workspace_size(len(dims_list), _lib.i32_array([len(d) for d in dims_list]),
                                             _lib.i64_array([x for d in dims_list for x in d]), dtype,
                                             _lib.i32_array([r for rk in ranks_list for r in rk]), ctypes.byref(o),
                                             streams)


def test_batched_workspace_is_one_slice_per_stream(L):
    dims_list = [[30, 20, 10], [40, 12, 11, 9], [16, 16, 16]]
    ranks_list = [[4, 4, 4], [3, 3, 3, 3], [5, 5, 5]]
    one = max(_ws(L, d, r, p=5) for d, r in zip(dims_list, ranks_list))
    slice_ = (one + 255) // 256 * 256
    assert _batched_ws(L, dims_list, ranks_list, streams=1, p=5) == slice_
    assert _batched_ws(L, dims_list, ranks_list, streams=2, p=5) == 2 * slice_
    # streams are capped at the tensor count
    assert _batched_ws(L, dims_list, ranks_list, streams=16, p=5) == 3 * slice_
    # streams = 0 with FP64 / FP32 truncated requests: the grouped engine, one slice per tensor
    # plus the launch tables (recorded on the host: a few KB per tensor)
    slices = sum((_ws(L, d, r, dtype=dt, p=5) + 255) // 256 * 256 for d, r in zip(dims_list, ranks_list)
                 for dt in [0])
    g = _batched_ws(L, dims_list, ranks_list, streams=0, p=5)
    assert slices < g < slices + (1 << 20)
    slices32 = sum((_ws(L, d, r, dtype=1, p=5) + 255) // 256 * 256 for d, r in zip(dims_list, ranks_list))
    g32 = _batched_ws(L, dims_list, ranks_list, streams=0, dtype=1, p=5)
    assert slices32 < g32 < slices32 + (1 << 20)
    # the split form whose first mode (mode 0, I_0 <= 128, r + p <= 32) runs on the small-row
    # tensor-core kernels is recorded for the grouped engine too
    slices4 = sum((_ws(L, d, r, dtype=4, p=5) + 255) // 256 * 256 for d, r in zip(dims_list, ranks_list))
    g4 = _batched_ws(L, dims_list, ranks_list, streams=0, dtype=4, p=5)
    assert slices4 < g4 < slices4 + (1 << 20)
    # requests outside the grouped engine (a converted input form whose first mode runs elsewhere,
    # or no truncation) keep the stream engine at streams = 0: min(8, count) slices
    big = [[130, 20, 10], [40, 12, 11, 9], [16, 16, 16]]
    one4 = max(_ws(L, d, r, dtype=4, p=5) for d, r in zip(big, ranks_list))
    assert _batched_ws(L, big, ranks_list, streams=0, dtype=4, p=5) == 3 * ((one4 + 255) // 256 * 256)
    one_nt = max(_ws(L, d, r, p=5, truncate=False) for d, r in zip(dims_list, ranks_list))
    assert _batched_ws(L, dims_list, ranks_list, streams=0, p=5, truncate=False) == 3 * ((one_nt + 255) // 256 * 256)


def test_batched_plan_argument_checks(L):
    from paper_1905_07311_gb300 import _lib

    dims = _lib.i64_array([30, 20, 10, 16, 16, 16])
    orders = _lib.i32_array([3, 3])
    ranks = _lib.i32_array([4, 4, 4, 5, 5, 5])
    xs = (ctypes.c_void_p * 2)(1, 1)
    fs = (ctypes.c_void_p * 6)(*([1] * 6))
    cs = (ctypes.c_void_p * 2)(1, 1)
    h = ctypes.c_void_p()
    o = _lib.make_options(p=5)
    # no plan pointer
    assert L.rsthosvd_batched_plan_create(2, orders, dims, 1, xs, ranks, ctypes.byref(o), fs, cs, None, None,
                                          None, 0, None) == 1
    # a converted input form whose first mode is outside the small-row tensor-core kernels
    # (I_0 = 130 > 128) is not on the grouped engine
    big = _lib.i64_array([130, 20, 10, 16, 16, 16])
    assert L.rsthosvd_batched_plan_create(2, orders, big, 4, xs, ranks, ctypes.byref(o), fs, cs, None, None,
                                          None, 0, ctypes.byref(h)) == 6
    assert "grouped engine" in L.rh_last_error().decode() and not h.value
    # workspace too small (checked before anything touches the device)
    assert L.rsthosvd_batched_plan_create(2, orders, dims, 1, xs, ranks, ctypes.byref(o), fs, cs, None, None,
                                          ctypes.c_void_p(1 << 20), 16, ctypes.byref(h)) == 2
    assert L.rsthosvd_batched_plan_launches(None) == -1
    L.rsthosvd_batched_plan_destroy(None)


def test_batched_argument_checks(L):
    from paper_1905_07311_gb300 import _lib

    dims_list = [[30, 20, 10], [10, 40, 40]]
    ranks_list = [[4, 4, 4], [8, 4, 4]]                 # tensor 1 breaks r + p <= I_n at p = 5
    assert _batched_ws(L, dims_list, ranks_list, p=5) == 0
    assert _batched_ws(L, dims_list, ranks_list, p=5, clamp=True) > 0
    o = _lib.make_options(p=5)
    xs = (ctypes.c_void_p * 2)(1, 1)
    fs = (ctypes.c_void_p * 6)(*([1] * 6))
    cs = (ctypes.c_void_p * 2)(1, 1)
    code = L.rsthosvd_batched(2, _lib.i32_array([3, 3]), _lib.i64_array([30, 20, 10, 10, 40, 40]), 0, xs,
                              _lib.i32_array([4, 4, 4, 8, 4, 4]), ctypes.byref(o), fs, cs, None, None, 0, None, 0,
                              None)
    assert code == 1 and L.rh_last_error().decode().startswith("tensor 1:")
    # an order outside [1, 8], no tensors, or too many streams
    assert _batched_ws(L, [[4] * 9], [[1] * 9], p=1) == 0
    assert L.rsthosvd_batched_workspace_size(0, None, None, 0, None, None, 0) == 0
    assert _batched_ws(L, [[30, 20, 10]], [[4, 4, 4]], streams=64, p=5) > 0    # capped at count = 1
    # a processing order applies to every tensor of a batch: its first order_i entries must be a
    # permutation of 0 .. order_i - 1 for each tensor
    assert _batched_ws(L, [[30, 20, 10]], [[4, 4, 4]], p=5, rho=[2, 1, 0]) > 0
    assert _batched_ws(L, [[30, 20, 10], [9, 8, 7, 6]], [[4, 4, 4], [3, 3, 3, 3]], p=1, rho=[0, 1, 2, 3]) > 0
    assert _batched_ws(L, [[30, 20, 10], [9, 8, 7, 6]], [[4, 4, 4], [3, 3, 3, 3]], p=1, rho=[3, 0, 1, 2]) == 0


def test_svd_route_option(L):
    from paper_1905_07311_gb300 import _lib

    assert _lib.make_options().svd_route == 0
    assert _ws(L, [30, 20, 10], [4, 4, 4], p=5, svd_route=1) > 0
    code, msg = _call_invalid(L, [30, 20, 10], [4, 4, 4], p=5, svd_route=2)
    assert code == 1 and "svd_route" in msg


def test_power_iters_option(L):
    """rh_options.power_iters (subspace iteration): 0 by default, 0..8 accepted and growing the
    workspace (dense-operand sketch partials, basis of range(B^T)); the adaptive range finder
    runs without it."""
    from paper_1905_07311_gb300 import _lib

    assert _lib.make_options().power_iters == 0
    base = _ws(L, [30, 20, 10], [4, 4, 4], p=5)
    assert _ws(L, [30, 20, 10], [4, 4, 4], p=5, power_iters=2) >= base > 0
    code, msg = _call_invalid(L, [30, 20, 10], [4, 4, 4], p=5, power_iters=9)
    assert code == 1 and "power_iters" in msg
    code, msg = _call_invalid(L, [30, 20, 10], [4, 4, 4], p=5, power_iters=-1)
    assert code == 1
    d3 = _lib.i64_array([30, 20, 10])
    mr = _lib.i32_array([4, 4, 4])
    o = ctypes.byref(_lib.make_options(p=5, power_iters=1))
    assert L.adaptive_rank_workspace_size(3, d3, _lib.RH_F32, 1, mr, o) == 0


def _err(L):
    return L.rh_last_error().decode()


def test_every_entry_point_validates_before_the_device(L):
    """Each call below fails on its arguments alone (RH_EINVAL = 1, RH_ENOMEM = 2,
    RH_EUNSUPPORTED = 6); on this machine any device call would instead give RH_ECUDA = 3."""
    from paper_1905_07311_gb300 import _lib

    P = ctypes.c_void_p
    one, big = P(1), 1 << 30
    d3 = _lib.i64_array([30, 20, 10])
    ks = _lib.i32_array([4, 4, 4])
    ptr3 = (P * 3)(1, 1, 1)
    o = ctypes.byref(_lib.make_options(p=5))
    r3 = _lib.i32_array([0, 0, 0])

    # thin QR (Alg. 1 step 2): 1 <= n <= min(m, 64)
    assert L.rh_orthonormalize(4, 5, one, one, None, one, big, None) == 1
    assert L.rh_orthonormalize(100, 65, one, one, None, one, big, None) == 1
    assert L.rh_orthonormalize(100, 5, None, one, None, one, big, None) == 1
    assert L.rh_orthonormalize(100, 5, one, one, None, one, 1, None) == 2
    assert L.rh_orthonormalize_workspace_size(4, 5) == 0 < L.rh_orthonormalize_workspace_size(100, 5)
    # mode product (Sec. 2.1)
    assert L.rh_mode_product(3, d3, 1, one, 3, 4, one, 1, 1, one, None) == 1      # mode out of range
    assert L.rh_mode_product(3, d3, 1, one, 0, 0, one, 1, 1, one, None) == 1      # k = 0
    assert L.rh_mode_product(3, d3, 1, None, 0, 4, one, 1, 1, one, None) == 1
    assert L.rh_mode_product(3, d3, 0, one, 0, 4, one, 1, 1, one, None) == 1      # FP64 in, FP32 out
    assert L.rh_mode_product_bf16(3, d3, 1, one, 4, one, one, one, big, None) == 1
    assert L.rh_mode_product_bf16(3, _lib.i64_array([32, 20, 10]), 2, one, 65, one, one, one, big, None) == 6
    # I_0 % 8 != 0 with I_0 > 128 (neither the persistent nor the small-row kernel), or k > 32 there
    assert L.rh_mode_product_bf16(3, _lib.i64_array([130, 20, 10]), 2, one, 4, one, one, one, big, None) == 6
    assert L.rh_mode_product_bf16(3, d3, 2, one, 33, one, one, one, big, None) == 6
    # left SVD of a short mode (Alg. 1 step 4)
    assert L.rh_left_svd(3, _lib.i64_array([65, 20, 10]), 1, one, 0, one, one, one, big, None) == 1
    assert L.rh_left_svd(3, d3, 1, None, 2, one, one, one, big, None) == 1
    assert L.rh_left_svd(3, d3, 1, one, 2, one, one, one, 1, None) == 2
    # BF16 split
    assert L.rh_split_bf16x2(one, -1, one, None) == 1
    assert L.rh_split_bf16x2(None, 8, one, None) == 1
    assert L.rh_split_bf16x2(None, 0, None, None) == 0                            # nothing to do
    # core and direct residual
    assert L.core_ttm(3, d3, 1, one, ptr3, _lib.i32_array([0, 4, 4]), one, one, big, None) == 1
    assert L.core_ttm(3, d3, 1, None, ptr3, ks, one, one, big, None) == 1
    assert L.core_ttm(3, d3, 1, one, ptr3, ks, one, one, 1, None) == 2 and "need" in _err(L)
    assert L.rh_tucker_residual(3, d3, 1, one, ptr3, ks, None, one, one, big, None) == 1
    assert L.rh_tucker_residual(3, d3, 1, one, ptr3, ks, one, one, one, 1, None) == 2
    # adaptive rank (Alg. 4 / 5)
    assert L.adaptive_rank(3, d3, 1, one, 0.0, 0, 4, ks, o, ptr3, one, r3, None, one, big, None) == 1
    assert L.adaptive_rank(3, d3, 1, one, 0.1, 2, 4, ks, o, ptr3, one, r3, None, one, big, None) == 1
    assert L.adaptive_rank(3, d3, 1, one, 0.1, 0, 0, ks, o, ptr3, one, r3, None, one, big, None) == 1
    assert L.adaptive_rank(3, d3, 2, one, 0.1, 0, 4, ks, o, ptr3, one, r3, None, one, big, None) == 6
    assert "Alg. 5" in _err(L)
    assert L.adaptive_rank(3, _lib.i64_array([100, 100, 100]), 1, one, 0.1, 0, 4, _lib.i32_array([60, 4, 4]), o,
                           ptr3, one, r3, None, one, big, None) == 6
    assert L.adaptive_rank(3, d3, 1, one, 0.1, 0, 4, ks, o, ptr3, one, r3, None, one, 1, None) == 2
    # the three-piece split form is not an adaptive input form
    assert L.adaptive_rank(3, d3, _lib.RH_F32_BF16X3, one, 0.1, 1, 4, ks, o, ptr3, one, r3, None, one, big,
                           None) == 1
    assert "dense input form" in _err(L)
    # sparse sketch and SP-STHOSVD (Alg. 6)
    assert L.rhosvd_sketch_coo(3, d3, -1, ptr3, one, 0, 4, 0, 0, 1, one, one, big, None) == 1
    assert L.rhosvd_sketch_coo(3, d3, 10, ptr3, one, 3, 4, 0, 0, 1, one, one, big, None) == 1
    assert L.rhosvd_sketch_coo(3, d3, 10, ptr3, one, 0, 65, 0, 0, 1, one, one, big, None) == 1
    assert L.rhosvd_sketch_coo(3, d3, 10, ptr3, one, 0, 4, 0, 0, 7, one, one, big, None) == 1   # omega_prec
    assert L.rhosvd_sketch_coo(3, d3, 10, ptr3, one, 0, 4, 0, 0, 1, one, one, 1, None) == 2
    strict = _lib.i32_array([4, 4, 5])     # mode 2 (processed last): ell = 10 is not < I_2 = 10
    assert L.sp_sthosvd_coo(3, d3, 10, ptr3, one, strict, o, ptr3, None, one, None, one, big, None) == 1
    assert "must be < min" in _err(L)
    assert L.sp_sthosvd_coo_workspace_size(3, d3, 10, strict, o) == 0
    assert L.sp_sthosvd_coo_workspace_size(3, d3, 10, strict, ctypes.byref(_lib.make_options(p=5, clamp=True))) > 0
    assert L.sp_sthosvd_coo(3, d3, 10, ptr3, None, ks, o, ptr3, None, one, None, one, big, None) == 1
    assert L.sp_sthosvd_coo(3, d3, 10, ptr3, one, ks, o, ptr3, None, one, None, one, 1, None) == 2
    bad_sel = ctypes.byref(_lib.make_options(p=5, select=9))
    assert L.sp_sthosvd_coo(3, d3, 10, ptr3, one, ks, bad_sel, ptr3, None, one, None, one, big, None) == 1
    bad_om = ctypes.byref(_lib.make_options(p=5, omega_prec=4))
    assert L.sp_sthosvd_coo(3, d3, 10, ptr3, one, ks, bad_om, ptr3, None, one, None, one, big, None) == 1
    # SP-HOSVD: the strict size rule on the input sizes, every mode
    assert L.sp_hosvd_coo(3, d3, 10, ptr3, one, strict, o, ptr3, None, one, None, one, big, None) == 1
    assert L.sp_hosvd_coo_workspace_size(3, d3, 10, ks, o) > 0
    assert L.sp_hosvd_coo(3, d3, 10, ptr3, None, ks, o, ptr3, None, one, None, one, big, None) == 1
    assert L.sp_hosvd_coo(3, d3, 10, ptr3, one, ks, o, ptr3, None, one, None, one, 1, None) == 2
    # host-buffer R-STHOSVD and R-HOSVD (Alg. 3, Alg. 2)
    bad = _lib.i32_array([26, 4, 4])       # r_0 + p = 31 > I_0 = 30
    assert L.rsthosvd_host(3, d3, 1, one, bad, o, ptr3, one, None, None, one, big, None) == 1
    assert L.rsthosvd_host(3, d3, 1, None, ks, o, ptr3, one, None, None, one, big, None) == 1
    assert L.rsthosvd_host(3, d3, 1, one, ks, o, ptr3, one, None, None, one, 1, None) == 2
    assert L.rsthosvd_host_workspace_size(3, d3, 1, ks, o) > L.rsthosvd_workspace_size(3, d3, 1, ks, o)
    assert L.rhosvd(3, d3, 1, one, bad, o, ptr3, one, None, None, one, big, None) == 1
    assert L.rhosvd(3, d3, 1, one, ks, o, ptr3, one, None, None, one, 1, None) == 2
    assert L.rhosvd_sketch_static(3, d3, 1, one, 0, 65, 0, 0, one, None, None) == 1
    # plans and profiling with nothing to act on
    assert L.rsthosvd_batched_plan_launches(None) == -1
    assert L.rsthosvd_batched_plan_run(None, None) == 1
    L.rsthosvd_batched_plan_destroy(None)
    assert L.rh_profile_collect(None, None, None, 0) == 0


def test_fp8_layout_sizes(L):
    """Block-scaled E4M3 storage: the mode-1 fibres at a stride ld = I_1 rounded up to 16 bytes,
    then, from the next 16-byte boundary, one FP32 scale per 128 bytes of storage."""
    from paper_1905_07311_gb300 import _lib

    def layout(dims):
        ld, so, ns, by = ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_size_t()
        assert L.rh_fp8_layout(len(dims), _lib.i64_array(dims), ctypes.byref(ld), ctypes.byref(so),
                               ctypes.byref(ns), ctypes.byref(by)) == 0
        return ld.value, so.value, ns.value, by.value

    ld, so, ns, by = layout([128, 48, 40])
    assert ld == 128 and so == 128 * 48 * 40 and ns == so // 128 and by == so + 4 * ns
    ld, so, ns, by = layout([30, 7, 3])        # ragged: 30 -> 32 bytes per fibre, 672 bytes of data
    assert ld == 32 and so == 672 and ns == 6 and by == 672 + 4 * 6
    ld, so, ns, by = layout([5, 3])            # 48 bytes of data, one partly used scale block
    assert ld == 16 and so == 48 and ns == 1 and by == 52
    assert L.rh_fp8_layout(3, _lib.i64_array([128, 0, 40]), None, None, None, None) == 1


def test_header_is_plain_c_and_links(L):
    """include/rhosvd.h is a C header: a C99 program (strict, warnings as errors) includes it,
    links against the library and answers a workspace query without a device."""
    import shutil

    from paper_1905_07311_gb300 import _lib

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    out = os.path.join(ROOT, "_build", "c_abi_check")
    os.makedirs(out, exist_ok=True)
    src = os.path.join(out, "main.c")
    with open(src, "w") as f:
        f.write('#include "rhosvd.h"\n#include <stdio.h>\n'
                "int main(void) {\n"
                "  rh_options o;\n  rh_options_default(&o);\n"
                "  int64_t dims[3] = {30, 20, 10};\n  int32_t ranks[3] = {4, 4, 4};\n"
                "  size_t ws = rsthosvd_workspace_size(3, dims, RH_F32, ranks, &o);\n"
                '  printf("%zu %d\\n", ws, (int)RH_SELECT_DEIM);\n'
                "  return ws > 0 ? 0 : 1;\n}\n")
    exe = os.path.join(out, "main")
    libdir = os.path.dirname(_lib.LIB_PATH)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    src, "-L", libdir, "-lrhosvd", f"-Wl,-rpath,{libdir}", "-o", exe], check=True)
    res = subprocess.run([exe], capture_output=True, text=True, check=True)
    ws, deim = res.stdout.split()
    assert int(ws) == _ws(L, [30, 20, 10], [4, 4, 4], dtype=1) and int(deim) == 2


def test_three_piece_form_plans(L):
    """RH_F32_BF16X3 is planned like the two-piece split form (a first mode outside the tensor-core
    kernels on the CUDA cores), and refused with subspace iteration, whose sketch reads head + tail."""
    from paper_1905_07311_gb300 import _lib

    x3, x2 = _lib.RH_F32_BF16X3, _lib.RH_F32_BF16X2
    assert _ws(L, [256, 128, 96], [20, 20, 20], dtype=x3, p=10) > 0
    assert _ws(L, [90, 64, 40], [6, 5, 4], dtype=x3, p=5) > 0
    assert _ws(L, [256, 128, 96], [20, 20, 20], dtype=x3, p=10, power_iters=1) == 0
    assert "subspace iteration" in L.rh_last_error().decode()
    assert _ws(L, [256, 128, 96], [20, 20, 20], dtype=x2, p=10, power_iters=1) > 0
    dims = _lib.i64_array([256, 40, 30])
    assert L.rhosvd_sketch_workspace_size(3, dims, x3, 0, 25) > 0
    assert L.rh_mode_product_workspace_size(3, dims, x3, 0, 25) > 0
