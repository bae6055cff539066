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
    names = re.findall(r"^\s*(?:rh_status|size_t|const char\*|void|uint64_t)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared()
    for n in ["rh_omega", "rhosvd_sketch", "rh_orthonormalize", "rsthosvd", "rh_last_error", "rh_version"]:
        assert n in names


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
    # requests outside the grouped engine (a converted input form, or no truncation) keep the
    # stream engine at streams = 0: min(8, count) slices
    one4 = max(_ws(L, d, r, dtype=4, p=5) for d, r in zip(dims_list, ranks_list))
    assert _batched_ws(L, dims_list, ranks_list, streams=0, dtype=4, p=5) == 3 * ((one4 + 255) // 256 * 256)
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
    # a converted input form is not on the grouped engine
    assert L.rsthosvd_batched_plan_create(2, orders, dims, 4, xs, ranks, ctypes.byref(o), fs, cs, None, None,
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
    # a custom processing order is not accepted for a batch
    assert _batched_ws(L, [[30, 20, 10]], [[4, 4, 4]], p=5, rho=[2, 1, 0]) == 0


def test_svd_route_option(L):
    from paper_1905_07311_gb300 import _lib

    assert _lib.make_options().svd_route == 0
    assert _ws(L, [30, 20, 10], [4, 4, 4], p=5, svd_route=1) > 0
    code, msg = _call_invalid(L, [30, 20, 10], [4, 4, 4], p=5, svd_route=2)
    assert code == 1 and "svd_route" in msg
