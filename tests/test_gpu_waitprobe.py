"""Reporting of a bounded tensor-core wait that gave up.

Every mbarrier wait of the tensor-core kernels is bounded; when one gives up, the kernel records a
code in the call's wait status, and the calls report it: info bit 16 on the mode concerned
(rsthosvd, rsthosvd_host), the first int32 of the workspace (rhosvd_sketch, rh_mode_product_bf16),
RH_ETIMEOUT (adaptive_rank).  ``rh_test_wait_probe(k)`` makes tensor-core launch number k wait on a
barrier that nothing arrives at, with a short limit, before it allocates tensor memory or issues
any copy or MMA, so the give-up happens with nothing in flight.  These tests make that wait run
out and check each reporting path; no GPU fault or hang is involved.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

PROBE_CODE = 64
DIMS = [128, 64, 48]
RANKS = [6, 5, 4]


@pytest.fixture(scope="module")
def rh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07311_gb300 import build

    build.build()
    import paper_1905_07311_gb300 as rh

    yield rh
    rh._lib.lib().rh_test_wait_probe(-1)


def _probe(rh, k):
    rh._lib.lib().rh_test_wait_probe(int(k))


def _x(dims, seed=0):
    rs = np.random.default_rng(seed)
    X = rs.standard_normal(int(np.prod(dims))).astype(np.float32)
    return torch.from_numpy(X).cuda()


def test_probe_sets_bit16_on_one_mode_only(rh):
    X = _x(DIMS)
    call = rh.RsthosvdCall(DIMS, "f32_bf16x2", RANKS, p=4, rho=[0, 1, 2])
    _probe(rh, -1)
    T = call.run(X)
    torch.cuda.synchronize()
    clean = T.info.cpu().numpy().copy()
    assert not np.any(clean & 16), clean
    assert clean[0] & 4            # the first mode ran on the tensor cores
    seen = []
    for k in range(0, 12):
        _probe(rh, k)
        T = call.run(X)
        torch.cuda.synchronize()
        info = T.info.cpu().numpy().copy()
        hit = [n for n in range(3) if info[n] & 16]
        if not hit:
            break                   # k is past the last tensor-core launch of the call
        assert len(hit) == 1, (k, info)   # the wait status is cleared once a mode has reported it
        seen.append(hit[0])
    _probe(rh, -1)
    assert seen and seen[0] == 0
    assert seen == sorted(seen)     # launches are counted in the order the modes run
    # the probe is off again: a clean call reports nothing
    T = call.run(X)
    torch.cuda.synchronize()
    assert not np.any(T.info.cpu().numpy() & 16)


def test_probe_in_sketch_workspace_status(rh):
    from paper_1905_07311_gb300 import _lib

    X = _x(DIMS, 1)
    d = len(DIMS)
    da = _lib.i64_array(DIMS)
    ell = 12
    ws_bytes = _lib.lib().rhosvd_sketch_workspace_size(d, da, _lib.RH_F32_BF16X2, 0, ell)
    ws = torch.full((ws_bytes,), 0, dtype=torch.uint8, device="cuda")
    Y = torch.empty((ell, DIMS[0]), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for k, want in ((-1, 0), (0, PROBE_CODE)):
        _probe(rh, k)
        code = _lib.lib().rhosvd_sketch(d, da, _lib.RH_F32_BF16X2, ctypes.c_void_p(X.data_ptr()), 0, ell, 7, 0,
                                        ctypes.c_void_p(Y.data_ptr()), None, ctypes.c_void_p(ws.data_ptr()),
                                        ws_bytes, st)
        _lib.check(code)
        torch.cuda.synchronize()
        assert int(ws[:4].view(torch.int32).item()) == want
    _probe(rh, -1)


def test_probe_in_mode_product_workspace_status(rh):
    from paper_1905_07311_gb300 import _lib

    X = _x(DIMS, 2)
    d = len(DIMS)
    da = _lib.i64_array(DIMS)
    k = 10
    A = torch.from_numpy(np.linalg.qr(np.random.default_rng(3).standard_normal((DIMS[0], k)))[0].T.copy()).cuda()
    M = DIMS[1] * DIMS[2]
    Y = torch.empty(k * M, dtype=torch.float32, device="cuda")
    ws_bytes = _lib.lib().rh_mode_product_workspace_size(d, da, _lib.RH_F32_BF16X2, 0, k)
    ws = torch.zeros(ws_bytes, dtype=torch.uint8, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kk, want in ((-1, 0), (0, PROBE_CODE)):
        _probe(rh, kk)
        _lib.check(_lib.lib().rh_mode_product_bf16(d, da, _lib.RH_F32_BF16X2, ctypes.c_void_p(X.data_ptr()), k,
                                                   ctypes.c_void_p(A.data_ptr()), ctypes.c_void_p(Y.data_ptr()),
                                                   ctypes.c_void_p(ws.data_ptr()), ws_bytes, st))
        torch.cuda.synchronize()
        assert int(ws[:4].view(torch.int32).item()) == want
    _probe(rh, -1)


def test_probe_makes_adaptive_return_timeout(rh):
    from paper_1905_07311_gb300 import _lib

    X = _x(DIMS, 4)
    _probe(rh, 0)
    with pytest.raises(_lib.RhError) as e:
        rh.adaptive(X, DIMS, 1e-2, variant="sthosvd", block=4, max_ranks=[8, 8, 8], p=4, rho=[0, 1, 2],
                    form="f32_bf16x2")
    assert e.value.code == 5        # RH_ETIMEOUT
    _probe(rh, -1)
    T = rh.adaptive(X, DIMS, 1e-2, variant="sthosvd", block=4, max_ranks=[8, 8, 8], p=4, rho=[0, 1, 2],
                    form="f32_bf16x2")
    assert len(T.ranks) == 3


def test_probe_reaches_host_info(rh):
    X = _x(DIMS, 5).cpu().pin_memory()
    call = rh.RsthosvdHostCall(DIMS, "f32_bf16x2", RANKS, p=4, rho=[0, 1, 2])
    _probe(rh, 0)
    call.run(X)
    torch.cuda.synchronize()
    info = call.info.numpy().copy()
    assert info[0] & 16 and not (info[1] & 16) and not (info[2] & 16), info
    _probe(rh, -1)
    call.run(X)
    torch.cuda.synchronize()
    assert not np.any(call.info.numpy() & 16)
