"""rhosvd_sketch_static: the sketch entry point that allocates nothing (the caller passes only
X, Y and norm2; the scratch is a static device array inside the library).  Its output must match
rhosvd_sketch within the sketch tolerance of the parity tests, on two calls in a row with
different shapes and dtypes, so that contents left in the shared array by the first call
cannot leak into the second.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07311_gb300 import build

    build.build()
    import paper_1905_07311_gb300 as rh

    return rh


def _static(rh, Xd, dims, mode, ell, seed, tid):
    from paper_1905_07311_gb300 import _lib

    Y = torch.empty((ell, dims[mode]), dtype=torch.float64, device=Xd.device)
    nrm = torch.empty(1, dtype=torch.float64, device=Xd.device)
    dt = _lib.RH_F64 if Xd.dtype == torch.float64 else _lib.RH_F32
    code = _lib.lib().rhosvd_sketch_static(len(dims), _lib.i64_array(dims), dt, ctypes.c_void_p(Xd.data_ptr()),
                                           mode, ell, seed, tid, ctypes.c_void_p(Y.data_ptr()),
                                           ctypes.c_void_p(nrm.data_ptr()),
                                           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _lib.check(code)
    return Y, nrm


CASES = [((150, 37, 41), np.float32, 1, 33), ((129, 257), np.float64, 0, 64), ((1024, 512), np.float32, 0, 60)]


def test_static_sketch_matches_workspace_sketch_on_consecutive_calls(rh):
    from oracle import rng as orng
    from oracle.tensor import unfold

    for k, (shape, dtype, mode, ell) in enumerate(CASES):
        rs = np.random.default_rng(100 + k)
        X = rs.standard_normal(shape).astype(dtype)
        Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
        seed, tid = 1234 + k, k
        Ys, ns = _static(rh, Xd, list(shape), mode, ell, seed, tid)
        Yw, nw = rh.rhosvd_sketch(Xd, list(shape), mode, ell, seed=seed, tensor_id=tid, with_norm=True)
        torch.cuda.synchronize()
        Xm = unfold(X.astype(np.float64), mode)
        M = Xm.shape[1]
        bound = np.abs(Xm) @ np.abs(orng.omega(seed, tid, mode, np.arange(M), ell).astype(np.float64))
        c, u = ((512 + M / 512 + 8), 2.0 ** -24) if dtype == np.float32 else (M + 8, 2.0 ** -53)
        diff = np.abs(Ys.cpu().numpy().T - Yw.cpu().numpy().T)
        assert np.all(diff <= 2 * c * u * bound + 1e-300)
        tol = 1e-12 if dtype == np.float64 else 32 * 2.0 ** -24
        assert abs(float(ns.item()) - float(nw.item())) <= tol * float(nw.item())


def test_static_sketch_rejects_sizes_beyond_the_array(rh):
    from paper_1905_07311_gb300 import _lib

    dims = [40000, 3]                 # 40000 * 64 * 8 bytes > 16 MiB even with one split
    # full-size buffers: a regression of the size check gives a wrong return code, not an
    # out-of-bounds access
    X = torch.zeros(40000 * 3, dtype=torch.float64, device="cuda")
    Y = torch.zeros(64 * 40000, dtype=torch.float64, device="cuda")
    code = _lib.lib().rhosvd_sketch_static(2, _lib.i64_array(dims), _lib.RH_F64, ctypes.c_void_p(X.data_ptr()), 0,
                                           64, 0, 0, ctypes.c_void_p(Y.data_ptr()), None, None)
    assert code == 1
    assert "16 MiB" in _lib.lib().rh_last_error().decode()
