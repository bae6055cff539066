"""The slab partition of R-STHOSVD on one GPU (``paper_1905_07311_gb300.slab`` with the library backend
and a single rank): slabs resident on the device, slabs in pinned host memory streamed to the device
(the out-of-core form: the tensor is never whole on the device), and the tensor-core first mode.
Against the oracle's R-STHOSVD (Alg. 3, modes in order) with the gates of the plain algorithm:
|err - err_oracle| <= 1e-12 (FP64) / 1e-5 (FP32 and the BF16-split first mode, whose Omega the
oracle rounds to BF16), leading subspaces to 1e-10 / 1e-4 (1e-3 with the split first mode).
Needs a GB300.
"""

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


from oracle import tucker as otk  # noqa: E402
from oracle.tensor import rel_error  # noqa: E402
from workloads import lowrank_plus_noise_np  # noqa: E402


def _slabs(X, bounds, dtype, host):
    from paper_1905_07311_gb300.slab import Slab

    out = []
    for k0, k1 in bounds:
        t = torch.from_numpy(np.ascontiguousarray(np.ravel(X[..., k0:k1], order="F")).astype(dtype))
        if host:
            out.append(Slab(k0, k1, t.pin_memory(), device=torch.device("cuda")))
        else:
            out.append(Slab(k0, k1, t.cuda()))
    return out


def _check(res, X, ranks, p, seed, f64, omega_round=None, gate=None, tau=None):
    out = otk.rsthosvd(X, ranks, p, seed, rho=list(range(X.ndim)), record=True, omega_round=omega_round)
    A = [f.cpu().numpy().T.copy() for f in res.factors]
    G = np.reshape(res.core.cpu().numpy(), res.core_dims, order="F")
    e_g, e_o = rel_error(X, G, A), rel_error(X, out["core"], out["factors"])
    assert abs(e_g - e_o) <= (1e-12 if f64 else 1e-5), (e_g, e_o)
    tau = tau if tau is not None else (1e-5 if f64 else 1e-2)
    gate = gate if gate is not None else (1e-10 if f64 else 1e-4)
    for rec in out["records"]:
        n = rec["mode"]
        sv = rec["sv_B"]
        k = max(1, int(np.sum(sv >= tau * sv[0])))
        U = out["factors"][n][:, :k]
        Qa, _ = np.linalg.qr(A[n])
        assert np.linalg.norm(U - Qa @ (Qa.T @ U), 2) <= gate, n
        assert np.abs(A[n].T @ A[n] - np.eye(A[n].shape[1])).max() <= (1e-12 if f64 else 2e-5)
    nx = float(res.norm_x2.item())
    assert abs(nx - np.sum(X ** 2)) <= (1e-12 if f64 else 1e-6) * np.sum(X ** 2)
    return e_g


@pytest.mark.parametrize("host", [False, True])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_slab_rsthosvd_matches_oracle(rh, dtype, host):
    from paper_1905_07311_gb300 import slab

    dims, ranks, p, seed = [90, 70, 64], [8, 7, 6], 5, 13
    X = lowrank_plus_noise_np(dims, [10, 10, 10], 0.8, 1e-3, seed=61)
    Xe = X.astype(dtype).astype(np.float64)
    slabs = _slabs(X, [(0, 20), (20, 23), (23, 64)], dtype, host)
    be = slab.LibraryBackend("f64" if dtype == np.float64 else "f32")
    res = slab.rsthosvd_slabs(slabs, dims, ranks, p=p, seed=seed, backend=be)
    torch.cuda.synchronize()
    _check(res, Xe, ranks, p, seed, dtype == np.float64)


def test_slab_rsthosvd_4way(rh):
    from paper_1905_07311_gb300 import slab

    dims, ranks, p, seed = [30, 24, 20, 18], [4, 4, 3, 3], 3, 5
    X = lowrank_plus_noise_np(dims, [5] * 4, 0.8, 1e-3, seed=62)
    res = slab.rsthosvd_slabs(_slabs(X, slab.even_slabs(18, 4), np.float64, False), dims, ranks, p=p, seed=seed,
                              backend=slab.LibraryBackend("f64"))
    torch.cuda.synchronize()
    _check(res, X, ranks, p, seed, True)


def test_slab_rsthosvd_tensor_core_first_mode_streamed(rh):
    """The first mode's sketch and mode product on the tensor cores (FP32 slabs split into BF16 head
    and tail on the fly, Omega in BF16), every slab streamed from pinned host memory twice."""
    from paper_1905_07311_gb300 import slab

    dims, ranks, p, seed = [128, 72, 60], [10, 8, 6], 6, 3
    X = lowrank_plus_noise_np(dims, [12, 12, 12], 0.8, 1e-3, seed=63).astype(np.float32)
    slabs = _slabs(X, slab.even_slabs(60, 5), np.float32, True)
    res = slab.rsthosvd_slabs(slabs, dims, ranks, p=p, seed=seed, backend=slab.LibraryBackend("f32_bf16x2"))
    torch.cuda.synchronize()
    _check(res, X.astype(np.float64), ranks, p, seed, False, omega_round={0: "bf16"}, gate=1e-3, tau=0.05)


def test_slab_single_slab_equals_library_call_error(rh):
    """One slab is the whole tensor: the same decomposition as the library's rsthosvd (FP64, both at
    the oracle's error to 1e-12)."""
    from paper_1905_07311_gb300 import slab

    dims, ranks, p, seed = [50, 40, 30], [5, 4, 3], 4, 8
    X = lowrank_plus_noise_np(dims, [6, 6, 6], 0.8, 1e-3, seed=64)
    res = slab.rsthosvd_slabs(_slabs(X, [(0, 30)], np.float64, False), dims, ranks, p=p, seed=seed,
                              backend=slab.LibraryBackend("f64"))
    T = rh.rsthosvd(torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda(), dims, ranks, p=p, seed=seed,
                    rho=[0, 1, 2])
    torch.cuda.synchronize()
    A1 = [f.cpu().numpy().T for f in res.factors]
    A2 = [f.cpu().numpy().T for f in T.factors]
    G1 = np.reshape(res.core.cpu().numpy(), res.core_dims, order="F")
    G2 = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    assert abs(rel_error(X, G1, A1) - rel_error(X, G2, A2)) <= 1e-12
