"""Adaptive-rank randomized HOSVD / STHOSVD (Sec. 4, Alg. 4 and Alg. 5) through the C ABI against the
oracle (needs a GB300).

Both sides use the same reading of the adaptive range finder (blocked randomized QB on one Gaussian
stream, tolerance eps ||X|| / sqrt(d), p more columns, SVD trim) and the same Omega bits, so the
chosen ranks must be equal wherever no residual sits within rounding of tau^2; the cases below keep
every residual away from its threshold.  Relative errors agree to 1e-12 (FP64) / 1e-5 (FP32) and the
factors are orthonormal.
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
from workloads import hilbert, lowrank_plus_noise_np  # noqa: E402


def dev(X, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).ravel(order="F")).astype(dtype)).cuda()


def _check(rh, X, eps, variant, block, p, dtype, max_ranks=None, rho=None):
    Xd = dev(X, dtype)
    Xe = X.astype(dtype).astype(np.float64)
    T = rh.adaptive(Xd, list(X.shape), eps, variant=variant, block=block, max_ranks=max_ranks, p=p, seed=4, rho=rho)
    torch.cuda.synchronize()
    if variant == "sthosvd":
        out = otk.adaptive_rsthosvd(Xe, eps, block, p, 4, rho=rho, max_ranks=max_ranks)
    else:
        out = otk.adaptive_rhosvd(Xe, eps, block, p, 4, max_ranks=max_ranks)
    ranks_o = [f.shape[1] for f in out["factors"]]
    assert T.ranks == ranks_o, (T.ranks, ranks_o)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.ranks, order="F")
    e_g = rel_error(Xe, G, A)
    e_o = rel_error(Xe, out["core"], out["factors"])
    f64 = dtype == np.float64
    assert abs(e_g - e_o) <= (1e-12 if f64 else 1e-5), (e_g, e_o)
    assert e_g <= eps * (1 + 1e-6) + (0 if f64 else 1e-6)
    for a in A:
        assert np.abs(a.T @ a - np.eye(a.shape[1])).max() <= (1e-12 if f64 else 2e-5)
    nx = float(T.norms.cpu().numpy()[0])
    assert abs(nx - np.sum(Xe ** 2)) <= (1e-12 if f64 else 16 * 2.0 ** -24) * np.sum(Xe ** 2)
    return T, out


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("variant", ["sthosvd", "hosvd"])
@pytest.mark.parametrize("eps,block", [(3e-1, 1), (5e-2, 4), (1e-2, 8)])
def test_adaptive_matches_oracle(rh, dtype, variant, eps, block):
    X = lowrank_plus_noise_np([48, 40, 36], [14, 12, 10], 0.7, 1e-4, seed=31)
    _check(rh, X, eps, variant, block, 5, dtype)


def test_adaptive_4way_with_caps_and_order(rh):
    X = lowrank_plus_noise_np([24, 20, 18, 16], [6, 6, 5, 5], 0.6, 1e-4, seed=32)
    _check(rh, X, 2e-2, "sthosvd", 2, 3, np.float64, max_ranks=[8, 6, 6, 4], rho=[2, 0, 3, 1])


def test_adaptive_hilbert_fp64(rh):
    """The paper's 1-based Hilbert tensor (the Table 4 family), small enough for the oracle."""
    X = hilbert([40, 40, 40], offset=3)
    for eps in (1e-3, 1e-5):
        T, out = _check(rh, X, eps, "sthosvd", 1, 5, np.float64)
        assert all(r < 20 for r in T.ranks)
