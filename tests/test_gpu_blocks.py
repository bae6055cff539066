"""Building blocks through the C ABI against their definitions (needs a GB300).

* rh_mode_product: Y_(n) = A^T X_(n) (Sec. 2.1) against the oracle's mode product;
  element-wise bound c u (|A|^T |X_(n)|) with c = I_n + 2 (recursive sum of I_n terms).
* rh_left_svd: singular values of B_(n) against LAPACK (numpy.linalg.svd) within
  c eps sigma_1 (backward-stable QR + Jacobi: c = 64 * I_n); leading singular subspaces with a
  gap of at least 10% agree to c eps / gap.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle.tensor import ttm, unfold  # noqa: E402


@pytest.fixture(scope="module")
def rh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07311_gb300 import build

    build.build()
    import paper_1905_07311_gb300 as rh

    return rh


def dev(X, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).ravel(order="F")).astype(dtype)).cuda()


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,k", [((150, 37, 41), 13), ((3, 200, 5, 7), 64), ((1000, 3), 1), ((33, 129, 2), 40)])
def test_mode_product_matches_definition(rh, dtype, shape, k):
    rs = np.random.default_rng(7)
    X = rs.standard_normal(shape).astype(dtype)
    for n in range(len(shape)):
        A = rs.standard_normal((shape[n], k)).astype(dtype)
        Y, od = rh.mode_product(dev(X, dtype), list(shape), n, torch.from_numpy(A.T.copy()).cuda())
        Yg = np.reshape(Y.cpu().numpy(), od, order="F").astype(np.float64)
        Yr = ttm(X.astype(np.float64), A.astype(np.float64).T, n)
        bound = ttm(np.abs(X.astype(np.float64)), np.abs(A.astype(np.float64)).T, n)
        u = 2.0 ** -24 if dtype == np.float32 else 2.0 ** -53
        assert np.all(np.abs(Yg - Yr) <= (shape[n] + 2) * u * bound + 1e-300)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_mode_product_untransposed_wide_output(rh, dtype):
    rs = np.random.default_rng(10)
    X = rs.standard_normal((20, 7, 30)).astype(dtype)
    for n, k in [(0, 200), (1, 150), (2, 65)]:
        A = rs.standard_normal((k, X.shape[n])).astype(dtype)        # k x I_n, Y = X x_n A
        Y, od = rh.mode_product(dev(X, dtype), [20, 7, 30], n, torch.from_numpy(A.T.copy()).cuda(), transpose=False)
        Yg = np.reshape(Y.cpu().numpy(), od, order="F").astype(np.float64)
        Yr = ttm(X.astype(np.float64), A.astype(np.float64), n)
        bound = ttm(np.abs(X.astype(np.float64)), np.abs(A.astype(np.float64)), n)
        u = 2.0 ** -24 if dtype == np.float32 else 2.0 ** -53
        assert od[n] == k
        assert np.all(np.abs(Yg - Yr) <= (X.shape[n] + 2) * u * bound + 1e-300)


def test_mode_product_fp32_to_fp64_output(rh):
    rs = np.random.default_rng(8)
    X = rs.standard_normal((40, 30, 20)).astype(np.float32)
    A = rs.standard_normal((30, 10)).astype(np.float32)
    Y, od = rh.mode_product(dev(X, np.float32), [40, 30, 20], 1, torch.from_numpy(A.T.copy()).cuda(),
                            out_dtype=torch.float64)
    assert Y.dtype == torch.float64
    Yr = ttm(X.astype(np.float64), A.astype(np.float64).T, 1)
    assert np.allclose(np.reshape(Y.cpu().numpy(), od, order="F"), Yr, rtol=0, atol=1e-4)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,mode", [((60, 20000), 0), ((7, 25, 300), 1), ((900, 41), 1), ((5, 3, 64, 2), 2),
                                        ((1, 1, 1), 0)])
def test_left_svd_matches_lapack(rh, dtype, shape, mode):
    rs = np.random.default_rng(9)
    I = shape[mode]
    X = rs.standard_normal(shape)
    # graded spectrum on the short mode
    X = ttm(X, np.diag(0.7 ** np.arange(I)), mode).astype(dtype)
    U, sv = rh.left_svd(dev(X, dtype), list(shape), mode)
    U = U.cpu().numpy().T
    sv = sv.cpu().numpy()
    Bm = unfold(X.astype(np.float64), mode)
    Ur, sr, _ = np.linalg.svd(Bm, full_matrices=False)
    eps = 2.0 ** -24 if dtype == np.float32 else 2.0 ** -53
    c = 64 * max(I, 8)
    assert np.all(np.abs(sv[: sr.size] - sr) <= c * eps * sr[0])
    assert np.abs(U.T @ U - np.eye(I)).max() <= c * eps
    for kk in range(1, sr.size):
        gap = (sr[kk - 1] - sr[kk]) / sr[0]
        if gap >= 0.1 and sr[kk - 1] > 0:
            Qk = U[:, :kk]
            d = np.linalg.norm(Ur[:, :kk] - Qk @ (Qk.T @ Ur[:, :kk]), 2)
            assert d <= c * eps / gap, (kk, d)
