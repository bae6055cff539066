"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  Needs a GB300.

Tolerances and where they come from:
* Omega: bit-exact (both sides implement the same specification operation by operation).
* Sketch: element-wise |Y_gpu - Y| <= c u (|X_(n)| |Omega|), the standard bound for a
  recursive sum of c terms with unit roundoff u.  FP32 path: products and sums in FP32,
  at most 512 terms per inner accumulator plus M/512 folds, then FP64 across CTAs, so
  c = 512 + M/512 + 8, u = 2^-24.  FP64 path: c = M + 8, u = 2^-53.
* QR: orthonormality and range, ||Y - Q Q^T Y|| <= 1e-13 ||Y|| (FP64 Householder /
  CholeskyQR2 are both backward stable at this level for the sizes used).
* R-STHOSVD: |err_gpu - err_oracle| <= 1e-12 (FP64) / 1e-5 (FP32) absolute on the relative
  Tucker error, both errors formed by a direct FP64 reconstruction.  Subspaces: the
  leading k columns of the oracle's factor, k = #{sigma_i(B) >= tau sigma_1(B)}, must lie in
  the GPU factor's span to 1e-10 (FP64, tau = 1e-5) / 1e-4 (FP32, tau = 1e-2).  The
  rounding error of B is ~eps ||B||, so the leading-k subspace moves by about
  eps / tau (1e-15 / 1e-5 = 1e-10; 1e-7 .. 1e-6 / 1e-2 <= 1e-4).
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


from oracle import rng as orng  # noqa: E402
from oracle import tucker as otk  # noqa: E402
from oracle.tensor import rel_error, unfold  # noqa: E402
from workloads import hilbert, lowrank_plus_noise_np  # noqa: E402


def dev(X, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).ravel(order="F")).astype(dtype)).cuda()


def mat(t):
    return t.cpu().numpy().T.copy()


def core_np(T):
    return np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")


def subspace_gap(A_ref, sv_ref, A, tau):
    k = int(np.sum(sv_ref >= tau * sv_ref[0]))
    k = max(1, min(k, A_ref.shape[1]))
    U = A_ref[:, :k]
    Qa, _ = np.linalg.qr(A)
    return np.linalg.norm(U - Qa @ (Qa.T @ U), 2), k


# ---------------------------------------------------------------------------------
# a1: Omega
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("seed,tid,mode,row0,nrows,ell", [
    (0, 0, 0, 0, 1000, 64),
    ((1 << 40) + 12345, 5, 3, (1 << 33) - 100, 333, 13),
    (7, (1 << 28) - 1, 15, 123456789, 77, 1),
    (2, 0, 1, 0, 4097, 60),
])
def test_omega_bit_exact(rh, seed, tid, mode, row0, nrows, ell):
    g = rh.omega(seed, tid, mode, row0, nrows, ell).cpu().numpy().T
    o = orng.omega(seed, tid, mode, np.arange(row0, row0 + nrows, dtype=np.int64), ell)
    assert np.array_equal(g.view(np.uint32), o.view(np.uint32))


# ---------------------------------------------------------------------------------
# a2: sketch
# ---------------------------------------------------------------------------------
SKETCH_SHAPES = [((150, 37, 41), None), ((3, 200, 5, 7), None), ((1000,), None), ((1000, 3), None),
                 ((129, 257), None), ((17, 19, 23), None)]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shape,_", SKETCH_SHAPES)
@pytest.mark.parametrize("ell", [1, 7, 33, 64])
def test_sketch_matches_oracle(rh, dtype, shape, _, ell):
    rs = np.random.default_rng(hash((shape, ell)) % 2 ** 32)
    X = rs.standard_normal(shape).astype(dtype)
    Xd = dev(X, dtype)
    seed, tid = 99, 3
    for n in range(len(shape)):
        Y, nrm = rh.rhosvd_sketch(Xd, shape, n, ell, seed=seed, tensor_id=tid, with_norm=True)
        Yg = mat(Y)
        Xm = unfold(X.astype(np.float64), n)
        M = Xm.shape[1]
        Om = orng.omega(seed, tid, n, np.arange(M), ell).astype(np.float64)
        Yr = Xm @ Om
        bound = np.abs(Xm) @ np.abs(Om)
        if dtype == np.float32:
            c, u = 512 + M / 512 + 8, 2.0 ** -24
        else:
            c, u = M + 8, 2.0 ** -53
        assert np.all(np.abs(Yg - Yr) <= c * u * bound + 1e-300), (n, np.max(np.abs(Yg - Yr) / (bound + 1e-300)))
        ref = float(np.sum(X.astype(np.float64) ** 2))
        assert abs(float(nrm.item()) - ref) <= (1e-12 if dtype == np.float64 else 2e-6) * ref
        Y2 = rh.rhosvd_sketch(Xd, shape, n, ell, seed=seed, tensor_id=tid)
        assert torch.equal(Y, Y2)          # deterministic reduction order


# ---------------------------------------------------------------------------------
# a3: QR
# ---------------------------------------------------------------------------------
def _check_q(Y, Q):
    n = Y.shape[1]
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 1e-13 * max(n, 8)
    assert np.linalg.norm(Y - Q @ (Q.T @ Y)) <= 1e-13 * max(1.0, np.linalg.norm(Y))


def test_orthonormalize_well_conditioned_uses_cholqr2(rh):
    rs = np.random.default_rng(0)
    Y = rs.standard_normal((1000, 40)) @ np.diag(np.logspace(0, -3, 40))
    Qg, info = rh.orthonormalize(torch.from_numpy(Y.T.copy()).cuda())
    Q = mat(Qg)
    _check_q(Y, Q)
    assert int(info.item()) == 0
    Qr, _ = np.linalg.qr(Y)
    assert np.linalg.norm(Q @ Q.T - Qr @ Qr.T, 2) <= 1e-10


def test_orthonormalize_ill_conditioned_falls_back_to_householder(rh):
    X = hilbert([200, 200, 200], offset=1)
    Om = orng.omega(0, 0, 0, np.arange(40000), 25).astype(np.float64)
    Y = unfold(X, 0) @ Om
    Qg, info = rh.orthonormalize(torch.from_numpy(Y.T.copy()).cuda())
    Q = mat(Qg)
    assert int(info.item()) == 1
    _check_q(Y, Q)


def test_orthonormalize_rank_deficient(rh):
    rs = np.random.default_rng(1)
    B = rs.standard_normal((300, 5))
    Y = np.hstack([B, B @ rs.standard_normal((5, 7))])
    Qg, info = rh.orthonormalize(torch.from_numpy(Y.T.copy()).cuda())
    Q = mat(Qg)
    assert int(info.item()) == 1
    _check_q(Y, Q)


# ---------------------------------------------------------------------------------
# a2-a5: R-STHOSVD end to end
# ---------------------------------------------------------------------------------
def _compare(rh, X, ranks, p, seed, dtype, rho=None, tau=None, gate=None, err_tol=None, alg="rsthosvd", **kw):
    Xd = dev(X, dtype)
    if alg == "rsthosvd":
        T = rh.rsthosvd(Xd, list(X.shape), ranks, p=p, seed=seed, rho=rho, **kw)
    else:
        T = rh.rhosvd(Xd, list(X.shape), ranks, p=p, seed=seed, **kw)
    torch.cuda.synchronize()
    Xe = X.astype(dtype).astype(np.float64)          # the exact input the GPU saw
    if alg == "rsthosvd":
        out = otk.rsthosvd(Xe, ranks, p, seed, rho=rho, record=True, clamp=kw.get("clamp", False))
    else:
        out = otk.rhosvd(Xe, ranks, p, seed, record=True, clamp=kw.get("clamp", False))
    A = [mat(f) for f in T.factors]
    G = core_np(T)
    e_g = rel_error(Xe, G, A)
    e_o = rel_error(Xe, out["core"], out["factors"])
    f64 = dtype == np.float64
    tau = tau if tau is not None else (1e-5 if f64 else 1e-2)
    gate = gate if gate is not None else (1e-10 if f64 else 1e-4)
    err_tol = err_tol if err_tol is not None else (1e-12 if f64 else 1e-5)
    assert abs(e_g - e_o) <= err_tol, (e_g, e_o)
    for rec in out["records"]:
        n = rec["mode"]
        d, k = subspace_gap(out["factors"][n], rec["sv_B"], A[n], tau)
        assert d <= gate, (n, d, k)
        assert np.abs(A[n].T @ A[n] - np.eye(A[n].shape[1])).max() <= (1e-12 if f64 else 2e-5)
    nx, ng = T.norms.cpu().numpy()
    # ||X||^2: FP64 sums of per-thread partials of at most 16 squares (FP32 partials on the FP32 path)
    assert abs(nx - np.sum(Xe ** 2)) <= (1e-12 if f64 else 16 * 2.0 ** -24) * np.sum(Xe ** 2)
    assert abs(ng - np.sum(G ** 2)) <= 1e-12 * max(np.sum(G ** 2), 1e-300)
    return T, e_g, e_o, out


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rsthosvd_small_3way(rh, dtype):
    X = lowrank_plus_noise_np([40, 35, 30], [6, 6, 6], 0.7, 1e-3, seed=3)
    _compare(rh, X, [5, 6, 4], 5, 11, dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rsthosvd_4way_ragged(rh, dtype):
    X = lowrank_plus_noise_np([37, 21, 18, 13], [4, 4, 3, 3], 0.8, 1e-3, seed=4)
    _compare(rh, X, [3, 4, 3, 2], 4, 5, dtype, rho=[2, 0, 3, 1])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rsthosvd_many_tiles(rh, dtype):
    X = lowrank_plus_noise_np([300, 200, 130], [25, 25, 25], 0.9, 1e-3, seed=5)
    _compare(rh, X, [20, 20, 20], 10, 1, dtype)


def test_rsthosvd_f32_gram_route_taken(rh):
    """Decay 0.9, r = 20 of 25: the truncation gap is far above 1e-5 sigma_1^2, so every mode's
    truncation SVD goes through the Gram matrix (info bit 2) and still matches the oracle."""
    X = lowrank_plus_noise_np([300, 200, 130], [25, 25, 25], 0.9, 1e-3, seed=5)
    T, _, _, _ = _compare(rh, X, [20, 20, 20], 10, 1, np.float32)
    assert [v & 2 for v in T.info.cpu().numpy().tolist()] == [2, 2, 2]


def test_rsthosvd_f32_deep_truncation_takes_the_double_float_gram(rh):
    """Decay 0.4 and r = 10: sigma_r^2 - sigma_{r+1}^2 is below 1e-5 sigma_1^2, where FP32 Gram
    sums cannot resolve the retained subspace; the double-float Gram matrix (~2^-44) can, so its
    route runs (info bit 8) and matches the oracle."""
    X = lowrank_plus_noise_np([90, 80, 70], [14, 14, 14], 0.4, 1e-7, seed=12)
    T, e_g, e_o, _ = _compare(rh, X, [10, 10, 10], 4, 3, np.float32)
    assert [v & 10 for v in T.info.cpu().numpy().tolist()] == [8, 8, 8]


def test_rsthosvd_f32_double_float_gram_wide(rh):
    """ell = 40 (Gram blocks sized to 40 columns), decay 0.8: sigma_34^2 - sigma_35^2 ~ 1e-7
    sigma_1^2 rejects the FP32 Gram matrix, sigma_40^2 ~ 3e-8 sigma_1^2 is well inside what the
    double-float one resolves.  (With a steeper spectrum, e.g. decay 0.55, sigma_40^2 ~ 5e-21
    sigma_1^2 is singular even in double-float and the tall-skinny QR takes over.)"""
    X = lowrank_plus_noise_np([300, 200, 130], [44, 44, 44], 0.8, 1e-4, seed=14)
    T, e_g, e_o, _ = _compare(rh, X, [34, 34, 34], 6, 7, np.float32)
    assert [v & 10 for v in T.info.cpu().numpy().tolist()] == [8, 8, 8]


def test_rsthosvd_f32_numerically_singular_gram_falls_back_to_qr(rh):
    """Decay 0.55, ell = 40: sigma_40^2 ~ 5e-21 sigma_1^2, the double-float Cholesky breaks down
    and the tall-skinny QR of B^T runs (neither Gram bit)."""
    X = lowrank_plus_noise_np([300, 200, 130], [44, 44, 44], 0.55, 1e-7, seed=14)
    T, e_g, e_o, _ = _compare(rh, X, [34, 34, 34], 6, 7, np.float32)
    assert [v & 10 for v in T.info.cpu().numpy().tolist()] == [0, 0, 0]


@pytest.mark.parametrize("shape,core,ranks,p,decay", [([90, 80, 70], 14, 10, 4, 0.4),
                                                      ([300, 200, 130], 44, 34, 6, 0.55)])
def test_rsthosvd_f32_tall_skinny_qr_route(rh, shape, core, ranks, p, decay):
    """svd_route = 1: the Householder QR of B^T (256-row blocks and merge levels; 32- and
    64-column instantiations, unit-stride and strided views of B) for every mode."""
    X = lowrank_plus_noise_np(shape, [core] * 3, decay, 1e-7, seed=15)
    T, e_g, e_o, _ = _compare(rh, X, [ranks] * 3, p, 7, np.float32, svd_route=1)
    assert [v & 10 for v in T.info.cpu().numpy().tolist()] == [0, 0, 0]


def test_rsthosvd_f32_rank_deficient_sketch(rh):
    """Exact multilinear rank 4 with ell = 9: B B^T is singular up to rounding, so its FP32 Gram
    may or may not be numerically definite (either truncation route may run); the result must
    still recover the rank-4 tensor and match the oracle."""
    X = lowrank_plus_noise_np([50, 45, 40], [4, 4, 4], 0.8, 0.0, seed=13)
    T, e_g, _, _ = _compare(rh, X, [4, 4, 4], 5, 2, np.float32, gate=1e-3)
    assert e_g < 1e-5


def test_rsthosvd_hilbert_200_config(rh):
    """200^3 tensor 1/(i+j+k+1), rank 20, p = 5, seed 0, order 1,2,3; FP64."""
    X = hilbert([200, 200, 200], offset=1)
    T, e_g, e_o, _ = _compare(rh, X, [20, 20, 20], 5, 0, np.float64, rho=[0, 1, 2])
    assert e_g < 1e-12 and e_o < 1e-12
    assert T.info.cpu().numpy().tolist() == [1, 1, 1]   # Householder branch on the ill-conditioned sketches
    Gd, Ad = otk.sthosvd(X, [20, 20, 20], rho=[0, 1, 2])
    assert e_g < 10 * rel_error(X, Gd, Ad)


def test_rsthosvd_exact_rank_recovery(rh):
    X = lowrank_plus_noise_np([60, 50, 40], [4, 3, 5], 0.9, 0.0, seed=6)
    T, e_g, _, _ = _compare(rh, X, [4, 3, 5], 6, 2, np.float64, gate=1e-8)
    assert e_g < 1e-13


def test_rsthosvd_matrix_is_randomized_svd(rh):
    rs = np.random.default_rng(7)
    U, _ = np.linalg.qr(rs.standard_normal((300, 80)))
    V, _ = np.linalg.qr(rs.standard_normal((80, 80)))
    X = (U * 0.8 ** np.arange(80)) @ V.T
    # after mode 0 the core is 10 x 80, so mode 1 needs clamping (ell <= 10)
    _compare(rh, X, [10, 10], 5, 3, np.float64, rho=[0, 1], clamp=True)


def test_rsthosvd_vector_and_unit_mode(rh):
    x = np.random.default_rng(8).standard_normal((50,))
    T = rh.rsthosvd(dev(x, np.float64), [50], [1], p=0)
    torch.cuda.synchronize()
    a = mat(T.factors[0])[:, 0]
    g = T.core.cpu().numpy()[0]
    assert np.allclose(a * g, x, atol=1e-13)
    X = lowrank_plus_noise_np([40, 1, 30], [3, 1, 3], 0.5, 1e-3, seed=9)
    _compare(rh, X, [3, 1, 3], 2, 4, np.float64, clamp=True)


def test_rsthosvd_zero_tensor(rh):
    X = np.zeros((30, 20, 10))
    T = rh.rsthosvd(dev(X, np.float64), [30, 20, 10], [3, 3, 3], p=2)
    torch.cuda.synchronize()
    assert np.all(T.core.cpu().numpy() == 0)
    for f in T.factors:
        A = mat(f)
        assert np.all(np.isfinite(A))
        assert np.abs(A.T @ A - np.eye(A.shape[1])).max() < 1e-12


def test_rsthosvd_untruncated_matches_oracle_without_truncation(rh):
    X = lowrank_plus_noise_np([40, 30, 20], [5, 5, 5], 0.7, 1e-3, seed=10)
    Xd = dev(X, np.float64)
    T = rh.rsthosvd(Xd, [40, 30, 20], [4, 4, 4], p=3, seed=2, truncate=False)
    torch.cuda.synchronize()
    assert T.core_dims == [7, 7, 7]
    out = otk.rsthosvd(X, [4, 4, 4], 3, 2, truncate=False)
    e_g = rel_error(X, core_np(T), [mat(f) for f in T.factors])
    e_o = rel_error(X, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-12


def test_rsthosvd_deterministic(rh):
    X = lowrank_plus_noise_np([64, 48, 40], [8, 8, 8], 0.7, 1e-3, seed=11)
    Xd = dev(X, np.float32)
    a = rh.rsthosvd(Xd, [64, 48, 40], [6, 6, 6], p=4, seed=5)
    b = rh.rsthosvd(Xd, [64, 48, 40], [6, 6, 6], p=4, seed=5)
    torch.cuda.synchronize()
    assert torch.equal(a.core, b.core)
    assert all(torch.equal(x, y) for x, y in zip(a.factors, b.factors))


# ---------------------------------------------------------------------------------
# a6: R-HOSVD (Alg. 2) and the core G = X x_n A_n^T
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rhosvd_matches_oracle(rh, dtype):
    X = lowrank_plus_noise_np([40, 35, 30], [6, 6, 6], 0.7, 1e-3, seed=13)
    _compare(rh, X, [5, 6, 4], 5, 21, dtype, alg="rhosvd")


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rhosvd_4way_many_tiles(rh, dtype):
    X = lowrank_plus_noise_np([150, 40, 33, 9], [5, 5, 5, 4], 0.8, 1e-3, seed=14)
    _compare(rh, X, [5, 5, 5, 3], 4, 3, dtype, alg="rhosvd")


def test_rhosvd_hilbert_200(rh):
    X = hilbert([200, 200, 200], offset=1)
    T, e_g, e_o, _ = _compare(rh, X, [20, 20, 20], 5, 0, np.float64, alg="rhosvd")
    assert e_g < 1e-12


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_core_ttm_matches_definition(rh, dtype):
    from oracle.tensor import multi_ttm

    rs = np.random.default_rng(15)
    dims, ks = [70, 45, 33, 5], [7, 64, 3, 5]
    X = rs.standard_normal(dims).astype(dtype)
    A = [rs.standard_normal((dims[n], ks[n])) for n in range(4)]
    G, kk = rh.core_ttm(dev(X, dtype), dims, [torch.from_numpy(a.T.copy()).cuda() for a in A])
    Gg = np.reshape(G.cpu().numpy(), kk, order="F")
    Ae = [a.astype(dtype).astype(np.float64) for a in A]      # factors in the tensor's precision
    Gr = multi_ttm(X.astype(np.float64), Ae, transpose=True)
    tol = 1e-12 if dtype == np.float64 else 2e-5
    assert np.abs(Gg - Gr).max() <= tol * np.abs(Gr).max()


# ---------------------------------------------------------------------------------
# a7: direct residual
# ---------------------------------------------------------------------------------
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tucker_residual_matches_direct_error(rh, dtype):
    X = lowrank_plus_noise_np([80, 70, 60], [8, 8, 8], 0.7, 1e-2, seed=16)
    Xd = dev(X, dtype)
    T = rh.rsthosvd(Xd, [80, 70, 60], [6, 7, 5], p=4, seed=2)
    out = rh.tucker_residual(Xd, [80, 70, 60], T.factors, T.core).cpu().numpy()
    Xe = X.astype(dtype).astype(np.float64)
    e_ref = rel_error(Xe, core_np(T), [mat(f) for f in T.factors])
    e_gpu = float(np.sqrt(out[0] / out[1]))
    assert abs(out[1] - np.sum(Xe ** 2)) <= 1e-10 * np.sum(Xe ** 2)
    # FP32: X_hat is formed in FP32 (relative rounding ~1e-7 per entry of the reconstruction)
    assert abs(e_gpu - e_ref) <= (1e-12 if dtype == np.float64 else 2e-6)


def test_tucker_residual_hilbert_tiny_error(rh):
    X = hilbert([200, 200, 200], offset=1)
    Xd = dev(X, np.float64)
    T = rh.rsthosvd(Xd, [200, 200, 200], [20, 20, 20], p=5, seed=0, rho=[0, 1, 2])
    out = rh.tucker_residual(Xd, [200, 200, 200], T.factors, T.core).cpu().numpy()
    e_ref = rel_error(X, core_np(T), [mat(f) for f in T.factors])
    assert e_ref < 1e-12
    assert abs(float(np.sqrt(out[0] / out[1])) - e_ref) <= 1e-13
