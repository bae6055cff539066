"""Pins for the oracle functions of the next rows (CPU only): randomized subspace iteration in
RandSVD (Sec. 5 remark 2, Sec. 6; Halko, Martinsson and Tropp 2011, Alg. 4.3) and SP-HOSVD
(Sec. 5 remark 1).  Each check is fixed by the mathematics, not by the oracle itself:

* the range of the iterated sketch is range((X X^T)^q X Omega), formed directly by matrix powers;
* with many steps the range finder reaches the optimal rank-ell error sigma_{ell+1} and the
  leading singular subspace, so R-STHOSVD / R-HOSVD become STHOSVD / HOSVD;
* the expectation bound of the power scheme (Halko et al. 2011, Cor. 10.10), seed-averaged, and
  the error falling as q grows;
* SP-HOSVD: identity rows, |A_ij| <= 2, ||A_j||_2 <= g(I_j, ell_j), core entries of X, exact
  recovery at exact multilinear rank, and the bound of Thm. pass_error that the paper states for it.
"""

import math

import numpy as np
import pytest

from oracle import rng, tucker
from oracle.rng import omega
from oracle.tensor import frob, multi_ttm, rel_error, unfold
from workloads import lowrank_plus_noise_np


def _proj(A):
    Q, _ = np.linalg.qr(A)
    return Q @ Q.T


def _matrix(m, n, s, seed):
    rs = np.random.default_rng(seed)
    U, _ = np.linalg.qr(rs.standard_normal((m, len(s))))
    V, _ = np.linalg.qr(rs.standard_normal((n, len(s))))
    return (U * s) @ V.T, U, V


def _omega(n, ell, seed):
    return omega(seed, 0, 0, np.arange(n), ell).astype(np.float64)


# ---- randomized subspace iteration ----------------------------------------------------------
@pytest.mark.parametrize("q", [1, 2, 3])
def test_power_range_is_the_powered_sketch(q):
    """Well-conditioned X (singular values in [1, 4]): (X X^T)^q X Omega keeps full rank in FP64,
    so its range, formed by matrix powers, is the reference."""
    Xm, _, _ = _matrix(30, 50, np.linspace(4.0, 1.0, 30), seed=1)
    Om = _omega(50, 8, seed=q)
    _, _, _, info = tucker.randsvd(Xm, 5, Om, q=q)
    Yd = np.linalg.matrix_power(Xm @ Xm.T, q) @ Xm @ Om
    assert np.abs(info["Q"] @ info["Q"].T - _proj(Yd)).max() < 1e-10
    # and q = 0 is the plain sketch of Alg. 1
    _, _, _, info0 = tucker.randsvd(Xm, 5, Om, q=0)
    assert np.abs(info0["Q"] @ info0["Q"].T - _proj(Xm @ Om)).max() < 1e-12


def test_power_reaches_the_optimal_subspace():
    s = 0.8 ** np.arange(60)
    Xm, U, _ = _matrix(80, 120, s, seed=2)
    ell, r = 10, 6
    Uh, sh, _, info = tucker.randsvd(Xm, r, _omega(120, ell, seed=3), q=60)
    Q = info["Q"]
    err2 = np.linalg.norm(Xm - Q @ (Q.T @ Xm), 2)
    assert abs(err2 - s[ell]) <= 1e-8 * s[0]                     # Eckart-Young: sigma_{ell+1}
    assert np.abs(_proj(Uh) - _proj(U[:, :r])).max() < 1e-8
    assert np.allclose(sh, s[:r], rtol=1e-10)


def test_power_expectation_bound_and_improvement():
    """Halko, Martinsson and Tropp 2011, Cor. 10.10: with B = (A A^T)^q A,
    E ||(I - P_Y) A|| <= [(1 + sqrt(k/(p-1))) s_{k+1}^{2q+1}
                          + e sqrt(k+p)/p (sum_{j>k} s_j^{2(2q+1)})^{1/2}]^{1/(2q+1)}."""
    s = 1.0 / np.sqrt(np.arange(1, 61))                          # slow decay
    Xm, _, _ = _matrix(60, 80, s, seed=4)
    k, p = 5, 4
    means = []
    for q in range(3):
        errs = []
        for seed in range(40):
            _, _, _, info = tucker.randsvd(Xm, k, _omega(80, k + p, seed), q=q)
            Q = info["Q"]
            errs.append(np.linalg.norm(Xm - Q @ (Q.T @ Xm), 2))
        t = 2 * q + 1
        bound = ((1 + math.sqrt(k / (p - 1))) * s[k] ** t
                 + math.e * math.sqrt(k + p) / p * math.sqrt(np.sum(s[k:] ** (2 * t)))) ** (1.0 / t)
        assert np.mean(errs) <= bound
        assert min(errs) >= s[k + p] * (1 - 1e-12)               # no rank-(k+p) basis beats sigma_{k+p+1}
        means.append(np.mean(errs))
    assert means[0] > means[1] > means[2]


def test_rsthosvd_with_many_power_steps_is_sthosvd():
    X = lowrank_plus_noise_np([14, 12, 10], [5, 5, 5], 0.7, 1e-2, seed=5)
    ranks = [3, 3, 3]
    Gd, Ad = tucker.sthosvd(X, ranks)
    out = tucker.rsthosvd(X, ranks, 2, seed=6, q=60)
    for n in range(3):
        assert np.abs(_proj(out["factors"][n]) - _proj(Ad[n])).max() < 1e-9
    assert abs(rel_error(X, out["core"], out["factors"]) - rel_error(X, Gd, Ad)) < 1e-12
    # the untruncated range finder spans the leading ell-dimensional subspaces instead
    ut = tucker.rsthosvd(X, ranks, 2, seed=6, q=60, truncate=False)
    G = X
    for n in tucker.default_order(X.shape):
        U, _, _ = np.linalg.svd(unfold(G, n), full_matrices=False)
        assert np.abs(_proj(ut["factors"][n]) - _proj(U[:, :5])).max() < 1e-9
        G = np.moveaxis(np.tensordot(ut["factors"][n].T, G, axes=(1, n)), 0, n)


def test_rhosvd_with_many_power_steps_is_hosvd():
    X = lowrank_plus_noise_np([14, 12, 10], [5, 5, 5], 0.7, 1e-2, seed=7)
    ranks = [3, 3, 3]
    Gd, Ad = tucker.hosvd(X, ranks)
    out = tucker.rhosvd(X, ranks, 2, seed=8, q=60)
    for n in range(3):
        assert np.abs(_proj(out["factors"][n]) - _proj(Ad[n])).max() < 1e-9
    assert abs(rel_error(X, out["core"], out["factors"]) - rel_error(X, Gd, Ad)) < 1e-12


def test_power_keeps_exact_recovery():
    X = lowrank_plus_noise_np([20, 18, 16], [4, 5, 3], 0.8, 0.0, seed=9)
    for alg in (tucker.rsthosvd, tucker.rhosvd):
        out = alg(X, [4, 5, 3], 3, seed=10, q=2)
        assert rel_error(X, out["core"], out["factors"]) < 1e-13


# ---- SP-HOSVD -------------------------------------------------------------------------------
def _sparse_tensor(seed, dims=(30, 28, 26), density=0.08):
    rs = np.random.default_rng(seed)
    X = np.zeros(dims)
    for i in range(1, 9):
        vecs = [np.where(rs.random(n) < 0.3, rs.random(n), 0.0) for n in dims]
        X += (4.0 / i ** 2) * np.einsum("i,j,k->ijk", *vecs)
    X += np.where(rs.random(dims) < density, rs.random(dims), 0.0) * 1e-2
    return X


def test_sp_hosvd_invariants():
    X = _sparse_tensor(0)
    ranks, p = [4, 4, 4], 3
    out = tucker.sp_hosvd(X, ranks, p, seed=5)
    for n, (A, P) in enumerate(zip(out["factors"], out["selected"])):
        ell = ranks[n] + p
        assert A.shape == (X.shape[n], ell) and P.size == ell
        assert np.abs(A[P, :] - np.eye(ell)).max() < 1e-12
        assert np.abs(A).max() <= 2.0 + 1e-9
        assert np.linalg.norm(A, 2) <= math.sqrt(1 + 4 * ell * (X.shape[n] - ell))
    for i, j, k in [(0, 0, 0), (2, 5, 6), (6, 6, 6)]:
        assert out["core"][i, j, k] == X[out["selected"][0][i], out["selected"][1][j], out["selected"][2][k]]


def test_sp_hosvd_exact_recovery():
    """X_(j) = A_j P_j^T X_(j) once Q_j spans range(X_(j)); applied in every mode, X = G x_j A_j."""
    rs = np.random.default_rng(3)
    dims = (24, 22, 20)
    X = np.zeros(dims)
    for _ in range(3):
        X += np.einsum("i,j,k->ijk", *[np.where(rs.random(n) < 0.5, rs.random(n), 0.0) for n in dims])
    out = tucker.sp_hosvd(X, [2, 2, 2], 2, seed=1)
    assert rel_error(X, out["core"], out["factors"]) < 1e-12


def test_sp_hosvd_seed_averaged_bound():
    """The paper states for SP-HOSVD the upper bound of Thm. pass_error (modes in order 1..d)."""
    X = _sparse_tensor(1)
    ranks, p = [3, 3, 3], 3
    bound = tucker.sp_bound(X, ranks, p)
    errs = [frob(X - multi_ttm(o["core"], o["factors"]))
            for o in (tucker.sp_hosvd(X, ranks, p, seed=s) for s in range(10))]
    assert np.mean(errs) <= bound
    assert np.mean(errs) >= math.sqrt(max(tucker.delta2(X, ranks))) * (1 - 1e-9)


def test_sp_hosvd_size_rule_is_strict():
    """Alg. 6 needs r_j + p < min(I_j, prod of the other sizes): ell = I_j is rejected."""
    X = _sparse_tensor(2, dims=(10, 9, 8))
    with pytest.raises(ValueError):
        tucker.sp_hosvd(X, [3, 3, 5], 3, seed=1)                 # mode 2: ell = 8 = I_2
    out = tucker.sp_hosvd(X, [3, 3, 4], 3, seed=1)              # ell = 7 < 8
    assert [P.size for P in out["selected"]] == [6, 6, 7]


# ---- the other subset selections (Sec. 5 remark 3) --------------------------------------------
def _lu_pivot_rows(Q):
    """Rows chosen by Gaussian elimination with partial pivoting on Q (LAPACK getrf's swaps)."""
    import scipy.linalg

    _, piv = scipy.linalg.lu_factor(Q)
    perm = np.arange(Q.shape[0])
    for i, pv in enumerate(piv):
        perm[i], perm[pv] = perm[pv], perm[i]
    return np.sort(perm[: Q.shape[1]])


def _greedy_residual_rows(Q):
    """Column-pivoted QR of Q^T by its definition: repeatedly take the row of Q with the largest
    norm after projecting out the span of the rows taken so far."""
    chosen = []
    for _ in range(Q.shape[1]):
        if chosen:
            B, _ = np.linalg.qr(Q[chosen, :].T)
            R = Q - (Q @ B) @ B.T
        else:
            R = Q
        nrm = np.sum(R * R, axis=1)
        nrm[chosen] = -1.0
        chosen.append(int(np.argmax(nrm)))
    return np.sort(np.array(chosen))


@pytest.mark.parametrize("I,ell,seed", [(40, 6, 1), (120, 20, 2), (64, 63, 3), (9, 1, 4)])
def test_deim_is_partial_pivoting(I, ell, seed):
    """DEIM's greedy equals the row pivots of LU with partial pivoting of Q (Sorensen and Embree
    2016): the residual at step j is column j of the Schur complement."""
    Q = np.linalg.qr(np.random.default_rng(seed).standard_normal((I, ell)))[0]
    assert np.array_equal(tucker.deim_select(Q), _lu_pivot_rows(Q))


@pytest.mark.parametrize("I,ell,seed", [(40, 6, 5), (120, 20, 6), (64, 63, 7)])
def test_cpqr_is_the_greedy_residual_selection(I, ell, seed):
    Q = np.linalg.qr(np.random.default_rng(seed).standard_normal((I, ell)))[0]
    assert np.array_equal(tucker.cpqr_select(Q), _greedy_residual_rows(Q))
    # and sRRQR starts from it: with eta = infinity no swap is made
    assert np.array_equal(tucker.srrqr_select(Q, eta=np.inf), tucker.cpqr_select(Q))


# ---- orthonormalising post-processing (Sec. 5) -------------------------------------------------
@pytest.mark.parametrize("alg", ["sp_sthosvd", "sp_hosvd"])
def test_orthonormalize_keeps_the_approximation(alg):
    X = _sparse_tensor(3)
    out = getattr(tucker, alg)(X, [3, 3, 3], 3, seed=4)
    G, Qs = tucker.orthonormalize_tucker(out["core"], out["factors"])
    before = multi_ttm(out["core"], out["factors"])
    after = multi_ttm(G, Qs)
    assert frob(after - before) <= 1e-12 * frob(before)
    for Q, A in zip(Qs, out["factors"]):
        assert Q.shape == A.shape
        assert np.abs(Q.T @ Q - np.eye(Q.shape[1])).max() < 1e-14 * 10 * Q.shape[1]
        assert np.abs(_proj(Q) - _proj(A)).max() < 1e-12                 # same column spaces
    # orthonormal factors: the norm of the approximation is the norm of the core
    assert abs(frob(after) - frob(G)) <= 1e-12 * frob(G)


def test_orthonormalize_of_an_orthonormal_tucker_only_flips_signs():
    X = lowrank_plus_noise_np([14, 12, 10], [4, 4, 4], 0.7, 1e-2, seed=11)
    out = tucker.rsthosvd(X, [4, 4, 4], 3, seed=12)
    G, Qs = tucker.orthonormalize_tucker(out["core"], out["factors"])
    for Q, A in zip(Qs, out["factors"]):
        assert np.allclose(np.abs(Q), np.abs(A), atol=1e-13)
    assert np.allclose(np.abs(G), np.abs(out["core"]), atol=1e-12 * np.abs(out["core"]).max())


def test_sp_hosvd_coo_equals_dense():
    X = _sparse_tensor(4)
    idx = np.argwhere(X != 0)
    vals = X[X != 0]
    out = tucker.sp_hosvd(X, [3, 3, 3], 3, seed=2)
    oc = tucker.sp_hosvd_coo(idx, vals, X.shape, [3, 3, 3], 3, seed=2)
    for n in range(3):
        assert np.array_equal(oc["selected"][n], out["selected"][n])
        assert np.allclose(oc["factors"][n], out["factors"][n], atol=1e-10)
    assert np.array_equal(oc["core"], out["core"])


@pytest.mark.parametrize("method", ["srrqr", "cpqr", "deim", "uniform", "leverage"])
@pytest.mark.parametrize("omega_round", [None, "bf16"])
def test_sp_coo_forms_equal_dense_for_every_selection(method, omega_round):
    """Alg. 6 and SP-HOSVD from the nonzeros (unique Kolda rows, scatter-add) equal the dense forms
    (the unfolding times the full Omega matrix) for every selection of Sec. 5 and for Omega rounded to
    BF16 (the BF16-Omega form of the sparse sketch): two independent computations of each sketch."""
    X = _sparse_tensor(4)
    idx = np.argwhere(X != 0)
    vals = X[X != 0]
    kw = dict(method=method, omega_round=omega_round)
    for dense, coo in ((tucker.sp_sthosvd(X, [3, 3, 3], 3, seed=2, tensor_id=1, **kw),
                        tucker.sp_sthosvd_coo(idx, vals, X.shape, [3, 3, 3], 3, seed=2, tensor_id=1, **kw)),
                       (tucker.sp_hosvd(X, [3, 3, 3], 3, seed=2, tensor_id=1, **kw),
                        tucker.sp_hosvd_coo(idx, vals, X.shape, [3, 3, 3], 3, seed=2, tensor_id=1, **kw))):
        for n in range(3):
            assert np.array_equal(coo["selected"][n], dense["selected"][n])
            assert np.allclose(coo["factors"][n], dense["factors"][n], atol=1e-10)
            A = coo["factors"][n]
            assert np.array_equal(A[coo["selected"][n]], np.eye(A.shape[1])) or \
                np.allclose(A[coo["selected"][n]], np.eye(A.shape[1]), atol=1e-12)
        assert np.array_equal(coo["core"], dense["core"])


def test_bf16_omega_sketch_is_the_rounded_stream():
    """The BF16-Omega COO sketch is X_(n) times Omega with every normal rounded to BF16 (ties to
    even): against the FP32 stream it moves by at most 2^-9 |X_(n)| |Omega|, and the rounded values
    are BF16 numbers (low 16 bits zero)."""
    from oracle.tensor import unfold

    X = _sparse_tensor(5)
    idx = np.argwhere(X != 0)
    vals = X[X != 0]
    for n in range(3):
        Yb = tucker.coo_sketch(idx, vals, X.shape, n, 6, 3, 0, omega_round="bf16")
        Yf = tucker.coo_sketch(idx, vals, X.shape, n, 6, 3, 0)
        M = X.size // X.shape[n]
        om = rng.omega(3, 0, n, np.arange(M), 6)
        omb = rng.round_bf16(om)
        assert np.all((omb.view(np.uint32) & 0xFFFF) == 0)
        assert np.allclose(Yb, unfold(X, n) @ omb.astype(np.float64), rtol=0, atol=1e-12)
        assert np.all(np.abs(Yb - Yf) <= 2.0 ** -9 * (np.abs(unfold(X, n)) @ np.abs(om.astype(np.float64))) + 1e-15)


def test_uniform_sampling_draws_every_subset_equally():
    """Uniform sampling without replacement makes every ell-subset equally likely: C(5, 2) = 10
    subsets, 3000 seeds, each count within 5 standard deviations of 300."""
    import itertools

    Q = np.linalg.qr(np.random.default_rng(1).standard_normal((5, 2)))[0]
    counts = {c: 0 for c in itertools.combinations(range(5), 2)}
    for seed in range(3000):
        counts[tuple(int(x) for x in tucker.sample_select(Q, False, seed))] += 1
    sd = math.sqrt(3000 * 0.1 * 0.9)
    assert all(abs(v - 300) <= 5 * sd for v in counts.values()), counts


def test_leverage_sampling_follows_its_law():
    """Weights w_i = ||Q(i, :)||^2 (sum ell): a pair {a, b} is drawn with probability
    w_a/T w_b/(T - w_a) + w_b/T w_a/(T - w_b), T = sum w = 2, checked on 4000 seeds."""
    import itertools

    Q = np.linalg.qr(np.random.default_rng(2).standard_normal((4, 2)) * np.array([[3.0], [1.0], [0.5], [0.2]]))[0]
    w = np.sum(Q * Q, axis=1)
    T = w.sum()
    assert abs(T - 2.0) < 1e-12
    n = 4000
    counts = {c: 0 for c in itertools.combinations(range(4), 2)}
    for seed in range(n):
        counts[tuple(int(x) for x in tucker.sample_select(Q, True, seed, stream=5))] += 1
    for (a, b), v in counts.items():
        prob = w[a] / T * w[b] / (T - w[a]) + w[b] / T * w[a] / (T - w[b])
        sd = math.sqrt(n * prob * (1 - prob))
        assert abs(v - n * prob) <= 5 * sd + 1, ((a, b), v, n * prob)


def test_adaptive_bf16_omega_is_the_rounded_stream():
    """Alg. 5 with the BF16-rounded Omega on a mode (the BF16 storage forms): that mode's range
    finder sees the FP32 normals rounded to BF16 (ties to even), so its first block's sketch is
    X_(n) times the rounded columns, and the factor differs from the FP32 stream's by the rounding
    only (the rounded stream is not the FP32 one)."""
    from oracle.tensor import unfold
    from workloads import lowrank_plus_noise_np

    X = lowrank_plus_noise_np([24, 20, 18], [5, 5, 5], 0.7, 1e-3, seed=21)
    cols = tucker._omega_cols_fn(7, 0, 0, 20 * 18, "bf16")
    om = rng.omega(7, 0, 0, np.arange(20 * 18), 4)
    omb = rng.round_bf16(om).astype(np.float64)
    assert np.array_equal(cols(0, 4), omb)
    assert not np.array_equal(omb, om.astype(np.float64))
    tol = 0.05 * np.linalg.norm(X) / np.sqrt(3)
    Ab, ib = tucker.adapt_range_finder(unfold(X, 0), tol, 4, 2, cols)
    out = tucker.adaptive_rsthosvd(X, 0.05, 4, 2, 7, rho=[0, 1, 2], omega_round={0: "bf16"})
    assert np.allclose(out["factors"][0], Ab, atol=1e-13)
    out32 = tucker.adaptive_rsthosvd(X, 0.05, 4, 2, 7, rho=[0, 1, 2])
    assert out32["factors"][0].shape == Ab.shape
    assert not np.allclose(out32["factors"][0], Ab, atol=1e-13)
