"""Pins for the oracle's Tucker algorithms (oracle.tucker) -- CPU only.

Each check is fixed by the paper or by the mathematics, not by the oracle itself:
* exact recovery of tensors with exact multilinear rank (Alg. 1-3);
* R-STHOSVD with a full-width sketch equals STHOSVD (the range finder then spans
  the whole column space);
* HOSVD factors are the leading eigenvectors of X_(j) X_(j)^T (eigh, a different
  library route) and obey Thm. lem:mode_err;
* the STHOSVD equality of Thm. lem:st_mode_err and ||X||^2 - ||G||^2;
* seed-averaged expectation bounds (Thm. randsvd_err, rhosvd_err, rst_err, pass_error);
* Table 4 of the paper for the adaptive R-STHOSVD (golden file);
* SP-STHOSVD invariants of Thm. pass_error: identity submatrix, |A_ij| <= 2,
  ||A_j||_2 <= g(I_j, l_j), core entries taken from X, COO == dense.
"""

import math
import os

import numpy as np
import pytest

from oracle import tucker
from oracle.tensor import frob, multi_ttm, rel_error, ttm, unfold
from workloads import hilbert, lowrank_plus_noise_np


def _proj(A):
    Q, _ = np.linalg.qr(A)
    return Q @ Q.T


def test_default_order_is_decreasing_size():
    assert tucker.default_order([10, 30, 20, 30]) == [1, 3, 2, 0]


@pytest.mark.parametrize("alg", ["rhosvd", "rsthosvd"])
def test_exact_multilinear_rank_is_recovered(alg):
    X = lowrank_plus_noise_np([20, 18, 16], [4, 5, 3], 0.8, 0.0, seed=1)
    f = getattr(tucker, alg)
    out = f(X, [4, 5, 3], 3, seed=11)
    assert rel_error(X, out["core"], out["factors"]) < 1e-13
    for A in out["factors"]:
        assert np.abs(A.T @ A - np.eye(A.shape[1])).max() < 1e-14 * 10 * A.shape[1]


def test_exact_rank_4way():
    X = lowrank_plus_noise_np([9, 8, 7, 6], [2, 3, 2, 3], 0.9, 0.0, seed=2)
    out = tucker.rsthosvd(X, [2, 3, 2, 3], 2, seed=3)
    assert rel_error(X, out["core"], out["factors"]) < 1e-13


def test_full_width_sketch_equals_sthosvd():
    X = lowrank_plus_noise_np([8, 7, 6], [3, 3, 3], 0.7, 1e-2, seed=4)
    ranks = [3, 3, 3]
    Gd, Ad = tucker.sthosvd(X, ranks, rho=[0, 1, 2])
    # p = I_n - r_n on every mode: ell = I_n for this cubic-ish shape in order 0,1,2
    out = tucker.rsthosvd(X, ranks, 5, seed=9, rho=[0, 1, 2], clamp=True)
    for n in range(3):
        assert np.abs(_proj(out["factors"][n]) - _proj(Ad[n])).max() < 1e-12
    assert abs(rel_error(X, out["core"], out["factors"]) - rel_error(X, Gd, Ad)) < 1e-13


def test_hosvd_factors_are_gram_eigenvectors_and_obey_bound():
    X = lowrank_plus_noise_np([7, 6, 5], [3, 3, 3], 0.6, 5e-2, seed=5)
    ranks = [2, 3, 2]
    G, A = tucker.hosvd(X, ranks)
    for n in range(3):
        w, V = np.linalg.eigh(unfold(X, n) @ unfold(X, n).T)
        V = V[:, np.argsort(w)[::-1][: ranks[n]]]
        assert np.abs(_proj(A[n]) - V @ V.T).max() < 1e-10
    err2 = frob(X - multi_ttm(G, A)) ** 2
    assert err2 <= sum(tucker.delta2(X, ranks)) * (1 + 1e-12)


def test_sthosvd_error_equalities():
    X = lowrank_plus_noise_np([8, 7, 6], [3, 3, 3], 0.6, 5e-2, seed=6)
    ranks = [2, 2, 3]
    G, A = tucker.sthosvd(X, ranks, rho=[0, 1, 2])
    err2 = frob(X - multi_ttm(G, A)) ** 2
    # sum of successive-iterate differences (Thm. lem:st_mode_err, first equality)
    Xh_prev, s = X, 0.0
    for j in range(3):
        Gj = X
        for i in range(j + 1):
            Gj = ttm(Gj, A[i].T, i)
        Xh = Gj
        for i in range(j + 1):
            Xh = ttm(Xh, A[i], i)
        s += frob(Xh_prev - Xh) ** 2
        Xh_prev = Xh
    assert abs(err2 - s) < 1e-12 * frob(X) ** 2
    assert abs(err2 - (frob(X) ** 2 - frob(G) ** 2)) < 1e-12 * frob(X) ** 2
    assert err2 <= sum(tucker.delta2(X, ranks)) * (1 + 1e-12)


def test_randsvd_expectation_bound():
    rs = np.random.default_rng(8)
    m, n, r, p = 40, 60, 5, 4
    U, _ = np.linalg.qr(rs.standard_normal((m, m)))
    V, _ = np.linalg.qr(rs.standard_normal((n, m)))
    s = 0.7 ** np.arange(m)
    Xm = (U * s) @ V.T
    bound = (1 + r / (p - 1)) * np.sum(s[r:] ** 2)
    errs = []
    from oracle.rng import omega
    for seed in range(60):
        Om = omega(seed, 0, 0, np.arange(n), r + p).astype(np.float64)
        Uh, _, _, info = tucker.randsvd(Xm, r, Om)
        Q = info["Q"]
        errs.append(frob(Xm - Q @ (Q.T @ Xm)) ** 2)
    assert np.mean(errs) <= bound
    assert min(errs) >= np.sum(s[r + p:] ** 2) * (1 - 1e-9)   # cannot beat rank r+p optimum


@pytest.mark.parametrize("alg", ["rhosvd", "rsthosvd"])
def test_seed_averaged_tensor_bound(alg):
    X = lowrank_plus_noise_np([12, 11, 10], [6, 6, 6], 0.6, 1e-2, seed=9)
    ranks, p = [3, 3, 3], 3
    bound = tucker.randomized_bound(X, ranks, p)
    f = getattr(tucker, alg)
    errs = [frob(X - multi_ttm(o["core"], o["factors"]))
            for o in (f(X, ranks, p, seed=s) for s in range(30))]
    assert np.mean(errs) <= bound
    assert np.mean(errs) >= math.sqrt(max(tucker.delta2(X, ranks))) * (1 - 1e-9)


def test_rsthosvd_norm_identity_and_projector_lemma():
    X = lowrank_plus_noise_np([14, 12, 10], [4, 4, 4], 0.7, 1e-2, seed=10)
    out = tucker.rsthosvd(X, [4, 4, 4], 4, seed=1)
    G, A = out["core"], out["factors"]
    err2 = frob(X - multi_ttm(G, A)) ** 2
    assert err2 / frob(X) ** 2 > 1e-6
    assert abs(err2 - (frob(X) ** 2 - frob(G) ** 2)) < 1e-11 * frob(X) ** 2


def test_hilbert_200_rsthosvd_near_deterministic():
    X = hilbert([200, 200, 200], offset=1)
    Gd, Ad = tucker.sthosvd(X, [20, 20, 20], rho=[0, 1, 2])
    e_det = rel_error(X, Gd, Ad)
    out = tucker.rsthosvd(X, [20, 20, 20], 5, seed=0, rho=[0, 1, 2])
    e_r = rel_error(X, out["core"], out["factors"])
    assert e_det < 1e-12 and e_r < 1e-12
    assert e_r < 10 * e_det


def _table4(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "table4_adaptive_ranks.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows.append((int(t[0]), float(t[1]), tuple(int(x) for x in t[2:5])))
    return rows


@pytest.mark.parametrize("b", [1, 8])
def test_table4_adaptive_ranks(golden_dir, b):
    rows = _table4(golden_dir)
    assert len(rows) == 15
    cache = {}
    for I, eps, ranks in rows:
        X = cache.setdefault(I, hilbert([I, I, I], offset=3))
        out = tucker.adaptive_rsthosvd(X, eps, b, 5, seed=0, rho=[0, 1, 2])
        got = tuple(A.shape[1] for A in out["factors"])
        assert got == ranks, (I, eps, got, ranks)
        assert rel_error(X, out["core"], out["factors"]) <= eps


def test_adaptive_rhosvd_meets_tolerance():
    X = lowrank_plus_noise_np([16, 15, 14], [5, 5, 5], 0.5, 1e-3, seed=12)
    for eps in (1e-1, 1e-2):
        out = tucker.adaptive_rhosvd(X, eps, 2, 3, seed=4)
        assert rel_error(X, out["core"], out["factors"]) <= eps


def _sparse_tensor(seed, dims=(30, 28, 26), density=0.08):
    rs = np.random.default_rng(seed)
    X = np.zeros(dims)
    for i in range(1, 9):
        vecs = [np.where(rs.random(n) < 0.3, rs.random(n), 0.0) for n in dims]
        X += (4.0 / i ** 2) * np.einsum("i,j,k->ijk", *vecs)
    X += np.where(rs.random(dims) < density, rs.random(dims), 0.0) * 1e-2
    return X


def test_sp_sthosvd_invariants():
    X = _sparse_tensor(0)
    ranks, p = [4, 4, 4], 3
    out = tucker.sp_sthosvd(X, ranks, p, seed=5)
    for n, (A, P) in enumerate(zip(out["factors"], out["selected"])):
        ell = ranks[n] + p
        assert A.shape == (X.shape[n], ell) and P.size == ell
        assert np.abs(A[P, :] - np.eye(ell)).max() < 1e-12
        assert np.abs(A).max() <= 2.0 + 1e-9
        assert np.linalg.norm(A, 2) <= math.sqrt(1 + 4 * ell * (X.shape[n] - ell))
    core = X[np.ix_(*out["selected"])]
    assert np.array_equal(out["core"], core)


def test_sp_sthosvd_exact_recovery():
    rs = np.random.default_rng(3)
    dims = (24, 22, 20)
    X = np.zeros(dims)
    for _ in range(3):
        X += np.einsum("i,j,k->ijk", *[np.where(rs.random(n) < 0.5, rs.random(n), 0.0) for n in dims])
    out = tucker.sp_sthosvd(X, [2, 2, 2], 2, seed=1)
    assert rel_error(X, out["core"], out["factors"]) < 1e-12


def test_sp_sthosvd_coo_equals_dense():
    X = _sparse_tensor(4)
    idx = np.argwhere(X != 0)
    vals = X[X != 0]
    out = tucker.sp_sthosvd(X, [3, 3, 3], 3, seed=2)
    oc = tucker.sp_sthosvd_coo(idx, vals, X.shape, [3, 3, 3], 3, seed=2)
    for n in range(3):
        assert np.array_equal(oc["selected"][n], out["selected"][n])
        assert np.allclose(oc["factors"][n], out["factors"][n], atol=1e-10)
    assert np.array_equal(oc["core"], out["core"])


def test_sp_sthosvd_seed_averaged_bound():
    X = _sparse_tensor(1)
    ranks, p = [3, 3, 3], 3
    bound = tucker.sp_bound(X, ranks, p, rho=tucker.default_order(X.shape))
    errs = [frob(X - multi_ttm(o["core"], o["factors"]))
            for o in (tucker.sp_sthosvd(X, ranks, p, seed=s) for s in range(10))]
    assert np.mean(errs) <= bound


def test_srrqr_condition_and_determinant_growth():
    rs = np.random.default_rng(2)
    Q, _ = np.linalg.qr(rs.standard_normal((60, 6)) * np.array([1, 1, 1, 1e-2, 1e-3, 1e-4]))
    P = tucker.srrqr_select(Q, 2.0)
    A = Q @ np.linalg.inv(Q[P])
    mask = np.ones(60, dtype=bool)
    mask[P] = False
    assert np.abs(A[mask]).max() <= 2.0 + 1e-12
    # no single swap can raise |det(P^T Q)| by more than a factor 2
    d0 = abs(np.linalg.det(Q[P]))
    for i in np.nonzero(mask)[0][:20]:
        for j in range(6):
            S = P.copy()
            S[j] = i
            assert abs(np.linalg.det(Q[S])) <= 2.0 * d0 * (1 + 1e-9)


def test_adapt_range_finder_meets_its_tolerance_without_oversampling():
    # Sec. 4's guarantee for the trimmed basis: ||G - A A^T G||_F <= tol.  With p = 0 the range
    # finder stops with ||G - Q B||_F just below tol, so the trimming has to count that residual
    # next to the discarded singular values of B
    rs = np.random.default_rng(31)
    for trial in range(12):
        m, n = 40, 60
        U = np.linalg.qr(rs.standard_normal((m, m)))[0]
        V = np.linalg.qr(rs.standard_normal((n, m)))[0]
        s = 0.7 ** np.arange(m) * (1.0 + 0.1 * rs.random(m))
        G = (U * s) @ V.T
        tol = float(rs.uniform(0.02, 0.3)) * np.linalg.norm(G)
        omega = rs.standard_normal((n, m))
        A, info = tucker.adapt_range_finder(G, tol, 1 + trial % 4, 0, lambda c0, c1: omega[:, c0:c1])
        assert np.abs(A.T @ A - np.eye(A.shape[1])).max() < 1e-12
        assert np.linalg.norm(G - A @ (A.T @ G)) <= tol * (1 + 1e-12), trial
        # and no smaller rank would do: dropping A's last column breaks the tolerance
        if A.shape[1] > 1:
            A1 = A[:, :-1]
            assert np.linalg.norm(G - A1 @ (A1.T @ G)) > tol, trial


def test_adaptive_rhosvd_ranks_of_a_superdiagonal_tensor():
    # X(k, k, k) = 2^-k, k = 0..7: every unfolding has the singular values 2^-k, ||X||^2 =
    # (1 - 4^-8) / (3/4).  With eps = 0.08, Alg. 4's per-mode tolerance eps ||X|| / sqrt(3) has
    # tol^2 = 0.0028444; the discarded energy sum_{k > r} 4^-k is 0.0051880 for r = 4 and 0.0012817
    # for r = 5, so every mode keeps rank 5 (p = 8 makes Q span the whole range, B's singular values
    # are the 2^-k).  The approximation keeps the entries k < 5, so the error is
    # sqrt(0.0012817) / ||X|| = 0.0310 <= eps.
    X = np.zeros((8, 8, 8))
    for k in range(8):
        X[k, k, k] = 2.0 ** -k
    for b in (1, 2, 3):
        out = tucker.adaptive_rhosvd(X, 0.08, b, 8, seed=3)
        assert [A.shape[1] for A in out["factors"]] == [5, 5, 5], b
        e = rel_error(X, out["core"], out["factors"])
        assert abs(e - math.sqrt((4.0 ** -5 + 4.0 ** -6 + 4.0 ** -7) / ((1 - 4.0 ** -8) / 0.75))) < 1e-12


def test_randomized_bound_is_at_least_the_best_tucker_error():
    # Thm. rhosvd_err / rst_err bound the expected error, and no rank-(r_1, ..., r_d) Tucker
    # approximation has an error below max_j Delta_j (its mode-j unfolding has rank <= r_j), so the
    # bound can never be smaller -- also for a large oversampling p, where r / (p - 1) is small
    X = lowrank_plus_noise_np([20, 18, 16], [6, 6, 6], 0.8, 1e-2, seed=8)
    ranks = [4, 4, 4]
    lower = max(np.linalg.norm(np.linalg.svd(unfold(X, n), compute_uv=False)[4:]) for n in range(3))
    for p in (2, 5, 41, 401):
        assert tucker.randomized_bound(X, ranks, p) >= lower
    # and at p -> infinity the bound tends to the deterministic HOSVD bound sqrt(sum_j Delta_j^2)
    hosvd_bound = math.sqrt(sum(np.sum(np.linalg.svd(unfold(X, n), compute_uv=False)[4:] ** 2) for n in range(3)))
    assert abs(tucker.randomized_bound(X, ranks, 4001) / hosvd_bound - 1.0) < 2e-3


def test_clamped_sketch_width_obeys_the_size_requirement():
    # Alg. 1-3 need r + p <= min(I_n, product of the other current sizes); clamping takes the widest
    # sketch the requirement allows.  30 x 3 x 2, ranks (5, 2, 2), p = 10, modes in order 0, 1, 2:
    # R-STHOSVD: mode 0 has 6 other entries (ell 6, rank 5), mode 1 I = 3 (ell 3, rank 2), mode 2
    # I = 2 (ell 2); R-HOSVD: 6, 3 and 2 as well (I_1 = 3, I_2 = 2 bind there)
    X = lowrank_plus_noise_np([30, 3, 2], [3, 2, 2], 0.8, 1e-3, seed=6)
    for alg in ("rsthosvd", "rhosvd"):
        out = getattr(tucker, alg)(X, [5, 2, 2], 10, seed=1, clamp=True, record=True)
        assert [rec["ell"] for rec in out["records"]] == [6, 3, 2], alg
        assert [rec["Y"].shape[1] for rec in out["records"]] == [6, 3, 2], alg
        assert [A.shape[1] for A in out["factors"]] == [5, 2, 2], alg
    with pytest.raises(ValueError):
        tucker.rsthosvd(X, [5, 2, 2], 10, seed=1)


def test_factor_columns_follow_the_sign_convention():
    # the QR and the SVD of Alg. 1 fix each column only up to sign; the convention used on both
    # sides of the parity tests: a column's entry of largest magnitude is positive
    X = lowrank_plus_noise_np([12, 10, 9], [4, 4, 4], 0.8, 1e-2, seed=13)
    outs = [tucker.rsthosvd(X, [3, 3, 3], 2, seed=5), tucker.rhosvd(X, [3, 3, 3], 2, seed=5),
            tucker.rsthosvd(X, [3, 3, 3], 2, seed=5, truncate=False)]
    for out in outs:
        for A in out["factors"]:
            j = np.argmax(np.abs(A), axis=0)
            assert np.all(A[j, np.arange(A.shape[1])] > 0)


def test_sp_bound_of_a_superdiagonal_tensor():
    # Thm. pass_error's right side evaluated by hand on X(k, k, k) = 2^-k (8 x 8 x 8), ranks 2,
    # p = 2: ell = 4, the growth factor g(8, 4) = sqrt(1 + 4 * 4 * (8 - 4)) = sqrt(65) multiplies
    # up over the processed modes, Delta_j^2 = sum_{k >= 2} 4^-k = 0.08331298828125 on every mode and
    # sqrt(1 + r / (p - 1)) = sqrt(3): bound = sqrt(3) Delta (g + g^2 + g^3) = 298.5180588273678
    X = np.zeros((8, 8, 8))
    for k in range(8):
        X[k, k, k] = 2.0 ** -k
    assert abs(tucker.sp_bound(X, [2, 2, 2], 2) - 298.5180588273678) < 1e-9
    assert abs(tucker.randomized_bound(X, [2, 2, 2], 2) - math.sqrt(3 * 3 * 0.08331298828125)) < 1e-12


def test_adaptive_on_exactly_rank_deficient_unfoldings():
    # X(k, k, k) = 2^-k, k = 0..7, in a 10 x 9 x 8 array: the unfoldings have rank 8 < I_1 = 10, and
    # after the first truncation Alg. 5's next unfolding has rank 5 < I_2 = 9, so the oversampling
    # columns fall inside the range already found.  The range finder's Q must stay orthonormal there:
    # both algorithms keep the hand-computed rank 5 per mode (the superdiagonal case above), with
    # orthonormal factors and the error sqrt(sum_{k >= 5} 4^-k) / ||X||
    X = np.zeros((10, 9, 8))
    for k in range(8):
        X[k, k, k] = 2.0 ** -k
    want = math.sqrt((4.0 ** -5 + 4.0 ** -6 + 4.0 ** -7) / ((1 - 4.0 ** -8) / 0.75))
    for b in (1, 2, 3):
        for out in (tucker.adaptive_rhosvd(X, 0.08, b, 8, seed=3), tucker.adaptive_rsthosvd(X, 0.08, b, 8, seed=3)):
            assert [A.shape[1] for A in out["factors"]] == [5, 5, 5], b
            for A in out["factors"]:
                assert np.abs(A.T @ A - np.eye(A.shape[1])).max() < 1e-13
            assert abs(rel_error(X, out["core"], out["factors"]) - want) < 1e-12
    # the QB decomposition itself: an exactly rank-3 matrix with zero rows and oversampling past its
    # rank; Q stays orthonormal and ||G - Q B|| vanishes
    rs = np.random.default_rng(2)
    G = np.zeros((12, 30))
    G[:6] = rs.standard_normal((6, 3)) @ rs.standard_normal((3, 30))
    omega = rs.standard_normal((30, 12))
    A, info = tucker.adapt_range_finder(G, 1e-9 * np.linalg.norm(G), 2, 8, lambda c0, c1: omega[:, c0:c1])
    assert info["ell"] > 3 and A.shape[1] == 3 and info["res2"] < 1e-24 * np.linalg.norm(G) ** 2
    assert np.abs(A.T @ A - np.eye(3)).max() < 1e-13
    assert np.linalg.norm(G - A @ (A.T @ G)) < 1e-12 * np.linalg.norm(G)
