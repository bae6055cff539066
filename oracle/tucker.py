"""Tucker compression algorithms of the paper -- plain FP64 oracle (test infrastructure).

Each function follows the algorithm it names step by step, in the paper's order:

* ``randsvd``            Alg. 1 (RandSVD)
* ``hosvd``, ``sthosvd``  Sec. 2.2 (deterministic, full SVD of each unfolding)
* ``rhosvd``             Alg. 2 (R-HOSVD)
* ``rsthosvd``           Alg. 3 (R-STHOSVD)
* ``adapt_range_finder`` Sec. 4 (blocked randomized QB with an error indicator)
* ``adaptive_rhosvd``    Alg. 4,  ``adaptive_rsthosvd`` Alg. 5
* ``srrqr_select``       strong RRQR subset selection with eta = 2 (Alg. 6, step 4);
  ``cpqr_select``, ``deim_select``, ``sample_select`` the other selections of Sec. 5
* ``sp_sthosvd``         Alg. 6 (SP-STHOSVD), dense or COO input
* ``sp_hosvd``           SP-HOSVD, Alg. 6 with independent modes (Sec. 5 remark 1), dense or COO input
* ``orthonormalize_tucker`` the orthonormalising post-processing of Sec. 5
* ``randsvd(q=...)``     Alg. 1 with randomized subspace iteration (Sec. 5 remark 2, Sec. 6)

Library primitives used as single steps: numpy matmul, ``numpy.linalg.qr``
(Householder), ``numpy.linalg.svd``, ``scipy.linalg.qr`` with column pivoting.
Omega comes from ``oracle.rng.omega`` (this library's stream specification).
"""

import math

import numpy as np
import scipy.linalg

from . import rng
from .tensor import fold, frob, multi_ttm, ttm, unfold


# ---------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------
def default_order(dims):
    """Processing order: decreasing mode size, ties to the lower mode (Sec. 3.3)."""
    return sorted(range(len(dims)), key=lambda n: (-int(dims[n]), n))


def omega_matrix(seed, tensor_id, mode, nrows, ell, omega_round=None):
    """Omega_mode as an FP64 matrix (nrows x ell); FP32 normals promoted exactly.

    ``omega_round='bf16'`` rounds each normal to BF16 first (the BF16 forms); a dict maps
    modes to their rounding (modes not in it use the FP32 normals).
    """
    if isinstance(omega_round, dict):
        omega_round = omega_round.get(mode)
    om = rng.omega(seed, tensor_id, mode, np.arange(nrows, dtype=np.int64), ell)
    if omega_round == "bf16":
        om = rng.round_bf16(om)
    elif omega_round is not None:
        raise ValueError(omega_round)
    return om.astype(np.float64)


def _check_ell(ell, I, M, strict=False):
    ok = ell < min(I, M) if strict else ell <= min(I, M)
    if not ok:
        raise ValueError(f"r+p={ell} violates the size requirement against I={I}, prod(others)={M}")


def _ell(r, p, I, M, clamp, strict=False):
    ell = int(r) + int(p)
    if clamp:
        return min(ell, int(I), int(M))
    _check_ell(ell, I, M, strict)
    return ell


def canon_signs(U):
    """Column signs making the largest-magnitude entry of each column positive (first index on ties).

    The thin QR and the SVD of Alg. 1 fix their columns only up to sign.  In the
    sequential algorithms the sign of A_j changes the next core and hence the next
    sketch, so the library fixes this convention on both sides.
    """
    U = np.asarray(U)
    if U.shape[0] == 0:
        return np.ones(U.shape[1])
    idx = np.argmax(np.abs(U), axis=0)
    v = U[idx, np.arange(U.shape[1])]
    return np.where(v < 0, -1.0, 1.0)


def canon_qr(Y):
    """Thin Householder QR of Y with the column-sign convention of ``canon_signs`` applied to Q."""
    Q, _ = np.linalg.qr(Y)
    return Q * canon_signs(Q)


# ---------------------------------------------------------------------------------
# Alg. 1 -- RandSVD
# ---------------------------------------------------------------------------------
def randsvd(Xm, r, Omega, q=0):
    """Alg. 1: Y = X Omega; Y = QR; B = Q^T X; B = U_B S V^T; U = Q U_B(:, 1:r).

    ``q`` > 0 adds q steps of randomized subspace iteration to the range finder (the variant
    named in Sec. 5's remark on range finding and used with q = 1 for the Olivetti data in
    Sec. 6; Halko, Martinsson and Tropp 2011, Alg. 4.3): Q spans (X X^T)^q X Omega.  Read here
    in the re-orthonormalised form of the same reference (a thin QR after every application of
    X^T and of X), which spans the same subspace in exact arithmetic and keeps the directions
    below sigma_1 * u^(1/(2q+1)) that the plain power loses.

    Column signs of Q and of U follow ``canon_signs``; the flip of U's column k is
    applied to U_B(:, k) and V(:, k) as well, so U S V^T is unchanged.
    """
    Y = Xm @ Omega                                  # step 1
    Q = canon_qr(Y)                                 # step 2 (thin, Householder)
    for _ in range(int(q)):                         # subspace iteration
        W = canon_qr(Xm.T @ Q)
        Y = Xm @ W
        Q = canon_qr(Y)
    B = Q.T @ Xm                                    # step 3
    Ub, s, Vt = np.linalg.svd(B, full_matrices=False)   # step 4
    U = Q @ Ub[:, :r]                               # step 5
    sg = canon_signs(U)
    U = U * sg
    Ub = Ub.copy()
    Ub[:, :r] *= sg
    Vt = Vt.copy()
    Vt[:r] *= sg[:, None]
    return U, s[:r], Vt[:r].T, {"Y": Y, "Q": Q, "sv_B": s, "Ub": Ub}   # step 6


# ---------------------------------------------------------------------------------
# Sec. 2.2 -- deterministic HOSVD / STHOSVD
# ---------------------------------------------------------------------------------
def _leading_left_sv(Mat, r):
    U, s, _ = np.linalg.svd(Mat, full_matrices=False)
    return U[:, :r], s


def hosvd(X, ranks):
    """HOSVD: A_j = first r_j left singular vectors of X_(j); G = X x_j A_j^T."""
    X = np.asarray(X, dtype=np.float64)
    A = [_leading_left_sv(unfold(X, n), ranks[n])[0] for n in range(X.ndim)]
    return multi_ttm(X, A, transpose=True), A


def sthosvd(X, ranks, rho=None):
    """STHOSVD: for j in rho, A_j from the SVD of G_(j), then G <- G x_j A_j^T."""
    X = np.asarray(X, dtype=np.float64)
    rho = default_order(X.shape) if rho is None else list(rho)
    G = X
    A = [None] * X.ndim
    for n in rho:
        A[n] = _leading_left_sv(unfold(G, n), ranks[n])[0]
        G = ttm(G, A[n].T, n)
    return G, A


# ---------------------------------------------------------------------------------
# Alg. 2 / Alg. 3
# ---------------------------------------------------------------------------------
def rhosvd(X, ranks, p, seed, tensor_id=0, omega_round=None, clamp=False, record=False, q=0):
    """Alg. 2 (R-HOSVD): RandSVD of every X_(j) with its own Omega_j, then G = X x_j A_j^T.
    ``q``: subspace-iteration steps of every RandSVD (see ``randsvd``)."""
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    N = X.size
    A = [None] * d
    recs = []
    for n in range(d):
        I = X.shape[n]
        M = N // I
        ell = _ell(ranks[n], p, I, M, clamp)
        Om = omega_matrix(seed, tensor_id, n, M, ell, omega_round)     # step 2
        U, s, V, info = randsvd(unfold(X, n), min(ranks[n], ell), Om, q)  # step 3
        A[n] = U                                                         # step 4
        recs.append(dict(mode=n, ell=ell, **info))
    G = multi_ttm(X, A, transpose=True)                                 # step 6
    out = {"core": G, "factors": A}
    if record:
        out["records"] = recs
    return out


def rsthosvd(X, ranks, p, seed, rho=None, tensor_id=0, omega_round=None, clamp=False, record=False,
             truncate=True, q=0):
    """Alg. 3 (R-STHOSVD).

    G = X; for j = 1..d: Omega_{rho_j} over the current other-mode extent;
    [U, S, V] = RandSVD(G_(rho_j), r, p, Omega); A_{rho_j} = U; G_(rho_j) <- S V^T.
    ``truncate=False`` stops RandSVD after step 3: A_{rho_j} = Q, G_(rho_j) <- Q^T G_(rho_j)
    (the untruncated core G = X x_1 Q_1^T ... of the range finder).  ``q``: subspace-iteration
    steps of every RandSVD, on the current core's unfolding (see ``randsvd``).
    """
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    rho = default_order(X.shape) if rho is None else [int(n) for n in rho]
    if sorted(rho) != list(range(d)):
        raise ValueError("rho must be a permutation of the modes")
    G = X                                                                # step 1
    A = [None] * d
    recs = []
    for n in rho:                                                        # step 2
        shape = list(G.shape)
        I = shape[n]
        M = G.size // I
        ell = _ell(ranks[n], p, I, M, clamp)
        r = min(int(ranks[n]), ell)
        Om = omega_matrix(seed, tensor_id, n, M, ell, omega_round)       # step 3
        if not truncate:
            Gm = unfold(G, n)
            Y = Gm @ Om
            Q = canon_qr(Y)
            for _ in range(int(q)):
                Y = Gm @ canon_qr(Gm.T @ Q)
                Q = canon_qr(Y)
            A[n] = Q
            shape[n] = ell
            G = fold(Q.T @ Gm, n, shape)
            recs.append(dict(mode=n, ell=ell, Y=Y, Q=Q, sv_B=np.linalg.svd(Q.T @ Gm, compute_uv=False)))
            continue
        U, s, V, info = randsvd(unfold(G, n), r, Om, q)                  # step 4
        A[n] = U                                                         # step 5
        shape[n] = r
        G = fold(s[:, None] * V.T, n, shape)                             # step 6
        recs.append(dict(mode=n, ell=ell, **info))
    out = {"core": G, "factors": A, "rho": rho}                          # step 8
    if record:
        out["records"] = recs
    return out


# ---------------------------------------------------------------------------------
# Sec. 4 -- adaptive variants
# ---------------------------------------------------------------------------------
def adapt_range_finder(Gm, tol, b, p, omega_cols, cap=None):
    """AdaptRangeFinder(G, tol, b) as a blocked randomized QB (Sec. 4).

    Reading used (the paper names the algorithm of Martinsson-Voronin refined by
    Yu-Gu-Li without listing it):
      1. grow Q by blocks of b columns, Q_i = orth((I - Q Q^T) G Omega_i) with one
         re-orthogonalisation, B_i = Q_i^T G, until ||G - Q B||_F <= tol (absolute);
      2. add p further columns of the same Omega stream;
      3. SVD of B and trim to the smallest r whose discarded energy
         sum_{i>r} sigma_i^2 + ||G - Q B||_F^2 is <= tol^2 (r >= 1).
    The residuals are formed directly (no norm-difference cancellation).
    ``omega_cols(c0, c1)`` returns columns c0:c1 of Omega as FP64.
    Returns (A, info).
    """
    m, n = Gm.shape
    kmax = min(m, n) if cap is None else min(int(cap), m, n)
    Q = np.zeros((m, 0))
    B = np.zeros((0, n))
    tol2 = float(tol) ** 2
    gnorm = frob(Gm)

    def grow(Q, B, nb):
        k = Q.shape[1]
        Y = Gm @ omega_cols(k, k + nb)
        Y = Y - Q @ (Q.T @ Y)
        Qi, Ri = np.linalg.qr(Y)
        if np.abs(np.diag(Ri)).min() <= 1e-12 * gnorm:
            # part of the block lies in span(Q) up to rounding: G is exactly rank deficient and Q
            # already holds (part of) the block's range, so the QR of the rounding noise left by the
            # projection would give directions that are not orthogonal to Q.  The block's columns
            # are taken from a complete Householder QR of [Q, Y] instead (its columns k .. k + nb - 1
            # are orthonormal to Q), which keeps the QB decomposition's Q orthonormal; B gains rows of
            # (numerically) zero energy.
            Qi = np.linalg.qr(np.hstack([Q, Y]), mode="complete")[0][:, k:k + nb]
        Qi = Qi - Q @ (Q.T @ Qi)
        Qi = canon_qr(Qi)
        Bi = Qi.T @ Gm
        return np.hstack([Q, Qi]), np.vstack([B, Bi])

    k = 0
    while k < kmax:
        Q, B = grow(Q, B, min(b, kmax - k))
        k = Q.shape[1]
        if frob(Gm - Q @ B) ** 2 <= tol2:
            break
    k_found = k
    extra = min(int(p), min(m, n) - k)
    if extra > 0:
        Q, B = grow(Q, B, extra)
    res2 = frob(Gm - Q @ B) ** 2
    Ub, s, _ = np.linalg.svd(B, full_matrices=False)
    tails = np.array([np.sum(s[r:] ** 2) + res2 for r in range(1, s.size + 1)])
    ok = np.nonzero(tails <= tol2)[0]
    r = int(ok[0]) + 1 if ok.size else int(s.size)
    A = Q @ Ub[:, :r]
    A = A * canon_signs(A)
    return A, {"k": k_found, "ell": Q.shape[1], "rank": r, "sv_B": s, "res2": res2}


def _omega_cols_fn(seed, tensor_id, mode, nrows, omega_round=None):
    cache = {}
    if isinstance(omega_round, dict):
        omega_round = omega_round.get(mode)

    def cols(c0, c1):
        need = c1
        if cache.get("ell", 0) < need:
            ell = max(need, 2 * cache.get("ell", 0), 8)
            om = rng.omega(seed, tensor_id, mode, np.arange(nrows, dtype=np.int64), ell)
            if omega_round == "bf16":
                om = rng.round_bf16(om)
            elif omega_round is not None:
                raise ValueError(omega_round)
            cache["om"] = om.astype(np.float64)
            cache["ell"] = ell
        return cache["om"][:, c0:c1]

    return cols


def adaptive_rhosvd(X, eps, b, p, seed, tensor_id=0, max_ranks=None):
    """Alg. 4: A_j = AdaptRangeFinder(X_(j), eps ||X|| / sqrt(d), b); G = X x_j A_j^T."""
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    tol = eps * frob(X) / math.sqrt(d)
    A = [None] * d
    infos = []
    for n in range(d):
        Xm = unfold(X, n)
        cap = None if max_ranks is None else max_ranks[n]
        A[n], info = adapt_range_finder(Xm, tol, b, p, _omega_cols_fn(seed, tensor_id, n, Xm.shape[1]), cap)
        infos.append(info)
    return {"core": multi_ttm(X, A, transpose=True), "factors": A, "infos": infos}


def adaptive_rsthosvd(X, eps, b, p, seed, rho=None, tensor_id=0, max_ranks=None, omega_round=None):
    """Alg. 5: G = X; for j in rho: A = AdaptRangeFinder(G_(j), eps ||X|| / sqrt(d), b); G <- A^T G_(j).

    The tolerance is absolute, eps ||X||_F / sqrt(d) with the norm of the input X,
    so that the successive iterates obey the bound stated before Alg. 5.  ``omega_round`` as in
    omega_matrix (per-mode BF16 rounding of the normals).
    """
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    rho = default_order(X.shape) if rho is None else list(rho)
    tol = eps * frob(X) / math.sqrt(d)
    G = X
    A = [None] * d
    infos = []
    for n in rho:
        Gm = unfold(G, n)
        cap = None if max_ranks is None else max_ranks[n]
        A[n], info = adapt_range_finder(Gm, tol, b, p, _omega_cols_fn(seed, tensor_id, n, Gm.shape[1], omega_round),
                                        cap)
        infos.append(info)
        G = ttm(G, A[n].T, n)
    return {"core": G, "factors": A, "infos": infos, "rho": rho}


# ---------------------------------------------------------------------------------
# Sec. 5 -- structure-preserving STHOSVD
# ---------------------------------------------------------------------------------
def cpqr_select(Q):
    """Subset selection by column-pivoted QR of Q^T alone (Sec. 5 remark 3): the first ell pivots of
    scipy's pivoted Householder QR, sorted.  No bound on |A_ij| (it can fail on adversarial inputs)."""
    ell = Q.shape[1]
    _, _, piv = scipy.linalg.qr(Q.T, pivoting=True, mode="economic")
    return np.array(sorted(int(x) for x in piv[:ell]), dtype=np.int64)


def deim_select(Q):
    """Subset selection by DEIM (Sec. 5 selection operators; Chaturantabut and Sorensen 2010,
    Sorensen and Embree 2016): p_1 = argmax |Q(:, 1)|; for j = 2..ell interpolate column j at the
    indices so far, Q(P, 1:j-1) c = Q(P, j), and take p_j = argmax |Q(:, j) - Q(:, 1:j-1) c|
    (first index on ties).  Returns the indices sorted."""
    I, ell = Q.shape
    p = [int(np.argmax(np.abs(Q[:, 0])))]
    for j in range(1, ell):
        c = np.linalg.solve(Q[p, :j], Q[p, j])
        r = Q[:, j] - Q[:, :j] @ c
        p.append(int(np.argmax(np.abs(r))))
    return np.array(sorted(p), dtype=np.int64)


def sample_select(Q, leverage, seed, stream=0):
    """Subset selection by sampling (Sec. 5 remark 3: uniform or leverage-score sampling), read as
    ell rows drawn without replacement with weights 1 or ||Q(i, :)||^2: draw k takes the first
    untaken row (increasing i) whose running weight sum exceeds u_k times the untaken total (FP64
    sums in row order); u_k = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53 from the Philox4x32-10 words of
    counter (k, stream, 0, 0x53454C45) under key (seed lo, seed hi).  Returns the rows sorted."""
    I, ell = Q.shape
    if leverage:
        w = []
        for i in range(I):
            s_ = 0.0
            for c in range(ell):
                s_ = s_ + float(Q[i, c]) * float(Q[i, c])
            w.append(s_)
    else:
        w = [1.0] * I
    taken = [False] * I
    out = []
    k0, k1 = int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF
    for k in range(ell):
        words = rng.philox4x32_10(np.uint32(k), np.uint32(stream), np.uint32(0), np.uint32(0x53454C45),
                                  np.uint32(k0), np.uint32(k1))
        w0, w1 = int(np.asarray(words[0]).ravel()[0]), int(np.asarray(words[1]).ravel()[0])
        u = ((w0 >> 5) * 67108864.0 + (w1 >> 6)) * 2.0 ** -53
        T = 0.0
        for i in range(I):
            if not taken[i]:
                T = T + w[i]
        if not T > 0.0:
            raise ValueError("no sampling weight left")
        t = u * T
        pick, last, c = -1, -1, 0.0
        for i in range(I):
            if taken[i]:
                continue
            c = c + w[i]
            if w[i] > 0.0:
                last = i
            if c > t:
                pick = i
                break
        if pick < 0:
            pick = last
        taken[pick] = True
        out.append(pick)
    return np.array(sorted(out), dtype=np.int64)


def srrqr_select(Q, eta=2.0, max_swaps=100000):
    """Strong RRQR subset selection on Q^T (Alg. 6, step 4) with k = ell = rank.

    With k equal to the number of rows of Q^T the trailing block R_22 is empty and
    the strong-RRQR condition reduces to |(R_11^{-1} R_12)_{ij}| <= eta, i.e.
    max |A_ij| <= eta over the unselected rows of A = Q (P^T Q)^{-1}.
    Start from column-pivoted QR of Q^T; while some |A_ij| > eta swap selected
    row j with row i (largest |A_ij|, then lowest (i, j)).  Each swap multiplies
    |det(P^T Q)| by |A_ij| > eta, so the loop ends.  Returns sorted row indices.
    """
    I, ell = Q.shape
    _, _, piv = scipy.linalg.qr(Q.T, pivoting=True, mode="economic")
    sel = [int(x) for x in piv[:ell]]
    for _ in range(max_swaps):
        A = Q @ np.linalg.inv(Q[sel, :])
        mask = np.ones(I, dtype=bool)
        mask[sel] = False
        absA = np.abs(A) * mask[:, None]
        amax = absA.max()
        if amax <= eta:
            break
        i, j = [int(v) for v in np.argwhere(absA == amax)[0]]
        sel[j] = i
    return np.array(sorted(sel), dtype=np.int64)


SELECT_METHODS = ("srrqr", "cpqr", "deim", "uniform", "leverage")


def select_rows(Q, method="srrqr", eta=2.0, seed=0, stream=0):
    """The row selection of Alg. 6 step 6 by one of the methods of Sec. 5 (strong RRQR, the
    default; column-pivoted QR, DEIM, uniform or leverage-score sampling).  The sampling methods
    draw with (seed, stream); the library passes stream = (tensor_id << 4) | mode."""
    if method == "srrqr":
        return srrqr_select(Q, eta)
    if method == "cpqr":
        return cpqr_select(Q)
    if method == "deim":
        return deim_select(Q)
    if method in ("uniform", "leverage"):
        return sample_select(Q, method == "leverage", seed, stream)
    raise ValueError(method)


def sp_sthosvd(X, ranks, p, seed, rho=None, tensor_id=0, eta=2.0, record=False, method="srrqr", omega_round=None):
    """Alg. 6 (SP-STHOSVD) on a dense tensor (``method``: the row selection of step 6, see
    ``select_rows``; ``omega_round='bf16'``: Omega rounded to BF16).

    G = X; for j in rho: Y = G_(j) Omega_j; Y = Q R; P_j by strong RRQR on Q^T;
    A_j = Q (P_j^T Q)^{-1}; G_(j) <- P_j^T G_(j).  The core holds entries of X.
    Requires r_j + p < min(I_j, prod_{i != j} I_i) (strict).
    """
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    rho = default_order(X.shape) if rho is None else list(rho)
    G = X
    A = [None] * d
    sel = [None] * d
    recs = []
    for n in rho:
        I = G.shape[n]
        M = G.size // I
        ell = _ell(ranks[n], p, I, M, clamp=False, strict=True)
        Om = omega_matrix(seed, tensor_id, n, M, ell, omega_round)        # step 3
        Y = unfold(G, n) @ Om                                             # step 4
        Q, _ = np.linalg.qr(Y)                                            # step 5
        P = select_rows(Q, method, eta, seed, (int(tensor_id) << 4) | n)  # step 6
        A[n] = Q @ np.linalg.inv(Q[P, :])                                 # step 7
        sel[n] = P
        G = np.take(G, P, axis=n)                                         # step 8
        recs.append(dict(mode=n, ell=ell, Y=Y, Q=Q))
    out = {"core": G, "factors": A, "selected": sel, "rho": rho}
    if record:
        out["records"] = recs
    return out


def sp_hosvd(X, ranks, p, seed, tensor_id=0, eta=2.0, method="srrqr", omega_round=None):
    """SP-HOSVD (Sec. 5, first remark after Alg. 6): the modes of Alg. 6 handled independently.

    For every mode j of the input: Y = X_(j) Omega_j; Y = QR; P_j by strong RRQR on Q^T;
    A_j = Q (P_j^T Q)^{-1}.  The core is G = X x_1 P_1^T ... x_d P_d^T, the entries of X at the
    selected coordinates.  Alg. 6's strict size rule r_j + p < min(I_j, prod_{i != j} I_i) on the
    input sizes; Omega_j is the stream of R-HOSVD's mode j.
    """
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    A = [None] * d
    sel = [None] * d
    for n in range(d):
        I = X.shape[n]
        M = X.size // I
        ell = _ell(ranks[n], p, I, M, clamp=False, strict=True)
        Om = omega_matrix(seed, tensor_id, n, M, ell, omega_round)
        Y = unfold(X, n) @ Om
        Q, _ = np.linalg.qr(Y)
        P = select_rows(Q, method, eta, seed, (int(tensor_id) << 4) | n)
        A[n] = Q @ np.linalg.inv(Q[P, :])
        sel[n] = P
    G = X[np.ix_(*sel)]
    return {"core": G, "factors": A, "selected": sel}


def orthonormalize_tucker(core, factors):
    """Post-processing of Sec. 5 for the non-orthonormal factors of Alg. 6 and SP-HOSVD: a thin QR
    of every factor, A_j = Q_j R_j, and the aggregation of the triangles into the core,
    G <- G x_1 R_1 ... x_d R_d.  The approximation G x_j A_j is unchanged."""
    Qs, G = [], np.asarray(core, dtype=np.float64)
    for n, A in enumerate(factors):
        Q, R = np.linalg.qr(A)
        Qs.append(Q)
        G = ttm(G, R, n)
    return G, Qs


def _kolda_rows(idx, dims, n):
    """Kolda column index of the mode-n unfolding for COO coordinates (earlier modes fastest)."""
    row = np.zeros(idx.shape[0], dtype=np.int64)
    stride = 1
    for k in range(len(dims)):
        if k == n:
            continue
        row += idx[:, k].astype(np.int64) * stride
        stride *= int(dims[k])
    return row


def coo_sketch(idx, vals, dims, n, ell, seed, tensor_id=0, omega_round=None):
    """Y = G_(n) Omega_n from COO entries without densifying (Alg. 6, step 4).
    ``omega_round='bf16'``: every normal rounded to BF16 first (the BF16-Omega form)."""
    rows = _kolda_rows(idx, dims, n)
    urows, inv = np.unique(rows, return_inverse=True)
    om = rng.omega(seed, tensor_id, n, urows, ell)
    if omega_round == "bf16":
        om = rng.round_bf16(om)
    elif omega_round is not None:
        raise ValueError(omega_round)
    om = om.astype(np.float64)
    Y = np.zeros((int(dims[n]), ell))
    np.add.at(Y, idx[:, n].astype(np.int64), vals.astype(np.float64)[:, None] * om[inv])
    return Y


def sp_sthosvd_coo(idx, vals, dims, ranks, p, seed, rho=None, tensor_id=0, eta=2.0, method="srrqr",
                   omega_round=None):
    """Alg. 6 on a COO tensor (0-based coordinates ``idx`` of shape nnz x d).

    Same steps as ``sp_sthosvd``; G_(j) <- P_j^T G_(j) keeps the nonzeros whose
    mode-j coordinate is selected and renumbers that coordinate to its position in
    the (sorted) selection.  The final core is the dense ell_1 x ... x ell_d array
    of the surviving entries.  ``method`` picks the row selection of step 6 (``select_rows``,
    stream (tensor_id << 4) | mode for the sampling methods); ``omega_round='bf16'`` the
    BF16-Omega sketch.
    """
    idx = np.asarray(idx, dtype=np.int64).copy()
    vals = np.asarray(vals, dtype=np.float64).copy()
    dims = [int(x) for x in dims]
    d = len(dims)
    rho = default_order(dims) if rho is None else list(rho)
    A = [None] * d
    sel = [None] * d
    for n in rho:
        I = dims[n]
        M = int(np.prod(dims)) // I
        ell = _ell(ranks[n], p, I, M, clamp=False, strict=True)
        Y = coo_sketch(idx, vals, dims, n, ell, seed, tensor_id, omega_round)
        Q, _ = np.linalg.qr(Y)
        P = select_rows(Q, method, eta, seed, (int(tensor_id) << 4) | n)
        A[n] = Q @ np.linalg.inv(Q[P, :])
        sel[n] = P
        pos = np.full(I, -1, dtype=np.int64)
        pos[P] = np.arange(P.size)
        keep = pos[idx[:, n]] >= 0
        idx = idx[keep]
        vals = vals[keep]
        idx[:, n] = pos[idx[:, n]]
        dims[n] = int(P.size)
    core = np.zeros(dims)
    if idx.shape[0]:
        core[tuple(idx.T)] = vals
    return {"core": core, "factors": A, "selected": sel, "rho": rho}


def sp_hosvd_coo(idx, vals, dims, ranks, p, seed, tensor_id=0, eta=2.0, method="srrqr", omega_round=None):
    """SP-HOSVD (Sec. 5 remark 1) of a COO tensor: every mode's sketch from the input's nonzeros
    (``coo_sketch``), thin QR, strong-RRQR selection and A_j = Q (P_j^T Q)^{-1}; the core keeps the
    nonzeros whose every coordinate is selected, renumbered to positions in the sorted selections.
    ``method`` and ``omega_round`` as in ``sp_sthosvd_coo``."""
    idx = np.asarray(idx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    dims = [int(x) for x in dims]
    d = len(dims)
    N = int(np.prod(dims))
    A = [None] * d
    sel = [None] * d
    keep = np.ones(idx.shape[0], dtype=bool)
    new = idx.copy()
    for n in range(d):
        ell = _ell(ranks[n], p, dims[n], N // dims[n], clamp=False, strict=True)
        Y = coo_sketch(idx, vals, dims, n, ell, seed, tensor_id, omega_round)
        Q, _ = np.linalg.qr(Y)
        P = select_rows(Q, method, eta, seed, (int(tensor_id) << 4) | n)
        A[n] = Q @ np.linalg.inv(Q[P, :])
        sel[n] = P
        pos = np.full(dims[n], -1, dtype=np.int64)
        pos[P] = np.arange(P.size)
        new[:, n] = pos[idx[:, n]]
        keep &= new[:, n] >= 0
    core = np.zeros([s_.size for s_ in sel])
    if keep.any():
        core[tuple(new[keep].T)] = vals[keep]
    return {"core": core, "factors": A, "selected": sel}


# ---------------------------------------------------------------------------------
# error measures and the bounds of Sec. 3.2 / Sec. 5.2
# ---------------------------------------------------------------------------------
def delta2(X, ranks):
    """Delta_j^2(X) = sum_{i > r_j} sigma_i^2(X_(j)) (Eq. delta)."""
    X = np.asarray(X, dtype=np.float64)
    out = []
    for n in range(X.ndim):
        s = np.linalg.svd(unfold(X, n), compute_uv=False)
        out.append(float(np.sum(s[int(ranks[n]):] ** 2)))
    return out


def randomized_bound(X, ranks, p):
    """Right side of Thm. rhosvd_err / Thm. rst_err: (sum_j (1 + r_j/(p-1)) Delta_j^2)^{1/2}."""
    d2 = delta2(X, ranks)
    return math.sqrt(sum((1.0 + ranks[n] / (p - 1.0)) * d2[n] for n in range(len(ranks))))


def sp_bound(X, ranks, p, rho=None):
    """Right side of Thm. pass_error for processing order rho (default 1..d)."""
    X = np.asarray(X, dtype=np.float64)
    d = X.ndim
    rho = list(range(d)) if rho is None else list(rho)
    d2 = delta2(X, ranks)
    total, gprod = 0.0, 1.0
    for n in rho:
        ell = ranks[n] + p
        I = X.shape[n]
        gprod *= math.sqrt(1.0 + 4.0 * ell * (I - ell))
        total += gprod * math.sqrt(1.0 + ranks[n] / (p - 1.0)) * math.sqrt(d2[n])
    return total
