"""Pins for the oracle's tensor algebra (oracle.tensor) -- CPU only.

* unfolding and mode product against their entry-wise definitions (Sec. 2.1),
  written as explicit index loops on tiny tensors;
* the Kronecker form of a multi-mode product (Eq. kron), which fixes the column
  order of the unfolding;
* Lemma lem:proj (error decomposition for orthogonal projectors);
* the relative error of the zero approximation (1) and its invariance under scaling.
"""

import itertools

import numpy as np

from oracle.tensor import fold, frob, multi_ttm, rel_error, ttm, unfold


def _tiny(shape, seed=0):
    return np.random.default_rng(seed).standard_normal(shape)


def test_unfold_matches_fibre_definition():
    X = _tiny((3, 4, 2, 5))
    for n in range(4):
        M = unfold(X, n)
        others = [k for k in range(4) if k != n]
        assert M.shape == (X.shape[n], X.size // X.shape[n])
        for idx in itertools.product(*[range(s) for s in X.shape]):
            j, stride = 0, 1
            for k in others:                      # earlier modes vary fastest
                j += idx[k] * stride
                stride *= X.shape[k]
            assert M[idx[n], j] == X[idx]


def test_fold_inverts_unfold():
    X = _tiny((2, 3, 4))
    for n in range(3):
        assert np.array_equal(fold(unfold(X, n), n, X.shape), X)


def test_ttm_matches_entrywise_sum():
    X = _tiny((3, 4, 5), 1)
    A = _tiny((2, 4), 2)
    Y = ttm(X, A, 1)
    assert Y.shape == (3, 2, 5)
    for i, k, l in itertools.product(range(3), range(2), range(5)):
        s = sum(X[i, j, l] * A[k, j] for j in range(4))
        assert abs(Y[i, k, l] - s) < 1e-12


def test_kronecker_form_of_multi_mode_product():
    X = _tiny((3, 4, 2), 3)
    A = [_tiny((2, 3), 4), _tiny((5, 4), 5), _tiny((3, 2), 6)]
    Y = multi_ttm(X, A)
    for j in range(3):
        rest = [A[k] for k in reversed(range(3)) if k != j]     # A_d (x) ... (x) A_1 without A_j
        K = rest[0]
        for M in rest[1:]:
            K = np.kron(K, M)
        assert np.allclose(unfold(Y, j), A[j] @ unfold(X, j) @ K.T, atol=1e-12)


def test_projector_lemma():
    rs = np.random.default_rng(7)
    X = rs.standard_normal((5, 6, 4))
    P = []
    for n, r in zip(range(3), (2, 3, 2)):
        Q, _ = np.linalg.qr(rs.standard_normal((X.shape[n], r)))
        P.append(Q @ Q.T)
    lhs = frob(X - multi_ttm(X, P)) ** 2
    terms = []
    for j in range(3):
        T = X
        for i in range(j):
            T = ttm(T, P[i], i)
        T = ttm(T, np.eye(X.shape[j]) - P[j], j)
        terms.append(frob(T) ** 2)
    rhs = sum(frob(X - ttm(X, P[j], j)) ** 2 for j in range(3))
    assert abs(lhs - sum(terms)) < 1e-10 * lhs
    assert lhs <= rhs + 1e-12


def test_rel_error_of_the_zero_and_of_a_scaled_approximation():
    # ||X - 0|| / ||X|| = 1 for any X, and the relative error does not change when X and the
    # approximation are scaled together (||X|| = 2.5 here, so a norm of the wrong power shows)
    rs = np.random.default_rng(9)
    X = rs.standard_normal((4, 3, 5))
    X *= 2.5 / frob(X)
    A = [np.linalg.qr(rs.standard_normal((n, 2)))[0] for n in X.shape]
    assert abs(rel_error(X, np.zeros((2, 2, 2)), A) - 1.0) < 1e-15
    G = multi_ttm(X, A, transpose=True)
    e = rel_error(X, G, A)
    assert 0.0 < e < 1.0
    assert abs(rel_error(3.0 * X, 3.0 * G, A) - e) < 1e-14
    assert abs(e - frob(X - multi_ttm(G, A)) / 2.5) < 1e-14
