"""Tensor algebra of Sec. 2.1 -- oracle side (test infrastructure only).

Arrays are numpy ndarrays of shape (I_1, ..., I_d); index semantics only, the
memory order of the ndarray does not matter here.  The flat buffers the CUDA
library consumes are column-major (index 1 fastest), i.e. ``X.ravel(order='F')``.
"""

import numpy as np


def unfold(X, n):
    """Mode-n unfolding X_(n): I_n x prod_{k != n} I_k, columns are mode-n fibres.

    Column order: the remaining indices with the earliest mode varying fastest,
    which is the order Eq. kron (Sec. 2.1) implies for
    Y_(j) = A_j X_(j) (A_d (x) ... (x) A_{j+1} (x) A_{j-1} (x) ... (x) A_1)^T.
    """
    X = np.asarray(X)
    return np.reshape(np.moveaxis(X, n, 0), (X.shape[n], -1), order="F")


def fold(M, n, shape):
    """Inverse of ``unfold``: a matrix with rows indexed by mode n back to a tensor."""
    shape = tuple(int(s) for s in shape)
    rest = shape[:n] + shape[n + 1:]
    T = np.reshape(np.asarray(M), (shape[n],) + rest, order="F")
    return np.moveaxis(T, 0, n)


def ttm(X, A, n):
    """Mode-n product Y = X x_n A, defined by Y_(n) = A X_(n) (Sec. 2.1)."""
    A = np.asarray(A)
    shape = list(X.shape)
    shape[n] = A.shape[0]
    return fold(A @ unfold(X, n), n, shape)


def multi_ttm(X, mats, transpose=False, skip=None):
    """X x_1 M_1 x_2 M_2 ... x_d M_d (M_n^T when ``transpose``), modes in order 1..d."""
    Y = X
    for n, M in enumerate(mats):
        if skip is not None and n == skip:
            continue
        Y = ttm(Y, M.T if transpose else M, n)
    return Y


def tucker_full(core, factors):
    """X_hat = G x_1 A_1 ... x_d A_d (Tucker format, Sec. 2.1)."""
    return multi_ttm(np.asarray(core, dtype=np.float64), [np.asarray(A, dtype=np.float64) for A in factors])


def frob(X):
    return float(np.sqrt(np.sum(np.asarray(X, dtype=np.float64) ** 2)))


def rel_error(X, core, factors):
    """Direct ||X - X_hat||_F / ||X||_F, reconstructing X_hat in FP64 (no norm identity)."""
    X = np.asarray(X, dtype=np.float64)
    return frob(X - tucker_full(core, factors)) / frob(X)
