"""The host step of SP-STHOSVD (Alg. 6 steps 6-7: row selection and the interpolatory factor
A = Q (P^T Q)^{-1}) through the C ABI, on CPU, for the selections the library offers (strong RRQR,
the one Alg. 6 uses; column-pivoted QR, DEIM, uniform and leverage-score sampling, Sec. 5's
alternatives, the sampling ones with one Philox4x32-10 implementation on each side): the library runs them
on the host, so they are compared with the oracle here on identical inputs.  The selection is index
work and must equal the oracle's exactly; A follows from it and is checked against its definition.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
scipy_linalg = pytest.importorskip("scipy.linalg")

from oracle import tucker as otk  # noqa: E402


@pytest.fixture(scope="module")
def rh():
    from paper_1905_07311_gb300 import build

    build.build()
    import paper_1905_07311_gb300 as rh

    return rh


def _basis(I, ell, seed, row_scale=None):
    g = np.random.default_rng(seed).standard_normal((I, ell))
    if row_scale is not None:
        g *= row_scale[:, None]
    return np.linalg.qr(g)[0]


SEED, STREAM = 0x1234ABCD5678, 3


def _select(rh, Q, eta, method="srrqr"):
    sel, A = rh.subset_select(torch.from_numpy(np.ascontiguousarray(Q)), method, eta, seed=SEED, stream=STREAM)
    return sel.numpy().astype(np.int64), A.numpy().T


ORACLE = {"srrqr": lambda Q, eta: otk.srrqr_select(Q, eta=eta), "cpqr": lambda Q, eta: otk.cpqr_select(Q),
          "deim": lambda Q, eta: otk.deim_select(Q),
          "uniform": lambda Q, eta: otk.sample_select(Q, False, SEED, STREAM),
          "leverage": lambda Q, eta: otk.sample_select(Q, True, SEED, STREAM)}


def _check_valid(Q, sel, A, eta):
    I, ell = Q.shape
    assert np.all(np.diff(sel) > 0) and sel[0] >= 0 and sel[-1] < I
    assert np.array_equal(A[sel, :], np.eye(ell))                   # stored exactly
    rest = np.setdiff1d(np.arange(I), sel)
    if rest.size and eta is not None:
        assert np.abs(A[rest, :]).max() <= eta * (1 + 1e-12)
    ref = np.linalg.solve(Q[sel, :].T, Q.T).T                       # Q (P^T Q)^{-1}, another route
    cond = np.linalg.cond(Q[sel, :])
    assert np.abs(A - ref).max() <= 1e-13 * cond * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("I,ell,seed", [(50, 5, 1), (200, 20, 2), (64, 63, 3), (300, 40, 4), (1000, 64, 5),
                                        (9, 1, 6)])
@pytest.mark.parametrize("method,eta", [("srrqr", 2.0), ("srrqr", 1.0), ("cpqr", None), ("deim", None),
                                        ("uniform", None), ("leverage", None)])
def test_selection_equals_the_oracle(rh, I, ell, seed, method, eta):
    Q = _basis(I, ell, seed)
    sel, A = _select(rh, Q, 2.0 if eta is None else eta, method)
    assert np.array_equal(sel, ORACLE[method](Q, eta))
    _check_valid(Q, sel, A, eta)


def test_swaps_run(rh):
    """With eta = 1 the column-pivoted start is not always strong: the swap phase must move rows
    (a graded basis makes large |A_ij| likely) and still match the oracle."""
    moved = 0
    for seed in range(6):
        I, ell = 120, 12
        Q = _basis(I, ell, 100 + seed, row_scale=np.geomspace(1.0, 1e-3, I)[np.random.default_rng(seed).permutation(I)])
        sel, A = _select(rh, Q, 1.0)
        assert np.array_equal(sel, otk.srrqr_select(Q, eta=1.0))
        _check_valid(Q, sel, A, 1.0)
        start = np.sort(scipy_linalg.qr(Q.T, pivoting=True, mode="economic")[2][:ell])
        moved += int(not np.array_equal(start, sel))
    assert moved > 0


@pytest.mark.parametrize("method", ["srrqr", "cpqr", "deim"])
def test_closed_forms(rh, method):
    # ell = I: every row, A = I
    Q = _basis(7, 7, 8)
    sel, A = _select(rh, Q, 2.0, method)
    assert np.array_equal(sel, np.arange(7)) and np.array_equal(A, np.eye(7))
    # a basis supported on rows {3, 10, 17}: those rows are chosen and A is Q (P^T Q)^{-1} = E_P
    I, rows = 20, [3, 10, 17]
    Q = np.zeros((I, 3))
    R = np.linalg.qr(np.random.default_rng(9).standard_normal((3, 3)))[0]
    Q[rows, :] = R
    sel, A = _select(rh, Q, 2.0, method)
    assert list(sel) == rows
    E = np.zeros((I, 3))
    E[rows, :] = np.eye(3)
    assert np.array_equal(A, E)


def test_failures_are_reported(rh):
    Q = _basis(30, 4, 10)
    Q[:, 2] = 0.0                                   # rank-deficient: P^T Q is singular
    for method in ("srrqr", "cpqr"):
        with pytest.raises(rh.RhError, match="singular"):
            rh.subset_select(torch.from_numpy(Q), method)
    with pytest.raises(rh.RhError, match="rank deficient"):
        rh.subset_select(torch.from_numpy(Q), "deim")
    Q = np.full((30, 4), np.nan)
    for method in ("srrqr", "cpqr", "deim"):
        with pytest.raises(rh.RhError, match="non-finite|rank deficient"):
            rh.subset_select(torch.from_numpy(Q), method)
    with pytest.raises(rh.RhError, match="eta"):
        rh.subset_select(torch.from_numpy(_basis(30, 4, 11)), "srrqr", 0.5)
    sel, _ = rh.subset_select(torch.from_numpy(_basis(30, 4, 11)), "deim", 0.5)   # eta unused
    assert sel.numel() == 4
    with pytest.raises(rh.RhError, match="ell <= I"):
        rh.subset_select(torch.from_numpy(_basis(30, 4, 12).T.copy()))
    with pytest.raises(ValueError):
        rh.subset_select(torch.zeros((4, 2), dtype=torch.float32))
    with pytest.raises(ValueError):
        rh.subset_select(torch.from_numpy(_basis(30, 4, 12)), "volume")
    from paper_1905_07311_gb300 import _lib
    import ctypes
    one = ctypes.c_void_p(1)
    assert _lib.lib().rh_subset_select(30, 4, one, 5, 2.0, 0, 0, one, one) == 1       # unknown method


@pytest.mark.parametrize("method", ["uniform", "leverage"])
def test_sampling_depends_on_seed_and_stream(rh, method):
    Q = _basis(200, 10, 13)
    t = torch.from_numpy(Q)
    a, _ = rh.subset_select(t, method, seed=1, stream=0)
    b, _ = rh.subset_select(t, method, seed=1, stream=0)
    c, _ = rh.subset_select(t, method, seed=2, stream=0)
    d, _ = rh.subset_select(t, method, seed=1, stream=1)
    assert torch.equal(a, b) and not torch.equal(a, c) and not torch.equal(a, d)
    for s_, st in [(1, 0), (2, 0), (1, 1), (99, 7)]:
        sel, _ = rh.subset_select(t, method, seed=s_, stream=st)
        assert np.array_equal(sel.numpy(), otk.sample_select(Q, method == "leverage", s_, st))
