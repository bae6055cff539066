"""Sparse path (Alg. 6, SP-STHOSVD, Sec. 5) through the C ABI against the oracle (needs a GB300).

Sketch: |Y_gpu - Y| <= c u (|X_(n)| |Omega|) with u = 2^-24 and c = 512 + 8 (FP32 products and
sums over at most 512 entries per work item, FP64 across items).  SP-STHOSVD: the selection is
checked on the invariants that define it (A_n(P_n, :) = I, max |A_ij| <= 2, core entries are entries
of X) and, where it equals the oracle's, factors (to 1e-5: the FP32 sketch moves Q by ~1e-7 relative)
and core (exactly) are compared directly; exact recovery of an exact-multilinear-rank tensor given as
COO.
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
from oracle.tensor import rel_error  # noqa: E402
from workloads import lowrank_plus_noise_np, zipf_coo  # noqa: E402


def coo_dev(idx, vals):
    return [torch.from_numpy(np.ascontiguousarray(idx[:, k]).astype(np.int32)).cuda() for k in range(idx.shape[1])], \
        torch.from_numpy(vals.astype(np.float32)).cuda()


def dense_of(idx, vals, dims):
    X = np.zeros(dims)
    X[tuple(idx.T)] = vals
    return X


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("ell", [7, 33])
def test_sketch_coo_matches_oracle(rh, mode, ell):
    dims = [60, 50, 40]
    idx, vals = zipf_coo(dims, 4000, 1.1, 3.0, seed=41)
    cols, v = coo_dev(idx, vals)
    Y = rh.rhosvd_sketch_coo(cols, v, dims, mode, ell, seed=5, tensor_id=1).cpu().numpy().T
    Yo = otk.coo_sketch(idx, vals.astype(np.float64), dims, mode, ell, 5, 1)
    # bound: sum over the row's entries of |v| |Omega(p, c)|
    rows = otk._kolda_rows(idx.astype(np.int64), dims, mode)
    om = np.abs(orng.omega(5, 1, mode, rows, ell).astype(np.float64))
    bound = np.zeros_like(Yo)
    np.add.at(bound, idx[:, mode].astype(np.int64), np.abs(vals.astype(np.float64))[:, None] * om)
    assert np.all(np.abs(Y - Yo) <= (512 + 8) * 2.0 ** -24 * bound + 1e-300), np.max(np.abs(Y - Yo))


def test_sketch_coo_deterministic(rh):
    dims = [300, 200, 50]
    idx, vals = zipf_coo(dims, 50000, 1.1, 3.0, seed=42)
    cols, v = coo_dev(idx, vals)
    a = rh.rhosvd_sketch_coo(cols, v, dims, 0, 40, seed=1)
    b = rh.rhosvd_sketch_coo(cols, v, dims, 0, 40, seed=1)
    assert torch.equal(a, b)


@pytest.mark.parametrize("dims,nnz,ranks,p", [([80, 70, 60], 6000, [5, 5, 5], 3),
                                              ([120, 40, 30, 20], 9000, [4, 4, 3, 3], 2)])
def test_sp_sthosvd_matches_oracle(rh, dims, nnz, ranks, p):
    idx, vals = zipf_coo(dims, nnz, 1.1, 3.0, seed=43)
    cols, v = coo_dev(idx, vals)
    T = rh.sp_sthosvd_coo(cols, v, dims, ranks, p=p, seed=7)
    torch.cuda.synchronize()
    out = otk.sp_sthosvd_coo(idx, vals.astype(np.float64), dims, ranks, p, 7)
    X = dense_of(idx, vals.astype(np.float64), dims)
    d = len(dims)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    sel = [s.cpu().numpy().astype(np.int64) for s in T.selected]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    for n in range(d):
        assert np.array_equal(A[n][sel[n], :], np.eye(len(sel[n])))
        assert np.abs(A[n]).max() <= 2.0 + 1e-8
    # core entries are entries of X at the selected coordinates
    Xs = X
    for n in range(d):
        Xs = np.take(Xs, sel[n], axis=n)
    assert np.array_equal(G, Xs)
    e_g = rel_error(X, G, A)
    e_o = rel_error(X, out["core"], out["factors"])
    same = all(np.array_equal(sel[n], out["selected"][n]) for n in range(d))
    if same:
        # the sketch sums FP32 products (relative perturbation of Y ~1e-7), which moves Q and A by the
        # same order; the core is identical (entries of X)
        for n in range(d):
            assert np.abs(A[n] - out["factors"][n]).max() <= 1e-5 * max(1.0, np.abs(out["factors"][n]).max())
        assert abs(e_g - e_o) <= 1e-6
    else:   # another valid selection: the error must be of the same size
        assert e_g <= 1.5 * e_o + 1e-12
    nx, ng = T.norms.cpu().numpy()
    assert abs(nx - np.sum(X ** 2)) <= 1e-12 * np.sum(X ** 2)
    assert abs(ng - np.sum(G ** 2)) <= 1e-12 * max(np.sum(G ** 2), 1e-300)


def test_sp_sthosvd_exact_recovery(rh):
    dims = [30, 25, 20]
    X = lowrank_plus_noise_np(dims, [3, 3, 3], 0.8, 0.0, seed=44).astype(np.float32)
    idx = np.argwhere(np.ones(dims, dtype=bool))
    vals = X[tuple(idx.T)]
    cols, v = coo_dev(idx, vals)
    T = rh.sp_sthosvd_coo(cols, v, dims, [3, 3, 3], p=2, seed=8)
    torch.cuda.synchronize()
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    assert rel_error(X.astype(np.float64), G, A) <= 1e-5


@pytest.mark.parametrize("bad", [30, -1])
def test_out_of_range_index_is_an_error(rh, bad):
    """An index outside [0, I_n) of the mode being counted is reported (RH_EINVAL) instead of being
    used as an address; the context stays usable."""
    dims = [30, 20, 10]
    idx, vals = zipf_coo(dims, 2000, 1.1, 3.0, seed=45)
    idx = idx.copy()
    idx[17, 0] = bad
    cols, v = coo_dev(idx, vals)
    with pytest.raises(rh.RhError, match="outside"):
        rh.rhosvd_sketch_coo(cols, v, dims, 0, 8, seed=1)
    with pytest.raises(rh.RhError, match="outside"):
        rh.sp_sthosvd_coo(cols, v, dims, [3, 3, 3], p=2, seed=1)
    idx[17, 0] = 0
    cols, v = coo_dev(idx, vals)
    Y = rh.rhosvd_sketch_coo(cols, v, dims, 0, 8, seed=1)
    torch.cuda.synchronize()
    assert torch.isfinite(Y).all()
