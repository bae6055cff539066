"""Sparse-path variants through the C ABI against the oracle (needs a GB300): the BF16-Omega sketch
(Alg. 6 step 4 with every normal rounded to BF16), the table of distinct Omega rows, the row
selections of Sec. 5 in SP-STHOSVD, SP-HOSVD (Sec. 5, the modes of Alg. 6 taken independently) and
the orthonormalising post-processing of Sec. 5.

Tolerances: sketches |Y_gpu - Y| <= (512 + 8) 2^-24 (|X_(n)| |Omega|) (FP32 products and sums over at
most 512 entries, FP64 above), Omega being the rounded stream in the BF16 form on both sides;
structure-preserving results on their defining invariants (A_n(P_n, :) = I, core = entries of X)
and, when the selection equals the oracle's, factors to 1e-5 relative (the FP32 sketch moves Q by
~1e-7) and the core exactly; the post-processing leaves the approximation unchanged to 1e-12 and
matches the oracle's up to column signs.
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
from oracle.tensor import multi_ttm, rel_error  # noqa: E402
from workloads import zipf_coo  # noqa: E402


def coo_dev(idx, vals):
    return [torch.from_numpy(np.ascontiguousarray(idx[:, k]).astype(np.int32)).cuda() for k in range(idx.shape[1])], \
        torch.from_numpy(vals.astype(np.float32)).cuda()


def dense_of(idx, vals, dims):
    X = np.zeros(dims)
    X[tuple(idx.T)] = vals
    return X


def _sketch_bound(idx, vals, dims, mode, ell, seed, tid, bf16):
    rows = otk._kolda_rows(idx.astype(np.int64), dims, mode)
    om = orng.omega(seed, tid, mode, rows, ell)
    if bf16:
        om = orng.round_bf16(om)
    bound = np.zeros((dims[mode], ell))
    np.add.at(bound, idx[:, mode].astype(np.int64), np.abs(vals.astype(np.float64))[:, None] * np.abs(om.astype(np.float64)))
    return (512 + 8) * 2.0 ** -24 * bound


@pytest.mark.parametrize("omega", ["f32", "bf16"])
@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("ell", [5, 40, 64])
def test_sketch_coo_omega_forms_match_oracle(rh, omega, mode, ell):
    dims = [90, 70, 50]
    idx, vals = zipf_coo(dims, 20000, 1.1, 3.0, seed=51)
    cols, v = coo_dev(idx, vals)
    Y = rh.rhosvd_sketch_coo(cols, v, dims, mode, ell, seed=9, tensor_id=2, omega=omega).cpu().numpy().T
    Yo = otk.coo_sketch(idx, vals.astype(np.float64), dims, mode, ell, 9, 2,
                        omega_round="bf16" if omega == "bf16" else None)
    bound = _sketch_bound(idx, vals, dims, mode, ell, 9, 2, omega == "bf16")
    assert np.all(np.abs(Y - Yo) <= bound + 1e-300), np.max(np.abs(Y - Yo) - bound)


def test_sketch_coo_wide_unfolding_generates_rows(rh):
    """Mode 0 of 20 x 50000 x 50000 has 2.5e9 > 2^31 columns: every entry generates its Omega row
    (no table); modes 1 and 2 go through the table of distinct rows.  All three match the oracle."""
    dims = [20, 50000, 50000]
    idx, vals = zipf_coo(dims, 6000, 1.1, 3.0, seed=52)
    cols, v = coo_dev(idx, vals)
    for mode in range(3):
        for omega in ("f32", "bf16"):
            Y = rh.rhosvd_sketch_coo(cols, v, dims, mode, 12, seed=3, omega=omega).cpu().numpy().T
            Yo = otk.coo_sketch(idx, vals.astype(np.float64), dims, mode, 12, 3, 0,
                                omega_round="bf16" if omega == "bf16" else None)
            bound = _sketch_bound(idx, vals, dims, mode, 12, 3, 0, omega == "bf16")
            assert np.all(np.abs(Y - Yo) <= bound + 1e-300), (mode, omega)


def test_sketch_coo_bf16_deterministic_and_distinct_from_f32(rh):
    dims = [300, 200, 50]
    idx, vals = zipf_coo(dims, 50000, 1.1, 3.0, seed=53)
    cols, v = coo_dev(idx, vals)
    a = rh.rhosvd_sketch_coo(cols, v, dims, 0, 40, seed=1, omega="bf16")
    b = rh.rhosvd_sketch_coo(cols, v, dims, 0, 40, seed=1, omega="bf16")
    f = rh.rhosvd_sketch_coo(cols, v, dims, 0, 40, seed=1)
    assert torch.equal(a, b)
    assert not torch.equal(a, f)


def _check_sp(T, out, idx, vals, dims, hosvd=False):
    X = dense_of(idx, vals.astype(np.float64), dims)
    d = len(dims)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    sel = [s.cpu().numpy().astype(np.int64) for s in T.selected]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    for n in range(d):
        assert np.array_equal(np.sort(sel[n]), sel[n])
        assert np.array_equal(A[n][sel[n], :], np.eye(len(sel[n])))
    Xs = X
    for n in range(d):
        Xs = np.take(Xs, sel[n], axis=n)
    assert np.array_equal(G, Xs)          # the core is X at the selected coordinates
    e_g = rel_error(X, G, A)
    e_o = rel_error(X, out["core"], out["factors"])
    if all(np.array_equal(sel[n], out["selected"][n]) for n in range(d)):
        for n in range(d):
            assert np.abs(A[n] - out["factors"][n]).max() <= 1e-5 * max(1.0, np.abs(out["factors"][n]).max())
        assert np.array_equal(G, out["core"])
        # relative to the error: a poorly conditioned P^T Q (uniform sampling) amplifies both
        assert abs(e_g - e_o) <= 1e-5 * max(1.0, e_o)
        return True
    assert e_g <= 1.5 * e_o + 1e-12
    return False


@pytest.mark.parametrize("select", ["srrqr", "cpqr", "deim", "uniform", "leverage"])
def test_sp_sthosvd_selections_match_oracle(rh, select):
    # the sampling selections need a tensor without empty slices: a zero row of Q can be drawn
    # (uniform sampling ignores Q), and then P^T Q is singular on both sides
    dims, nnz = ([80, 70, 60], 6000) if select in ("srrqr", "cpqr", "deim") else ([40, 35, 30], 25000)
    idx, vals = zipf_coo(dims, nnz, 0.3, 3.0, seed=54) if nnz == 25000 else zipf_coo(dims, nnz, 1.1, 3.0, seed=54)
    cols, v = coo_dev(idx, vals)
    T = rh.sp_sthosvd_coo(cols, v, dims, [5, 5, 5], p=3, seed=7, tensor_id=1, select=select)
    torch.cuda.synchronize()
    out = otk.sp_sthosvd_coo(idx, vals.astype(np.float64), dims, [5, 5, 5], 3, 7, tensor_id=1, method=select)
    same = _check_sp(T, out, idx, vals, dims)
    if select == "srrqr":
        for f in T.factors:
            assert f.abs().max().item() <= 2.0 + 1e-8
    if select == "uniform":
        assert same            # the draws do not depend on Q


@pytest.mark.parametrize("omega", ["f32", "bf16"])
def test_sp_sthosvd_bf16_omega_matches_oracle(rh, omega):
    dims = [120, 40, 30, 20]
    idx, vals = zipf_coo(dims, 9000, 1.1, 3.0, seed=55)
    cols, v = coo_dev(idx, vals)
    T = rh.sp_sthosvd_coo(cols, v, dims, [4, 4, 3, 3], p=2, seed=11, omega=omega)
    torch.cuda.synchronize()
    out = otk.sp_sthosvd_coo(idx, vals.astype(np.float64), dims, [4, 4, 3, 3], 2, 11,
                             omega_round="bf16" if omega == "bf16" else None)
    _check_sp(T, out, idx, vals, dims)


@pytest.mark.parametrize("select", ["srrqr", "deim"])
@pytest.mark.parametrize("omega", ["f32", "bf16"])
def test_sp_hosvd_matches_oracle(rh, select, omega):
    dims = [80, 70, 60]
    idx, vals = zipf_coo(dims, 7000, 1.1, 3.0, seed=56)
    cols, v = coo_dev(idx, vals)
    T = rh.sp_hosvd_coo(cols, v, dims, [5, 4, 6], p=3, seed=13, select=select, omega=omega)
    torch.cuda.synchronize()
    out = otk.sp_hosvd_coo(idx, vals.astype(np.float64), dims, [5, 4, 6], 3, 13, method=select,
                           omega_round="bf16" if omega == "bf16" else None)
    _check_sp(T, out, idx, vals, dims, hosvd=True)
    X = dense_of(idx, vals.astype(np.float64), dims)
    nx, ng = T.norms.cpu().numpy()
    assert abs(nx - np.sum(X ** 2)) <= 1e-12 * np.sum(X ** 2)


def test_sp_hosvd_exact_recovery(rh):
    from workloads import lowrank_plus_noise_np

    dims = [30, 25, 20]
    X = lowrank_plus_noise_np(dims, [3, 3, 3], 0.8, 0.0, seed=57).astype(np.float32)
    idx = np.argwhere(np.ones(dims, dtype=bool))
    vals = X[tuple(idx.T)]
    cols, v = coo_dev(idx, vals)
    T = rh.sp_hosvd_coo(cols, v, dims, [3, 3, 3], p=2, seed=8)
    torch.cuda.synchronize()
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    assert rel_error(X.astype(np.float64), G, A) <= 1e-5


@pytest.mark.parametrize("variant", ["sthosvd", "hosvd"])
def test_orthonormalize_tucker_matches_oracle(rh, variant):
    """Sec. 5's post-processing on the interpolatory decomposition: the approximation is unchanged,
    the factors become orthonormal with the same ranges, ||G|| = ||X_hat||, and the result is the
    oracle's up to the column signs of the QR factors."""
    dims = [80, 70, 60]
    idx, vals = zipf_coo(dims, 6000, 1.1, 3.0, seed=58)
    cols, v = coo_dev(idx, vals)
    fn = rh.sp_sthosvd_coo if variant == "sthosvd" else rh.sp_hosvd_coo
    T = fn(cols, v, dims, [5, 5, 5], p=3, seed=7)
    torch.cuda.synchronize()
    A0 = [f.cpu().numpy().T.copy() for f in T.factors]
    G0 = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    Xh0 = multi_ttm(G0, A0)
    factors = [f.clone() for f in T.factors]
    core = T.core.clone()
    rh.orthonormalize_tucker(factors, core, dims)
    torch.cuda.synchronize()
    Q = [f.cpu().numpy().T.copy() for f in factors]
    G = np.reshape(core.cpu().numpy(), T.core_dims, order="F")
    Xh = multi_ttm(G, Q)
    assert np.linalg.norm(Xh - Xh0) <= 1e-12 * np.linalg.norm(Xh0)
    for q, a in zip(Q, A0):
        assert np.abs(q.T @ q - np.eye(q.shape[1])).max() <= 1e-13 * max(8, q.shape[1])
        assert np.linalg.norm(a - q @ (q.T @ a)) <= 1e-12 * np.linalg.norm(a)
    assert abs(np.linalg.norm(G) - np.linalg.norm(Xh0)) <= 1e-12 * np.linalg.norm(Xh0)
    Go, Qo = otk.orthonormalize_tucker(G0, A0)
    signs = [np.sign(np.sum(q * qo, axis=0)) for q, qo in zip(Q, Qo)]
    for q, qo, sg in zip(Q, Qo, signs):
        assert np.abs(q - qo * sg).max() <= 1e-12
    Gs = multi_ttm(Go, [np.diag(sg) for sg in signs])
    assert np.abs(G - Gs).max() <= 1e-12 * np.abs(Go).max()
