"""Randomized subspace iteration on the device (rh_options.power_iters; Sec. 5 "Variants", used with
one step for the Olivetti data in Sec. 6) against the oracle's ``randsvd(q=...)``.  Needs a GB300.

Each step forms B = Q^T G_(n) (the mode product), W = orth(B^T) (tall-skinny Householder R, then
W = B^T R^{-1} and one CholeskyQR pass: a QR of B^T, as the oracle's), Y = G_(n) W (a sketch against
the dense W) and Q = orth(Y).  Both sides' W are QR factors of B^T, so they differ by an upper
triangular factor and the QR of Y gives the same Q: the results are compared with the gates of the
plain algorithm (tests/test_gpu_parity.py): |err_gpu - err_oracle| <= 1e-12 (FP64) / 1e-5 (FP32)
and the leading subspaces to 1e-10 / 1e-4; the tensor-core form on the represented input (head +
tail) at 1e-5 and 1e-3 (tau = 0.05), as in tests/test_gpu_tc.py.
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


from oracle import tucker as otk  # noqa: E402
from oracle.tensor import rel_error  # noqa: E402
from workloads import hilbert, lowrank_plus_noise_np  # noqa: E402


def dev(X, dtype):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).ravel(order="F")).astype(dtype)).cuda()


def subspace_gap(A_ref, sv_ref, A, tau):
    k = int(np.sum(sv_ref >= tau * sv_ref[0]))
    k = max(1, min(k, A_ref.shape[1]))
    U = A_ref[:, :k]
    Qa, _ = np.linalg.qr(A)
    return np.linalg.norm(U - Qa @ (Qa.T @ U), 2)


def _compare(rh, X, ranks, p, seed, dtype, q, alg="rsthosvd", rho=None, **kw):
    Xd = dev(X, dtype)
    if alg == "rsthosvd":
        T = rh.rsthosvd(Xd, list(X.shape), ranks, p=p, seed=seed, rho=rho, power_iters=q, **kw)
    else:
        T = rh.rhosvd(Xd, list(X.shape), ranks, p=p, seed=seed, power_iters=q, **kw)
    torch.cuda.synchronize()
    Xe = X.astype(dtype).astype(np.float64)
    if alg == "rsthosvd":
        out = otk.rsthosvd(Xe, ranks, p, seed, rho=rho, record=True, q=q, clamp=kw.get("clamp", False))
    else:
        out = otk.rhosvd(Xe, ranks, p, seed, record=True, q=q, clamp=kw.get("clamp", False))
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g = rel_error(Xe, G, A)
    e_o = rel_error(Xe, out["core"], out["factors"])
    f64 = dtype == np.float64
    assert abs(e_g - e_o) <= (1e-12 if f64 else 1e-5), (e_g, e_o)
    for rec in out["records"]:
        n = rec["mode"]
        d = subspace_gap(out["factors"][n], rec["sv_B"], A[n], 1e-5 if f64 else 1e-2)
        assert d <= (1e-10 if f64 else 1e-4), (n, d)
        assert np.abs(A[n].T @ A[n] - np.eye(A[n].shape[1])).max() <= (1e-12 if f64 else 2e-5)
    assert not np.any(T.info.cpu().numpy() & 16)
    return T, e_g, e_o


# a slowly decaying spectrum with noise well above rounding: the regime where the power scheme pays
def _slow(shape, core, seed, noise=3e-2):
    return lowrank_plus_noise_np(list(shape), [core] * len(shape), 0.93, noise, seed=seed)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("q", [1, 2])
def test_power_rsthosvd_matches_oracle(rh, dtype, q):
    X = _slow([150, 70, 41], 24, seed=31)       # ragged tiles: 150 rows, 41 x 70 columns
    _compare(rh, X, [10, 8, 6], 5, 17, dtype, q)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_power_rsthosvd_4way_strided_modes(rh, dtype):
    """Modes processed out of order, so the mode products and W live in strided (L > 1) views."""
    X = _slow([23, 37, 18, 29], 9, seed=32)
    _compare(rh, X, [5, 6, 4, 5], 4, 9, dtype, 1, rho=[2, 0, 3, 1])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_power_rsthosvd_many_tiles(rh, dtype):
    X = _slow([300, 200, 130], 40, seed=33, noise=1e-2)
    _compare(rh, X, [20, 20, 20], 10, 1, dtype, 1)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_power_rhosvd_matches_oracle(rh, dtype):
    X = _slow([90, 64, 50], 20, seed=34)
    _compare(rh, X, [8, 7, 6], 5, 3, dtype, 1, alg="rhosvd")


def test_power_untruncated_matches_oracle(rh):
    X = _slow([70, 60, 50], 16, seed=35)
    Xd = dev(X, np.float64)
    T = rh.rsthosvd(Xd, [70, 60, 50], [6, 5, 4], p=3, seed=2, truncate=False, power_iters=1)
    torch.cuda.synchronize()
    out = otk.rsthosvd(X, [6, 5, 4], 3, 2, truncate=False, q=1)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    assert abs(rel_error(X, G, A) - rel_error(X, out["core"], out["factors"])) <= 1e-12


def test_power_lowers_the_error_of_a_slow_spectrum(rh):
    """The reason for the variant (Sec. 6): with a slowly decaying spectrum and noise, one step of
    subspace iteration brings the error closer to the deterministic STHOSVD's."""
    X = _slow([120, 100, 80], 40, seed=36, noise=1e-1)
    errs = []
    for q in (0, 1, 2):
        T = rh.rsthosvd(dev(X, np.float64), [120, 100, 80], [8, 8, 8], p=2, seed=4, power_iters=q)
        torch.cuda.synchronize()
        A = [f.cpu().numpy().T.copy() for f in T.factors]
        G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
        errs.append(rel_error(X, G, A))
    Gd, Ad = otk.sthosvd(X, [8, 8, 8])
    e_det = rel_error(X, Gd, Ad)
    assert errs[1] < errs[0] and errs[2] <= errs[1] * (1 + 1e-9), errs
    assert errs[2] - e_det < 0.5 * (errs[0] - e_det), (errs, e_det)


def test_power_hilbert_fp64(rh):
    """The 200^3 Hilbert configuration with one power step: trailing directions at the rounding floor
    (the W of B^T is rank deficient in FP64); the error still matches the oracle's to 1e-12."""
    X = hilbert([200, 200, 200], offset=1)
    T, e_g, e_o = _compare(rh, X, [20, 20, 20], 5, 0, np.float64, 1, rho=[0, 1, 2])
    assert e_g < 1e-12


@pytest.mark.parametrize("shape,ranks,p,rho", [((128, 64, 48), (10, 8, 6), 6, [0, 1, 2]),
                                               ((96, 40, 24, 16), (8, 6, 5, 4), 4, [0, 1, 2, 3])])
def test_power_f32_split_form_matches_oracle(rh, shape, ranks, p, rho):
    """RH_F32_BF16X2: the first mode's mode products on the tensor cores (X split into BF16 head and
    tail, Q into two pieces) and the power step's sketch on the CUDA cores over the same head + tail;
    the oracle sees the FP32 input with Omega rounded to BF16 on the tensor-core modes."""
    d = len(shape)
    X = _slow(list(shape), max(ranks) + 6, seed=37).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    T = rh.rsthosvd(Xd, list(shape), list(ranks), p=p, seed=5, rho=rho, form="f32_bf16x2", power_iters=1)
    torch.cuda.synchronize()
    info = T.info.cpu().numpy().tolist()
    assert info[0] & 4 and not any(x & 16 for x in info), info
    Xe = X.astype(np.float64)
    rnd = {m: "bf16" for m in range(d) if info[m] & 4}
    out = otk.rsthosvd(Xe, list(ranks), p, 5, rho=rho, omega_round=rnd, record=True, q=1)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g, e_o = rel_error(Xe, G, A), rel_error(Xe, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    for rec in out["records"]:
        m = rec["mode"]
        sv = rec["sv_B"]
        k = max(1, int(np.sum(sv >= 0.05 * sv[0])))
        U = out["factors"][m][:, :k]
        Qa, _ = np.linalg.qr(A[m])
        assert np.linalg.norm(U - Qa @ (Qa.T @ U), 2) <= 1e-3, m


def test_power_batched_equals_single_calls(rh):
    """The grouped engine records each tensor's program, subspace-iteration steps included, and
    must reproduce every single call bit for bit."""
    shapes = [[40, 30, 20], [25, 33, 17, 9], [64, 48, 36]]
    ranks = [[5, 4, 3], [4, 4, 3, 2], [8, 6, 5]]
    Xs = [dev(_slow(s, 6, seed=40 + i), np.float32) for i, s in enumerate(shapes)]
    Ts = rh.rsthosvd_batched(Xs, shapes, ranks, p=3, seed=7, power_iters=1)
    torch.cuda.synchronize()
    for i, (X, s, r) in enumerate(zip(Xs, shapes, ranks)):
        T1 = rh.rsthosvd(X, s, r, p=3, seed=7, tensor_id=i, power_iters=1)
        torch.cuda.synchronize()
        assert torch.equal(Ts[i].core, T1.core)
        for a, b in zip(Ts[i].factors, T1.factors):
            assert torch.equal(a, b)


def test_power_rejects_unsupported_requests(rh):
    from paper_1905_07311_gb300 import _lib

    X = dev(_slow([64, 32, 16], 6, seed=41), np.float32)
    with pytest.raises(_lib.RhError) as e:
        rh.rsthosvd(X, [64, 32, 16], [4, 4, 4], p=2, power_iters=9)
    assert e.value.code == 1
    Xb = rh.split_bf16x2(X)
    with pytest.raises(_lib.RhError) as e:
        rh.rsthosvd(Xb, [64, 32, 16], [4, 4, 4], p=2, form="bf16x2", power_iters=1)
    assert e.value.code == 6
