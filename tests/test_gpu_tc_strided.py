"""Tensor-core sketch and mode product of a mode with L > 1 (the unfolding's rows strided by L, read
through the 3-D view (l, i, r) of the tensor; FP32 values split on the fly into BF16 head + tail)
and R-HOSVD with every such mode on the tensor cores.  Needs a GB300.

Tolerances as for the first-mode kernels (tests/test_gpu_tc.py): the products of BF16 pieces are
exact, the sums FP32 inside a CTA and FP64 across CTAs, so |Y - Y_rep| <= (K + 8) 2^-24 (|X_rep|
|Omega|) with K the columns one CTA sums and X_rep = head + tail; the mode product |B - A_rep^T
X_rep| <= (I + 8) 2^-24 (|A_rep|^T |X_rep|) with A split into two pieces; R-HOSVD against the oracle
on the FP32 input with Omega rounded to BF16 on the tensor-core modes: 1e-5 on the error, 1e-3 on
the leading subspaces (tau = 0.05).
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
from workloads import lowrank_plus_noise_np  # noqa: E402


def _rep(X):
    """head + tail of the exact two-piece BF16 split of an FP32 array (ties to even)."""
    h = orng.round_bf16(X)
    t = orng.round_bf16((X - h).astype(np.float32))
    return h.astype(np.float64) + t.astype(np.float64)


@pytest.mark.parametrize("shape,mode", [((64, 200, 30), 1), ((16, 8, 300), 2), ((128, 1000, 3), 1),
                                        ((32, 32, 1000), 2), ((8, 8, 500, 3), 2), ((64, 7, 5, 9), 1)])
@pytest.mark.parametrize("ell", [1, 25, 64])
def test_strided_tc_sketch_matches_oracle(rh, shape, mode, ell):
    rs = np.random.default_rng(hash((shape, mode, ell)) % 2 ** 32)
    X = rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    seed, tid = 31, 4
    Y, nrm = rh.rhosvd_sketch_offset(Xd, list(shape), mode, ell, 0, seed=seed, tensor_id=tid, with_norm=True,
                                     form="f32_bf16x2")
    Y = Y.cpu().numpy().T
    Xrep = _rep(X)
    Xm = unfold(Xrep, mode)
    M = Xm.shape[1]
    Om = orng.round_bf16(orng.omega(seed, tid, mode, np.arange(M), ell)).astype(np.float64)
    Yr = Xm @ Om
    bound = np.abs(Xm) @ np.abs(Om)
    K = int(np.ceil(M / 64 / min(152, np.ceil(M / 64)))) * 64 + 64
    assert np.all(np.abs(Y - Yr) <= (K + 8) * 2.0 ** -24 * bound + 1e-300), np.max(np.abs(Y - Yr) / (bound + 1e-30))
    # ||X_rep||^2: FP32 sums of 32 squares per thread and tile, FP64 above
    ref = float(np.sum(Xrep ** 2))
    assert abs(float(nrm.item()) - ref) <= 40 * 2.0 ** -24 * ref


@pytest.mark.parametrize("shape,mode,k", [((128, 50, 30), 1, 60), ((16, 8, 300), 2, 25), ((256, 64, 9), 1, 64),
                                          ((32, 4, 40, 3), 2, 7), ((128, 1000, 3), 1, 1)])
def test_strided_tc_mode_product_matches_definition(rh, shape, mode, k):
    rs = np.random.default_rng(7)
    X = rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    I = shape[mode]
    A = rs.standard_normal((I, k))
    Y, out = rh.mode_product_split(Xd, list(shape), mode, torch.from_numpy(A.T.copy()).cuda())
    Yg = unfold(np.reshape(Y.cpu().numpy().astype(np.float64), out, order="F"), mode)
    Af = A.astype(np.float32)
    ah = orng.round_bf16(Af)
    at = orng.round_bf16((Af - ah).astype(np.float32))
    Arep = ah.astype(np.float64) + at.astype(np.float64)
    Xm = unfold(_rep(X), mode)
    Yr = Arep.T @ Xm
    bound = np.abs(Arep).T @ np.abs(Xm)
    assert np.all(np.abs(Yg - Yr) <= (I + 8) * 2.0 ** -24 * bound + 1e-300), np.max(np.abs(Yg - Yr))


@pytest.mark.parametrize("shape,ranks,p", [((128, 128, 64), (10, 9, 8), 6), ((64, 128, 96), (8, 8, 6), 4),
                                           ((32, 4, 128, 16), (6, 2, 6, 5), 2)])
def test_rhosvd_split_form_matches_oracle(rh, shape, ranks, p):
    d = len(shape)
    core = [min(max(ranks) + 2, n) for n in shape]
    X = lowrank_plus_noise_np(list(shape), core, 0.8, 1e-3, seed=71).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    T = rh.rhosvd(Xd, list(shape), list(ranks), p=p, seed=9, form="f32_bf16x2")
    torch.cuda.synchronize()
    info = T.info.cpu().numpy().tolist()
    assert not any(x & 16 for x in info), info
    tc_modes = [m for m in range(d) if info[m] & 4]
    assert 0 in tc_modes and len(tc_modes) >= 2, info
    Xe = X.astype(np.float64)
    out = otk.rhosvd(Xe, list(ranks), p, 9, omega_round={m: "bf16" for m in tc_modes}, record=True)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g, e_o = rel_error(Xe, G, A), rel_error(Xe, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    for rec in out["records"]:
        m = rec["mode"]
        sv = rec["sv_B"]
        kk = max(1, int(np.sum(sv >= 0.05 * sv[0])))
        U = out["factors"][m][:, :kk]
        Qa, _ = np.linalg.qr(A[m])
        assert np.linalg.norm(U - Qa @ (Qa.T @ U), 2) <= 1e-3, m
