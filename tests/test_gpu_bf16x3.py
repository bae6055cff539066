"""RH_F32_BF16X3: an FP32 tensor split exactly into three BF16 pieces inside the tensor-core kernels
(needs a GB300).

h = bf16(x), m = bf16(x - h), t = bf16(x - h - m) add up to x exactly (24 significant bits), so the
tensor cores see the FP32 values themselves: the sketch of mode 0 obeys the FP32-accumulation bound
|Y - X Omega_bf16| <= (K + 8) 2^-24 (|X| |Omega_bf16|) with X the FP32 tensor (the two-piece form
meets it only for X's 16-bit head + tail), the mode product the bound with the FP32 X and A split
into two pieces, ||X||^2 is the FP32 values' (FP32 sums of 32 squares per thread and tile, FP64
across), and R-STHOSVD matches the oracle run on the FP32 tensor with Omega rounded to BF16 on the
modes that ran on the tensor cores (info bit 4), with the two-piece form's gates.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import rng as orng  # noqa: E402
from oracle.tensor import unfold  # noqa: E402


@pytest.fixture(scope="module")
def rh():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1905_07311_gb300 import build

    build.build()
    import paper_1905_07311_gb300 as rh

    return rh


def _wide_f32(rs, shape):
    """Normal values with magnitudes spread over 2^-29 .. 2^29 (every bit of the significand matters)."""
    return (rs.standard_normal(shape) * np.exp(rs.uniform(-20, 20, shape))).astype(np.float32)


def _flat(X):
    return torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()


@pytest.mark.parametrize("shape", [(128, 300, 7), (200, 40, 40), (1024, 64, 33), (136, 77, 3)])
@pytest.mark.parametrize("ell", [1, 25, 64])
def test_x3_sketch_is_exact_in_x(rh, shape, ell):
    rs = np.random.default_rng(hash((shape, ell, 3)) % 2 ** 32)
    X = _wide_f32(rs, shape)
    Xd = _flat(X)
    seed, tid = 71, 4
    Y, n2 = rh.rhosvd_sketch_bf16(Xd, list(shape), ell, seed=seed, tensor_id=tid, pieces="f32x3", with_norm=True)
    Y = Y.cpu().numpy().T
    Xm = unfold(X.astype(np.float64), 0)
    M = Xm.shape[1]
    Om = orng.round_bf16(orng.omega(seed, tid, 0, np.arange(M), ell)).astype(np.float64)
    bound = np.abs(Xm) @ np.abs(Om)
    K = int(np.ceil(M / 64 / min(152, np.ceil(M / 64)))) * 64 + 64
    err = np.abs(Y - Xm @ Om)
    assert np.all(err <= (K + 8) * 2.0 ** -24 * bound + 1e-300), np.max(err / (bound + 1e-30))
    # the two-piece form reads head + tail (16 significant bits): on these magnitudes it misses the
    # FP32 bound that the three pieces meet
    Y2 = rh.rhosvd_sketch_bf16(Xd, list(shape), ell, seed=seed, tensor_id=tid, pieces="f32").cpu().numpy().T
    err2 = np.abs(Y2 - Xm @ Om)
    assert np.max(err2 / (bound + 1e-300)) > np.max(err / (bound + 1e-300))
    s2 = float(np.sum(X.astype(np.float64) ** 2))
    assert abs(n2.item() - s2) <= 40 * 2.0 ** -24 * s2


@pytest.mark.parametrize("shape,k", [((128, 300), 60), ((64, 129), 1), ((200, 7, 9), 25), ((1024, 300), 64)])
def test_x3_mode_product_is_exact_in_x(rh, shape, k):
    rs = np.random.default_rng(6)
    X = _wide_f32(rs, shape)
    Xd = _flat(X)
    Xm = unfold(X.astype(np.float64), 0)
    A = rs.standard_normal((shape[0], k))
    Af = A.astype(np.float32)
    ah = orng.round_bf16(Af)
    at = orng.round_bf16((Af - ah).astype(np.float32))
    Arep = ah.astype(np.float64) + at.astype(np.float64)
    Y = rh.mode_product_bf16(Xd, list(shape), torch.from_numpy(A.T.copy()).cuda(), pieces="f32x3").cpu().numpy()
    Yg = np.reshape(Y, (k, -1), order="F")
    Yr = Arep.T @ Xm
    bound = np.abs(Arep).T @ np.abs(Xm)
    assert np.all(np.abs(Yg - Yr) <= (shape[0] + 8) * 2.0 ** -24 * bound + 1e-300), np.max(np.abs(Yg - Yr) / bound)


@pytest.mark.parametrize("shape,ranks,p,rho", [((128, 60, 50), (6, 5, 4), 5, [0, 1, 2]),
                                               ((256, 128, 96), (20, 20, 20), 10, [0, 1, 2]),
                                               ((256, 72, 50), (20, 12, 10), 8, [0, 1, 2]),
                                               ((136, 40, 24, 36), (12, 8, 8, 8), 4, [0, 1, 2, 3]),
                                               # a first mode the tensor-core kernels do not take: FP32 on
                                               # the CUDA cores (no small-row route for three pieces)
                                               ((90, 64, 40), (6, 5, 4), 5, [0, 1, 2])])
def test_rsthosvd_x3_matches_oracle(rh, shape, ranks, p, rho):
    from oracle import tucker as otk
    from oracle.tensor import rel_error
    from workloads import lowrank_plus_noise_np

    d = len(shape)
    X = lowrank_plus_noise_np(list(shape), [max(ranks) + 2] * d, 0.8, 1e-3, seed=24).astype(np.float32)
    T = rh.rsthosvd(_flat(X), list(shape), list(ranks), p=p, seed=6, rho=rho, form="f32_bf16x3", clamp=True)
    torch.cuda.synchronize()
    info = T.info.cpu().numpy().tolist()
    assert not any(x & 16 for x in info), info   # no tensor-core wait gave up
    if shape[0] % 8 == 0:
        assert info[0] & 4, info
    else:
        assert not info[0] & 4, info
    Xe = X.astype(np.float64)
    rnd = {m: "bf16" for m in range(d) if info[m] & 4}
    out = otk.rsthosvd(Xe, list(ranks), p, 6, rho=rho, omega_round=rnd, record=True, clamp=True)
    A = [f.cpu().numpy().T for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g = rel_error(Xe, G, A)
    e_o = rel_error(Xe, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    for rec in out["records"]:
        m = rec["mode"]
        sv = rec["sv_B"]
        k = max(1, int(np.sum(sv >= 0.05 * sv[0])))
        U = out["factors"][m][:, :k]
        Qa, _ = np.linalg.qr(A[m])
        assert np.linalg.norm(U - Qa @ (Qa.T @ U), 2) <= 1e-3, m
    s2 = float(np.sum(Xe ** 2))
    assert abs(T.norms[0].item() - s2) <= 40 * 2.0 ** -24 * s2


def test_x3_is_rejected_where_unsupported(rh):
    X = torch.zeros(64 * 48 * 40, dtype=torch.float32, device="cuda")
    with pytest.raises(Exception):
        rh.rsthosvd(X, [64, 48, 40], [4, 4, 4], p=4, form="f32_bf16x3", power_iters=1)
