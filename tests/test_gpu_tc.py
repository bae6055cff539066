"""Tensor-core (tcgen05) paths through the C ABI against the oracle (needs a GB300).

BF16 forms: X is held as BF16 pieces (one piece: a BF16 tensor; two pieces: head + tail of an
FP32 tensor) and Omega is the library stream rounded to BF16 (ties to even), so every product is
exact and only the FP32 accumulation rounds: |Y_gpu - Y| <= (K + 8) 2^-24 (|X_rep| |Omega_bf16|)
with K the number of columns one CTA accumulates (at most ceil(M / 64 / CTAs) * 64), summed over
CTAs in FP64.
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


def bf16_bits_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def test_split_bf16x2_matches_definition(rh):
    rs = np.random.default_rng(0)
    x = (rs.standard_normal(4096) * np.exp(rs.uniform(-20, 20, 4096))).astype(np.float32)
    out = rh.split_bf16x2(torch.from_numpy(x).cuda()).cpu().numpy().view(np.uint16)
    h = orng.round_bf16(x)
    t = orng.round_bf16((x - h).astype(np.float32))
    assert np.array_equal(out[:4096], (h.view(np.uint32) >> 16).astype(np.uint16))
    assert np.array_equal(out[4096:], (t.view(np.uint32) >> 16).astype(np.uint16))
    rep = bf16_bits_to_f64(out[:4096]) + bf16_bits_to_f64(out[4096:])
    assert np.all(np.abs(rep - x) <= 2.0 ** -16 * np.abs(x))


@pytest.mark.parametrize("pieces", [1, 2])
@pytest.mark.parametrize("shape", [(128, 300, 7), (200, 40, 40), (1024, 64, 33), (96, 1000), (8, 5000)])
@pytest.mark.parametrize("ell", [1, 25, 64])
def test_tc_sketch_matches_oracle(rh, pieces, shape, ell):
    rs = np.random.default_rng(hash((shape, ell, pieces)) % 2 ** 32)
    X = rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    if pieces == 2:
        Xb = rh.split_bf16x2(Xd)
        bits = Xb.cpu().numpy().view(np.uint16)
        n = X.size
        rep = bf16_bits_to_f64(bits[:n]) + bf16_bits_to_f64(bits[n:])
    else:
        bits = (orng.round_bf16(X.ravel(order="F")).view(np.uint32) >> 16).astype(np.uint16)
        Xb = torch.from_numpy(bits.view(np.int16).copy()).cuda()
        rep = bf16_bits_to_f64(bits)
    Xrep = np.reshape(rep, shape, order="F")
    seed, tid = 77, 2
    Y = rh.rhosvd_sketch_bf16(Xb, list(shape), ell, seed=seed, tensor_id=tid, pieces=pieces).cpu().numpy().T
    Xm = unfold(Xrep, 0)
    M = Xm.shape[1]
    Om = orng.round_bf16(orng.omega(seed, tid, 0, np.arange(M), ell)).astype(np.float64)
    Yr = Xm @ Om
    bound = np.abs(Xm) @ np.abs(Om)
    K = int(np.ceil(M / 64 / min(152, np.ceil(M / 64)))) * 64 + 64
    assert np.all(np.abs(Y - Yr) <= (K + 8) * 2.0 ** -24 * bound + 1e-300), np.max(np.abs(Y - Yr) / (bound + 1e-30))


@pytest.mark.parametrize("pieces", [1, 2])
@pytest.mark.parametrize("shape,k", [((128, 300), 60), ((64, 129), 1), ((200, 7, 9), 25), ((1024, 300), 64)])
def test_tc_mode_product_matches_definition(rh, pieces, shape, k):
    """Y = A^T X_(1) with A split into two BF16 pieces: |Y - Y_rep| <= (I + 8) 2^-24 (|A_rep|^T |X_rep|)."""
    rs = np.random.default_rng(5)
    X = rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    if pieces == 2:
        Xb = rh.split_bf16x2(Xd)
        bits = Xb.cpu().numpy().view(np.uint16)
        rep = bf16_bits_to_f64(bits[:X.size]) + bf16_bits_to_f64(bits[X.size:])
    else:
        bits = (orng.round_bf16(X.ravel(order="F")).view(np.uint32) >> 16).astype(np.uint16)
        Xb = torch.from_numpy(bits.view(np.int16).copy()).cuda()
        rep = bf16_bits_to_f64(bits)
    Xm = unfold(np.reshape(rep, shape, order="F"), 0)
    A = rs.standard_normal((shape[0], k))
    Af = A.astype(np.float32)
    ah = orng.round_bf16(Af)
    at = orng.round_bf16((Af - ah).astype(np.float32))
    Arep = ah.astype(np.float64) + at.astype(np.float64)
    Y = rh.mode_product_bf16(Xb, list(shape), torch.from_numpy(A.T.copy()).cuda(), pieces=pieces).cpu().numpy()
    Yg = np.reshape(Y, (k, -1), order="F")
    Yr = Arep.T @ Xm
    bound = np.abs(Arep).T @ np.abs(Xm)
    assert np.all(np.abs(Yg - Yr) <= (shape[0] + 8) * 2.0 ** -24 * bound + 1e-300), np.max(np.abs(Yg - Yr))


# ---------------------------------------------------------------------------------
# R-STHOSVD on the tensor cores (BF16X2 form)
# ---------------------------------------------------------------------------------
# Gates: the GPU sees X_rep = head + tail exactly and rounds Omega_n to BF16 on every mode that ran
# on the tensor cores (info bit 4; the oracle rounds the same modes); a mode product on the tensor
# cores uses Q split into two BF16 pieces (|dQ| <= 2^-16 |Q|) and, after the first mode, the FP32
# core split into 16 significant bits: perturbations of B of ~2^-16 relative.  They move the
# leading-k factor subspace by ~2^-16 / tau (tau = 0.05 -> 3e-4, gate 1e-3) and the relative Tucker
# error only at second order (the residual is orthogonal to the perturbation of the projection), so
# the error gate stays 1e-5.
@pytest.mark.parametrize("shape,ranks,p,rho", [((128, 60, 50), (6, 5, 4), 5, [0, 1, 2]),
                                               ((256, 128, 96), (20, 20, 20), 10, [0, 1, 2]),
                                               ((1024, 40, 30), (8, 6, 5), 4, [0, 1, 2]),
                                               ((256, 96, 48), (12, 10, 8), 6, [0, 2, 1]),
                                               ((64, 48, 40, 16), (6, 5, 4, 3), 3, [0, 1, 2, 3]),
                                               ((64, 40, 24, 16), (6, 5, 4, 3), 3, [0, 1, 3, 2]),
                                               # ell % 4 == 0: truncated cores on the tensor cores, written
                                               # with the next mode fastest (Lp = 72) and in the usual
                                               # order (Lp = 20 < 32), ragged last tiles
                                               ((256, 72, 50), (20, 12, 10), 8, [0, 1, 2]),
                                               ((136, 40, 24, 36), (12, 8, 8, 8), 4, [0, 1, 2, 3])])
def test_rsthosvd_bf16x2_matches_oracle(rh, shape, ranks, p, rho):
    from oracle import tucker as otk
    from oracle.tensor import rel_error
    from workloads import lowrank_plus_noise_np

    d = len(shape)
    X = lowrank_plus_noise_np(list(shape), [max(ranks) + 2] * d, 0.8, 1e-3, seed=21).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    Xb = rh.split_bf16x2(Xd)
    T = rh.rsthosvd(Xb, list(shape), list(ranks), p=p, seed=3, rho=rho, form="bf16x2")
    torch.cuda.synchronize()
    info = T.info.cpu().numpy().tolist()
    assert info[0] & 4, info          # the first mode always runs on the tensor cores
    assert not any(x & 16 for x in info), info   # no tensor-core wait gave up
    if shape == (256, 128, 96):
        assert info[1] & 4, info      # mode 2 follows with a unit-stride core (I_2 = 128)
    bits = Xb.cpu().numpy().view(np.uint16)
    n = X.size
    Xrep = np.reshape(bf16_bits_to_f64(bits[:n]) + bf16_bits_to_f64(bits[n:]), shape, order="F")
    rnd = {m: "bf16" for m in range(d) if info[m] & 4}
    out = otk.rsthosvd(Xrep, list(ranks), p, 3, rho=rho, omega_round=rnd, record=True)
    A = [f.cpu().numpy().T for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g = rel_error(Xrep, G, A)
    e_o = rel_error(Xrep, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    for rec in out["records"]:
        m = rec["mode"]
        sv = rec["sv_B"]
        k = max(1, int(np.sum(sv >= 0.05 * sv[0])))
        U = out["factors"][m][:, :k]
        Qa, _ = np.linalg.qr(A[m])
        assert np.linalg.norm(U - Qa @ (Qa.T @ U), 2) <= 1e-3, m
    nx = float(T.norms.cpu().numpy()[0])
    # the persistent kernel's separate FP64 pass, or on the small-row kernel (mode 0 first,
    # I_0 <= 128, r + p <= 32) FP32 sums of at most 32 squares per thread and tile, FP64 above
    small = rho[0] == 0 and shape[0] <= 128 and ranks[0] + p <= 32
    assert abs(nx - np.sum(Xrep ** 2)) <= (40 * 2.0 ** -24 if small else 1e-10) * np.sum(Xrep ** 2)


# ---------------------------------------------------------------------------------
# RH_F32_BF16X2: an FP32 tensor split into head / tail inside the tensor-core kernels.  The pieces
# and the order of every product and sum are those of the two-piece form, so the outputs must be
# bit-identical to running the two-piece form on split_bf16x2(X).
# ---------------------------------------------------------------------------------
def _wide_f32(rs, shape):
    """Normal values with magnitudes spread over 2^-29 .. 2^29 (exercises the head / tail split)."""
    return (rs.standard_normal(shape) * np.exp(rs.uniform(-20, 20, shape))).astype(np.float32)


@pytest.mark.parametrize("shape", [(128, 300, 7), (200, 40, 40), (1024, 64, 33), (96, 1000), (8, 5000),
                                   (136, 77, 3)])
@pytest.mark.parametrize("ell", [1, 25, 64])
def test_f32_split_sketch_is_bit_identical_to_pieces(rh, shape, ell):
    rs = np.random.default_rng(hash((shape, ell, "f32")) % 2 ** 32)
    X = _wide_f32(rs, shape) if ell == 25 else rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    Xb = rh.split_bf16x2(Xd)
    Yp = rh.rhosvd_sketch_bf16(Xb, list(shape), ell, seed=9, tensor_id=4, pieces=2)
    Yf, nrm = rh.rhosvd_sketch_bf16(Xd, list(shape), ell, seed=9, tensor_id=4, pieces="f32", with_norm=True)
    assert torch.equal(Yp, Yf)
    bits = Xb.cpu().numpy().view(np.uint16)
    rep = bf16_bits_to_f64(bits[:X.size]) + bf16_bits_to_f64(bits[X.size:])
    ref = float(np.sum(rep ** 2))
    # FP32 sums of 32 squares per thread and tile (positive terms), FP64 above
    assert abs(float(nrm.item()) - ref) <= 66 * 2.0 ** -24 * ref


@pytest.mark.parametrize("shape,k", [((128, 300), 60), ((64, 129), 1), ((200, 7, 9), 25), ((1024, 300), 64),
                                     ((136, 77, 3), 17)])
def test_f32_split_mode_product_is_bit_identical_to_pieces(rh, shape, k):
    rs = np.random.default_rng(6)
    X = _wide_f32(rs, shape) if k == 25 else rs.standard_normal(shape).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    A = torch.from_numpy(rs.standard_normal((k, shape[0]))).cuda()
    Yp = rh.mode_product_bf16(rh.split_bf16x2(Xd), list(shape), A, pieces=2)
    Yf = rh.mode_product_bf16(Xd, list(shape), A, pieces="f32")
    assert torch.equal(Yp, Yf)


@pytest.mark.parametrize("shape,ranks,p", [((128, 60, 50), (6, 5, 4), 5), ((136, 45, 31), (5, 5, 5), 4),
                                           ((1024, 40, 30), (8, 6, 5), 4)])
def test_rsthosvd_f32_split_is_bit_identical_to_pieces(rh, shape, ranks, p):
    from workloads import lowrank_plus_noise_np

    X = lowrank_plus_noise_np(list(shape), [max(ranks) + 2] * 3, 0.8, 1e-3, seed=22).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    Tp = rh.rsthosvd(rh.split_bf16x2(Xd), list(shape), list(ranks), p=p, seed=3, rho=[0, 1, 2], form="bf16x2")
    Tp = [t.clone() for t in Tp.factors] + [Tp.core.clone(), Tp.norms.clone()]
    Tf = rh.rsthosvd(Xd, list(shape), list(ranks), p=p, seed=3, rho=[0, 1, 2], form="f32_bf16x2")
    for a, b in zip(Tp[:3], Tf.factors):
        assert torch.equal(a, b)
    assert torch.equal(Tp[3], Tf.core)
    assert Tp[4][1].item() == Tf.norms[1].item()
    assert abs(Tp[4][0].item() - Tf.norms[0].item()) <= 66 * 2.0 ** -24 * Tp[4][0].item()


# A first mode outside the tensor-core kernels (I_0 % 8 != 0 with I_0 > 128, or another mode
# processed first) runs in FP32 on the CUDA cores under RH_F32_BF16X2; every later mode whose core
# is written with it first (unit stride) goes to the tensor cores when I_n % 8 == 0.  A first mode 0
# with I_0 <= 128 and r + p <= 32 runs on the small-row tensor-core kernels and the later modes on
# the CUDA cores.  The oracle sees the exact FP32 input and rounds Omega to BF16 on exactly the modes
# that report info bit 4.  Tolerances as for the two-piece form.
@pytest.mark.parametrize("shape,ranks,p,rho,tc_modes", [((130, 64, 40), (6, 5, 4), 5, [0, 1, 2], [1, 2]),
                                                        ((60, 128, 50), (5, 6, 4), 5, None, []),
                                                        ((137, 24, 23, 16), (4, 4, 4, 4), 3, [0, 1, 2, 3], [1, 3]),
                                                        ((90, 64, 40), (6, 5, 4), 5, [0, 1, 2], [0]),
                                                        ((17, 24, 23, 16), (4, 4, 4, 4), 3, [0, 1, 2, 3], [0])])
def test_rsthosvd_f32_split_first_mode_on_cuda_cores(rh, shape, ranks, p, rho, tc_modes):
    from oracle import tucker as otk
    from oracle.tensor import rel_error
    from workloads import lowrank_plus_noise_np

    d = len(shape)
    X = lowrank_plus_noise_np(list(shape), [max(ranks) + 2] * d, 0.8, 1e-3, seed=23).astype(np.float32)
    Xd = torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda()
    T = rh.rsthosvd(Xd, list(shape), list(ranks), p=p, seed=5, rho=rho, form="f32_bf16x2", clamp=True)
    torch.cuda.synchronize()
    info = T.info.cpu().numpy().tolist()
    assert [m for m in range(d) if info[m] & 4] == tc_modes, info
    assert not any(x & 16 for x in info), info   # no tensor-core wait gave up
    Xe = X.astype(np.float64)
    rnd = {m: "bf16" for m in tc_modes}
    out = otk.rsthosvd(Xe, list(ranks), p, 5, rho=rho, omega_round=rnd, record=True, clamp=True)
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
