"""Low-precision storage forms on the tensor cores (needs a GB300).

E4M3 with per-128-byte FP32 scales (RH_FP8_E4M3): the kernels of the first mode dequantize each
tile, x = fl32(e4m3 * scale), and round it to one BF16 piece (ties to even), so
* the sketch, the mode product and the whole R-STHOSVD must be bit-identical to the BF16 form
  (RH_BF16) run on bf16(x) (the norm ||X||^2 only up to the order of its FP32 partial sums:
  relative 1e-6);
* against the oracle: relative Tucker error within 1e-5 absolute of the oracle's on the values
  the tensor cores see, bf16(x), with the same BF16-rounded Omega, and within 2 % of the oracle's
  on the tensor the bytes denote (oracle.storage), which is the agreement asked of the
  low-precision forms.
BF16 storage (RH_BF16): the oracle reads the BF16 values exactly; same gates.
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
from oracle.storage import fp8_dequantize  # noqa: E402
from oracle.tensor import rel_error  # noqa: E402
from workloads import bf16_bits_np, fp8_quantize_np, hilbert, lowrank_plus_noise_np  # noqa: E402


def _flat32(X):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X, dtype=np.float32).ravel(order="F"))).cuda()


def _rep_bf16x2(X):
    """head + tail of the FP32 values of X, as the tensor cores see them (float64)."""
    x = np.asarray(X, dtype=np.float32)
    h = orng.round_bf16(x)
    t = orng.round_bf16((x - h).astype(np.float32))
    return h.astype(np.float64) + t.astype(np.float64)


def _fp8(X):
    buf = fp8_quantize_np(X)
    return torch.from_numpy(buf).cuda(), fp8_dequantize(buf, X.shape)


def _bf16_of(X):
    """(int16 CUDA tensor of the BF16 bits, float64 values) of bf16(X) (ties to even), column-major."""
    x = np.asarray(X, dtype=np.float32)
    r = orng.round_bf16(x)
    bits = (np.ascontiguousarray(r.ravel(order="F")).view(np.uint32) >> 16).astype(np.uint16)
    return torch.from_numpy(bits.view(np.int16).copy()).cuda(), r.astype(np.float64)


@pytest.mark.parametrize("shape", [(128, 300, 7), (200, 40, 40), (1024, 64, 33), (96, 1000), (8, 5000)])
@pytest.mark.parametrize("ell", [1, 25, 64])
def test_fp8_sketch_bit_identical_to_bf16_of_dequantized(rh, shape, ell):
    rs = np.random.default_rng(hash((shape, ell)) % 2 ** 32)
    X = (rs.standard_normal(shape) * np.exp(rs.uniform(-4, 4, shape))).astype(np.float32)
    buf, Xdq = _fp8(X)
    Xb, Xbv = _bf16_of(Xdq)
    Y8, n8 = rh.rhosvd_sketch_bf16(buf, list(shape), ell, seed=5, tensor_id=3, pieces="fp8", with_norm=True)
    Yb = rh.rhosvd_sketch_bf16(Xb, list(shape), ell, seed=5, tensor_id=3, pieces=1)
    assert torch.equal(Y8, Yb)
    ref = float(np.sum(Xbv ** 2))
    assert abs(n8.item() - ref) <= 1e-6 * ref


@pytest.mark.parametrize("shape,k", [((128, 300), 60), ((200, 129), 1), ((200, 7, 9), 25), ((1024, 300), 64),
                                     ((8, 77, 3), 17)])
def test_fp8_mode_product_bit_identical_to_bf16_of_dequantized(rh, shape, k):
    rs = np.random.default_rng(7)
    X = rs.standard_normal(shape).astype(np.float32)
    buf, Xdq = _fp8(X)
    Xb, _ = _bf16_of(Xdq)
    A = torch.from_numpy(rs.standard_normal((k, shape[0]))).cuda()
    Y8 = rh.mode_product_bf16(buf, list(shape), A, pieces="fp8")
    Yb = rh.mode_product_bf16(Xb, list(shape), A, pieces=1)
    assert torch.equal(Y8, Yb)


def _check_vs_oracle(T, Xin, ranks, p, seed, rho, Xseen=None):
    """Xin: the tensor the storage denotes; Xseen: the values the first mode's tensor cores read
    (default: the head + tail split of Xin)."""
    d = Xin.ndim
    info = T.info.cpu().numpy().tolist()
    rnd = {m: "bf16" for m in range(d) if info[m] & 4}
    Xrep = _rep_bf16x2(Xin) if Xseen is None else Xseen
    A = [f.cpu().numpy().T for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g = rel_error(Xrep, G, A)
    out = otk.rsthosvd(Xrep, list(ranks), p, seed, rho=rho, omega_round=rnd)
    e_o = rel_error(Xrep, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    # the agreement asked of the low-precision forms: 2 % of the oracle's error on the input the
    # storage denotes, with the same Omega bits
    ref = otk.rsthosvd(np.asarray(Xin, dtype=np.float64), list(ranks), p, seed, rho=rho, omega_round=rnd)
    e_ref = rel_error(Xin, ref["core"], ref["factors"])
    e_in = rel_error(Xin, G, A)
    assert abs(e_in - e_ref) <= 0.02 * e_ref, (e_in, e_ref)
    return e_g, e_ref


@pytest.mark.parametrize("shape,ranks,p,rho", [((128, 60, 50), (6, 5, 4), 5, [0, 1, 2]),
                                               ((200, 64, 48), (12, 10, 8), 6, [0, 1, 2]),
                                               ((64, 40, 24, 16), (6, 5, 4, 3), 3, [0, 1, 3, 2])])
def test_rsthosvd_fp8(rh, shape, ranks, p, rho):
    d = len(shape)
    X = lowrank_plus_noise_np(list(shape), [max(ranks) + 2] * d, 0.8, 1e-3, seed=31).astype(np.float32)
    buf, Xdq = _fp8(X)
    Xb, Xbv = _bf16_of(Xdq)
    T8 = rh.rsthosvd(buf, list(shape), list(ranks), p=p, seed=4, rho=rho, form="fp8_e4m3")
    T8c = [f.clone() for f in T8.factors] + [T8.core.clone(), T8.norms.clone(), T8.info.clone()]
    Tf = rh.rsthosvd(Xb, list(shape), list(ranks), p=p, seed=4, rho=rho, form="bf16")
    torch.cuda.synchronize()
    for a, b in zip(T8c[:d], Tf.factors):
        assert torch.equal(a, b)
    assert torch.equal(T8c[d], Tf.core)
    assert torch.equal(T8c[d + 2], Tf.info)
    assert T8c[d + 1][1].item() == Tf.norms[1].item()
    assert abs(T8c[d + 1][0].item() - Tf.norms[0].item()) <= 1e-6 * Tf.norms[0].item()
    assert T8.info.cpu().numpy()[0] & 4
    _check_vs_oracle(T8, Xdq, ranks, p, 4, rho, Xseen=np.reshape(Xbv, Xdq.shape))


@pytest.mark.parametrize("form", ["fp8_e4m3", "bf16"])
def test_hilbert_200_low_precision_storage(rh, form):
    """The 200^3 tensor 1/(i+j+k+1) stored in E4M3 (block scales) or BF16; rank 20, p = 5, seed 0,
    order 1, 2, 3 (the FP64 configuration of the same tensor)."""
    X = hilbert([200, 200, 200], offset=1).astype(np.float32)
    Xseen = None
    if form == "fp8_e4m3":
        Xb, Xin = _fp8(X)
        Xseen = np.reshape(_bf16_of(Xin)[1], X.shape)
    else:
        bits = bf16_bits_np(X)
        Xb = torch.from_numpy(bits.view(np.int16).copy()).cuda()
        Xin = np.reshape((bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64), X.shape, order="F")
    T = rh.rsthosvd(Xb, [200, 200, 200], [20, 20, 20], p=5, seed=0, rho=[0, 1, 2], form=form)
    torch.cuda.synchronize()
    e_g, e_ref = _check_vs_oracle(T, Xin, [20, 20, 20], 5, 0, [0, 1, 2], Xseen=Xseen)
    # the error against the original tensor is the storage's quantisation error, not the method's
    A = [f.cpu().numpy().T for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_orig = rel_error(hilbert([200, 200, 200], offset=1), G, A)
    q = np.linalg.norm(Xin - hilbert([200, 200, 200], offset=1)) / np.linalg.norm(Xin)
    assert e_orig <= 1.01 * q + 1e-5, (e_orig, q)


# Adaptive R-STHOSVD (Alg. 5) on the stored forms: the first mode reads the stored tensor on the
# tensor cores with Omega rounded to BF16, the rest runs on the FP32 core.  The oracle runs the same
# reading of Alg. 5 on the represented input with the same Omega bits (BF16 on mode 1): the chosen
# ranks must agree and the errors within 1e-5.  E4M3 storage carries ~3 % quantisation noise that no
# low multilinear rank captures, so its tolerance is 5e-2; BF16 (2^-9) runs at 1e-2.
@pytest.mark.parametrize("form,eps,block", [("fp8_e4m3", 5e-2, 8), ("bf16", 1e-2, 8), ("f32_bf16x2", 1e-2, 4),
                                            ("bf16x2", 5e-2, 1)])
def test_adaptive_sthosvd_low_precision(rh, form, eps, block):
    shape = [96, 48, 40]
    X = lowrank_plus_noise_np(shape, [14, 12, 10], 0.7, 1e-4, seed=33).astype(np.float32)
    if form == "fp8_e4m3":
        Xb, Xin = _fp8(X)
        Xin = np.reshape(_bf16_of(Xin)[1], X.shape)   # the values the tensor cores read
    elif form == "bf16":
        bits = bf16_bits_np(X)
        Xb = torch.from_numpy(bits.view(np.int16).copy()).cuda()
        Xin = np.reshape((bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64), X.shape, order="F")
    elif form == "bf16x2":
        Xb = rh.split_bf16x2(_flat32(X))
        Xin = X.astype(np.float64)
    else:
        Xb = _flat32(X)
        Xin = X.astype(np.float64)
    T = rh.adaptive(Xb, shape, eps, variant="sthosvd", block=block, p=5, seed=4, form=form)
    torch.cuda.synchronize()
    Xrep = _rep_bf16x2(Xin)
    out = otk.adaptive_rsthosvd(Xrep, eps, block, 5, 4, omega_round={0: "bf16"})
    ranks_o = [f.shape[1] for f in out["factors"]]
    assert T.ranks == ranks_o, (T.ranks, ranks_o)
    A = [f.cpu().numpy().T.copy() for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.ranks, order="F")
    e_g = rel_error(Xrep, G, A)
    e_o = rel_error(Xrep, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    assert e_g <= eps * (1 + 1e-4)
    for a in A:
        assert np.abs(a.T @ a - np.eye(a.shape[1])).max() <= 2e-5
    nx = float(T.norms.cpu().numpy()[0])
    assert abs(nx - np.sum(Xrep ** 2)) <= 1e-6 * np.sum(Xrep ** 2)


def test_adaptive_low_precision_needs_mode0_first(rh):
    X = lowrank_plus_noise_np([40, 96, 32], [6, 6, 6], 0.7, 1e-4, seed=34).astype(np.float32)
    buf, _ = _fp8(X)
    with pytest.raises(ValueError):
        rh.adaptive(buf, [40, 96, 32], 5e-2, variant="sthosvd", p=5, form="fp8_e4m3")
    # the FP32-split form runs as plain FP32 instead
    T = rh.adaptive(_flat32(X), [40, 96, 32], 1e-2, variant="sthosvd", p=5, form="f32_bf16x2")
    T32 = rh.adaptive(_flat32(X), [40, 96, 32], 1e-2, variant="sthosvd", p=5)
    assert T.ranks == T32.ranks and torch.equal(T.core, T32.core)
