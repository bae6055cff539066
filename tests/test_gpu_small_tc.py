"""Small-row tensor-core kernels (a first mode with I_0 <= 128, r + p <= 32, any I_0) against the
oracle and the definitions (needs a GB300).

Every product on the tensor cores is exact (BF16 pieces times BF16 pieces), so only the sums round:
  sketch        |Y - X_rep Omega_bf16| <= (K + 8) 2^-24 (|X_rep| |Omega_bf16|), K the columns one CTA
                accumulates in FP32 (the chunk of the kernel's plan: ceil(ceil(M / 64) / S) 64 with
                S = max(1, min(c SMs, ceil(ceil(M / 64) / t))), c and t the launch-shape knobs), FP64
                across CTAs;
  mode product  |B - A_rep^T X_rep| <= (I + 8) 2^-24 (|A_rep|^T |X_rep|), A split into two pieces;
  R-STHOSVD     the oracle on the values the tensor cores read (head + tail of FP32, the BF16 values,
                the pieces, or bf16 of the dequantized E4M3 values) with Omega of the first mode
                rounded to BF16: relative error within 1e-5, leading subspaces to 1e-3 (tau = 0.05),
                and within 2 % of the oracle's error on the tensor the storage stands for (the FP32
                tensor; for E4M3 the values its bytes and scales denote).
The batched grouped engine runs BF16-form batches of uneven shapes whose results equal single calls
bit for bit, and so do batches planned under non-default launch-shape knobs, which keep the oracle's
error.
"""

import contextlib

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
from oracle.tensor import rel_error, unfold  # noqa: E402
from workloads import bf16_bits_np, fp8_quantize_np, lowrank_plus_noise_np  # noqa: E402


def _flat32(X):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X, dtype=np.float32).ravel(order="F"))).cuda()


def _bits_to_f64(b):
    return (b.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _rep_split(X):
    x = np.asarray(X, dtype=np.float32)
    h = orng.round_bf16(x)
    t = orng.round_bf16((x - h).astype(np.float32))
    return h.astype(np.float64) + t.astype(np.float64)


def _inputs(rh, X, form):
    """(device input of the form, float64 values the tensor cores read, the tensor the storage
    stands for: the FP32 tensor, or for E4M3 the values its bytes and scales denote)."""
    X = np.asarray(X, dtype=np.float32)
    if form == "f32":
        return _flat32(X), _rep_split(X), X.astype(np.float64)
    if form == "pieces":
        return rh.split_bf16x2(_flat32(X)), _rep_split(X), X.astype(np.float64)
    if form == "bf16":
        bits = bf16_bits_np(X)
        return (torch.from_numpy(bits.view(np.int16).copy()).cuda(),
                np.reshape(_bits_to_f64(bits), X.shape, order="F"), X.astype(np.float64))
    if form == "fp8":
        buf = fp8_quantize_np(X)
        deq = np.asarray(fp8_dequantize(buf, X.shape), dtype=np.float64)
        return (torch.from_numpy(buf).cuda(), orng.round_bf16(deq.astype(np.float32)).astype(np.float64), deq)
    raise ValueError(form)


def _input(rh, X, form):
    return _inputs(rh, X, form)[:2]


PIECES = {"f32": "f32", "pieces": 2, "bf16": 1, "fp8": "fp8"}
FORMS = {"f32": "f32_bf16x2", "pieces": "bf16x2", "bf16": "bf16", "fp8": "fp8_e4m3"}


def _chunk(M):
    """Columns per CTA of the small-row tensor-core sketch under the current launch-shape knobs."""
    from paper_1905_07311_gb300 import _lib

    L = _lib.lib()
    per_sm = L.rh_tuning_get(b"small_tc_sketch.ctas_per_sm")
    min_tiles = L.rh_tuning_get(b"small_tc_sketch.min_tiles")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = -(-M // 64)
    S = max(1, min(per_sm * sms, -(-tiles // min_tiles)))
    return -(-tiles // S) * 64


# I_0 % 8 != 0: rhosvd_sketch and the mode product take the small-row kernel
@pytest.mark.parametrize("form", ["f32", "pieces", "bf16", "fp8"])
@pytest.mark.parametrize("shape", [(17, 300, 7), (97, 50, 41), (127, 1000), (1, 5000), (65, 33, 9, 5)])
@pytest.mark.parametrize("ell", [1, 13, 32])
def test_small_sketch_matches_oracle(rh, form, shape, ell):
    rs = np.random.default_rng(hash((form, shape, ell)) % 2 ** 32)
    X = rs.standard_normal(shape).astype(np.float32)
    Xin, Xrep = _input(rh, X, form)
    wn = form in ("f32", "fp8")
    out = rh.rhosvd_sketch_bf16(Xin, list(shape), ell, seed=9, tensor_id=4, pieces=PIECES[form], with_norm=wn)
    Y = (out[0] if wn else out).cpu().numpy().T
    Xm = unfold(Xrep, 0)
    M = Xm.shape[1]
    Om = orng.round_bf16(orng.omega(9, 4, 0, np.arange(M), ell)).astype(np.float64)
    ref = Xm @ Om
    bound = (_chunk(M) + 8) * 2.0 ** -24 * (np.abs(Xm) @ np.abs(Om)) + 1e-300
    assert np.all(np.abs(Y - ref) <= bound), np.max(np.abs(Y - ref) / bound)
    if wn:
        # FP32 sums of at most 32 values per thread and tile (positive terms), FP64 above
        n2 = float(np.sum(Xrep ** 2))
        assert abs(float(out[1].item()) - n2) <= 40 * 2.0 ** -24 * n2


@pytest.mark.parametrize("form", ["f32", "pieces", "bf16", "fp8"])
@pytest.mark.parametrize("shape,k", [((17, 300, 7), 9), ((97, 50, 41), 32), ((127, 1000), 1), ((65, 33, 9, 5), 17),
                                     ((3, 4000), 3)])
def test_small_mode_product_matches_definition(rh, form, shape, k):
    rs = np.random.default_rng(hash((form, shape, k)) % 2 ** 32)
    X = rs.standard_normal(shape).astype(np.float32)
    Xin, Xrep = _input(rh, X, form)
    I = shape[0]
    A = rs.standard_normal((I, k))
    Y = rh.mode_product_bf16(Xin, list(shape), torch.from_numpy(A.T.copy()).cuda(), pieces=PIECES[form])
    M = X.size // I
    B = Y.cpu().numpy().astype(np.float64).reshape(M, k).T
    Af = A.astype(np.float32)
    ah = orng.round_bf16(Af)
    at = orng.round_bf16((Af - ah).astype(np.float32))
    Arep = ah.astype(np.float64) + at.astype(np.float64)
    Xm = unfold(Xrep, 0)
    ref = Arep.T @ Xm
    bound = (I + 8) * 2.0 ** -24 * (np.abs(Arep).T @ np.abs(Xm)) + 1e-300
    assert np.all(np.abs(B - ref) <= bound), np.max(np.abs(B - ref) / bound)


@pytest.mark.parametrize("form", ["f32", "pieces", "bf16", "fp8"])
@pytest.mark.parametrize("shape,ranks,p", [((90, 64, 40), (6, 5, 4), 5), ((17, 24, 23, 16), (4, 4, 4, 4), 3),
                                           ((128, 60, 50), (10, 8, 6), 6), ((45, 70, 33), (20, 10, 8), 12)])
def test_rsthosvd_small_first_mode_matches_oracle(rh, form, shape, ranks, p):
    d = len(shape)
    X = lowrank_plus_noise_np(list(shape), [min(max(ranks) + 2, n) for n in shape], 0.8, 1e-3,
                              seed=41).astype(np.float32)
    Xin, Xrep, Xden = _inputs(rh, X, form)
    rho = list(range(d))
    T = rh.rsthosvd(Xin, list(shape), list(ranks), p=p, seed=6, rho=rho, form=FORMS[form], clamp=True)
    torch.cuda.synchronize()
    info = T.info.cpu().numpy().tolist()
    assert [m for m in range(d) if info[m] & 4] == [0], info   # the first mode alone, on the tensor cores
    assert not any(x & 16 for x in info), info
    out = otk.rsthosvd(Xrep, list(ranks), p, 6, rho=rho, omega_round={0: "bf16"}, record=True, clamp=True)
    A = [f.cpu().numpy().T for f in T.factors]
    G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
    e_g, e_o = rel_error(Xrep, G, A), rel_error(Xrep, out["core"], out["factors"])
    assert abs(e_g - e_o) <= 1e-5, (e_g, e_o)
    for rec in out["records"]:
        m = rec["mode"]
        sv = rec["sv_B"]
        k = max(1, int(np.sum(sv >= 0.05 * sv[0])))
        U = out["factors"][m][:, :k]
        Qa, _ = np.linalg.qr(A[m])
        assert np.linalg.norm(U - Qa @ (Qa.T @ U), 2) <= 1e-3, m
    n2 = float(np.sum(Xrep ** 2))
    assert abs(float(T.norms[0].item()) - n2) <= 40 * 2.0 ** -24 * n2
    # against the tensor the storage stands for: within 2 % of the oracle's error there
    ref = otk.rsthosvd(Xden, list(ranks), p, 6, rho=rho, omega_round={0: "bf16"}, clamp=True)
    e_ref = rel_error(Xden, ref["core"], ref["factors"])
    assert abs(rel_error(Xden, G, A) - e_ref) <= 0.02 * e_ref


def test_rsthosvd_small_pieces_and_split_bit_identical(rh):
    """The split form and the two-piece form read the same pieces through the same sums."""
    X = lowrank_plus_noise_np([90, 64, 40], [8, 8, 8], 0.8, 1e-3, seed=42).astype(np.float32)
    Xd = _flat32(X)
    Tp = rh.rsthosvd(rh.split_bf16x2(Xd), [90, 64, 40], [6, 5, 4], p=5, seed=3, rho=[0, 1, 2], form="bf16x2")
    Tp = [t.clone() for t in Tp.factors] + [Tp.core.clone(), Tp.norms.clone()]
    Tf = rh.rsthosvd(Xd, [90, 64, 40], [6, 5, 4], p=5, seed=3, rho=[0, 1, 2], form="f32_bf16x2")
    for a, b in zip(Tp[:3], Tf.factors):
        assert torch.equal(a, b)
    assert torch.equal(Tp[3], Tf.core)
    assert torch.equal(Tp[4], Tf.norms)


def _uneven_batch(n, seed):
    rs = np.random.default_rng(seed)
    out = []
    for t in range(n):
        d = 3 + (t % 2)
        dims = [int(x) for x in rs.integers(16, 60 if d == 4 else 97, d)]
        ranks = [int(min(x, r)) for x, r in zip(dims, rs.integers(4, 17, d))]
        out.append((dims, ranks))
    return out


@pytest.mark.parametrize("form", ["bf16", "f32"])
def test_batched_small_form_grouped_equals_single_calls(rh, form):
    batch = _uneven_batch(10, 5)
    Xs, reps = [], []
    for t, (dims, ranks) in enumerate(batch):
        X = lowrank_plus_noise_np(dims, [min(max(ranks) + 1, n) for n in dims], 0.9, 1e-3, seed=100 + t)
        Xin, Xrep = _input(rh, X, form)
        Xs.append(Xin)
        reps.append(Xrep)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    call = rh.RsthosvdBatchedCall(dims_list, ranks_list, FORMS[form], p=5, seed=2, tensor_id=3, clamp=True, streams=0,
                                  rho="natural")
    plan = call.plan(Xs)          # the grouped engine (a batched plan needs it)
    Ts = plan.run()
    torch.cuda.synchronize()
    got = [([f.clone() for f in T.factors], T.core.clone(), T.norms.clone(), T.info.clone()) for T in Ts]
    plan.close()
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=2, tensor_id=3 + i, clamp=True,
                         rho=list(range(len(dims_list[i]))), form=FORMS[form])
        torch.cuda.synchronize()
        fs, core, norms, info = got[i]
        for a, b in zip(fs, T1.factors):
            assert torch.equal(a, b)
        assert torch.equal(core, T1.core)
        assert torch.equal(norms, T1.norms)
        assert torch.equal(info, T1.info)
        assert info[0].item() & 4 and not any(int(x) & 16 for x in info.cpu().numpy())
    # one tensor against the oracle on the values read
    dims, ranks = batch[0]
    out = otk.rsthosvd(reps[0], ranks, 5, 2, rho=list(range(len(dims))), tensor_id=3, omega_round={0: "bf16"},
                       clamp=True)
    A = [f.cpu().numpy().T for f in got[0][0]]
    G = np.reshape(got[0][1].cpu().numpy(), call.core_dims[0], order="F")
    assert abs(rel_error(reps[0], G, A) - rel_error(reps[0], out["core"], out["factors"])) <= 1e-5


@contextlib.contextmanager
def _knobs(per_sm, min_work):
    """Every launch-shape knob set: CTAs per SM to ``per_sm``, minimum work per CTA to ``min_work``;
    the table's values come back on exit."""
    from paper_1905_07311_gb300 import _lib

    L = _lib.lib()
    names = [L.rh_tuning_name(i) for i in range(L.rh_tuning_count())]
    try:
        for n in names:
            _lib.check(L.rh_tuning_set(n, per_sm if n.endswith(b"ctas_per_sm") else min_work))
        yield
    finally:
        for n in names:
            _lib.check(L.rh_tuning_set(n, 0))


# spread: one tile (or k step) per CTA, up to 16 CTAs per SM; packed: one CTA per SM, 64 tiles each
@pytest.mark.parametrize("setting", [(16, 1), (1, 64)], ids=["spread", "packed"])
@pytest.mark.parametrize("form", ["f32", "cuda_cores"])
def test_launch_shape_knobs_keep_parity(rh, setting, form):
    batch = _uneven_batch(8, 11)
    Xs, reps = [], []
    for t, (dims, ranks) in enumerate(batch):
        X = lowrank_plus_noise_np(dims, [min(max(ranks) + 1, n) for n in dims], 0.9, 1e-3, seed=300 + t)
        if form == "cuda_cores":
            Xs.append(_flat32(X))
            reps.append(np.asarray(X, dtype=np.float32).astype(np.float64))
        else:
            Xin, Xrep = _input(rh, X, form)
            Xs.append(Xin)
            reps.append(Xrep)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    dt = torch.float32 if form == "cuda_cores" else FORMS[form]
    rho = None if form == "cuda_cores" else "natural"
    with _knobs(*setting):
        if form == "f32":
            # the sketch bound with the chunk these knobs give
            X = np.random.default_rng(8).standard_normal((97, 50, 41)).astype(np.float32)
            Xin, Xrep = _input(rh, X, form)
            Y = rh.rhosvd_sketch_bf16(Xin, [97, 50, 41], 13, seed=9, tensor_id=4, pieces="f32")
            Y = (Y[0] if isinstance(Y, tuple) else Y).cpu().numpy().T
            Xm = unfold(Xrep, 0)
            Om = orng.round_bf16(orng.omega(9, 4, 0, np.arange(Xm.shape[1]), 13)).astype(np.float64)
            bound = (_chunk(Xm.shape[1]) + 8) * 2.0 ** -24 * (np.abs(Xm) @ np.abs(Om)) + 1e-300
            assert np.all(np.abs(Y - Xm @ Om) <= bound)
        call = rh.RsthosvdBatchedCall(dims_list, ranks_list, dt, p=5, seed=2, tensor_id=3, clamp=True, streams=0,
                                      rho=rho)
        plan = call.plan(Xs)
        Ts = plan.run()
        torch.cuda.synchronize()
        got = [([f.clone() for f in T.factors], T.core.clone(), T.norms.clone()) for T in Ts]
        plan.close()
        for i, X in enumerate(Xs):
            kw = {} if rho is None else {"rho": list(range(len(dims_list[i]))), "form": FORMS[form]}
            T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=2, tensor_id=3 + i, clamp=True, **kw)
            torch.cuda.synchronize()
            for a, b in zip(got[i][0], T1.factors):
                assert torch.equal(a, b)
            assert torch.equal(got[i][1], T1.core)
            assert torch.equal(got[i][2], T1.norms)
    for i, ((dims, ranks), Xr) in enumerate(zip(batch, reps)):
        if rho is None:
            out = otk.rsthosvd(Xr, ranks, 5, 2, tensor_id=3 + i, clamp=True)
        else:
            out = otk.rsthosvd(Xr, ranks, 5, 2, rho=list(range(len(dims))), tensor_id=3 + i,
                               omega_round={0: "bf16"}, clamp=True)
        A = [f.cpu().numpy().T for f in got[i][0]]
        G = np.reshape(got[i][1].cpu().numpy(), [a.shape[1] for a in A], order="F")
        assert abs(rel_error(Xr, G, A) - rel_error(Xr, out["core"], out["factors"])) <= 1e-5, (i, dims)
        if rho is None:
            n2 = float(np.sum(Xr ** 2))
            assert abs(got[i][2][0].item() - n2) <= 40 * 2.0 ** -24 * n2
