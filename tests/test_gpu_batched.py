"""Batched R-STHOSVD (Alg. 3 on each tensor of a batch of uneven shapes) through the C ABI.  Needs a GB300.

* Every tensor of a batch must equal, bit for bit, the single-tensor rsthosvd call with
  tensor_id = base + i: the batch only changes which stream a tensor runs on, and every
  reduction of the single call is deterministic.
* The single call itself is pinned to the oracle by tests/test_gpu_parity.py; here a subset of
  the batched workload (orders 3 and 4, sizes 16..96, ranks 4..16, low rank + 1e-3 noise) is
  also compared with the oracle directly at the FP32 tolerances of that file (relative Tucker
  error within 1e-5 absolute, orthonormal factors to 2e-5).
* A CUDA-graph capture of the batched call replays to the same bits.
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
from workloads import batch_recipe, lowrank_plus_noise_np  # noqa: E402


def _numel(dims):
    n = 1
    for v in dims:
        n *= v
    return n


def _small_batch(count, max_numel, orders=(3, 4)):
    out = []
    for dims, ranks, seed in batch_recipe():
        if len(dims) in orders and _numel(dims) <= max_numel:
            out.append((dims, ranks, seed))
        if len(out) == count:
            break
    return out


def _make(batch, dtype=np.float32):
    Xs_np, Xs = [], []
    for dims, ranks, seed in batch:
        X = lowrank_plus_noise_np(dims, ranks, 0.9, 1e-3, seed=seed).astype(dtype)
        Xs_np.append(X.astype(np.float64))
        Xs.append(torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda())
    return Xs_np, Xs


def _same(Ta, Tb):
    for fa, fb in zip(Ta.factors, Tb.factors):
        assert torch.equal(fa, fb)
    assert torch.equal(Ta.core, Tb.core)
    assert torch.equal(Ta.norms, Tb.norms)


def test_batched_matches_oracle(rh):
    batch = _small_batch(10, 400_000)
    Xe, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=4, tensor_id=100, clamp=True)
    torch.cuda.synchronize()
    for i, (T, X, (dims, ranks, _)) in enumerate(zip(Ts, Xe, batch)):
        out = otk.rsthosvd(X, ranks, 5, 4, tensor_id=100 + i, clamp=True)
        A = [f.cpu().numpy().T.copy() for f in T.factors]
        G = np.reshape(T.core.cpu().numpy(), T.core_dims, order="F")
        e_g = rel_error(X, G, A)
        e_o = rel_error(X, out["core"], out["factors"])
        assert abs(e_g - e_o) <= 1e-5, (i, dims, ranks, e_g, e_o)
        for a in A:
            assert np.abs(a.T @ a - np.eye(a.shape[1])).max() <= 2e-5
        nx = T.norms[0].item()
        assert abs(nx - np.sum(X ** 2)) <= 16 * 2.0 ** -24 * np.sum(X ** 2)


@pytest.mark.parametrize("form,streams", [(None, 0), (None, 3), ("f32_bf16x2", 8)])
def test_batched_equals_single_calls(rh, form, streams):
    batch = _small_batch(24, 2_000_000)
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=9, tensor_id=7, clamp=True, form=form,
                             streams=streams)
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=9, tensor_id=7 + i, clamp=True, form=form)
        torch.cuda.synchronize()
        _same(Ts[i], T1)


def test_batched_order5_and_mixed(rh):
    """Orders 3..5 in one batch (order-5 tensors at the small end of the size range)."""
    batch = []
    for dims, ranks, seed in batch_recipe():
        if _numel(dims) <= 3_000_000:
            batch.append((dims, ranks, seed))
        if len(batch) == 12:
            break
    assert {len(b[0]) for b in batch} >= {3, 4}
    batch.append(([16, 18, 17, 20, 16], [4, 5, 6, 4, 5], 77))
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=1, clamp=True, streams=4)
    torch.cuda.synchronize()
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=1, tensor_id=i, clamp=True)
        torch.cuda.synchronize()
        _same(Ts[i], T1)
        nx, ng = Ts[i].norms.cpu().numpy()
        assert ng <= nx * (1 + 1e-6)


def test_batched_graph_capture(rh):
    batch = _small_batch(16, 500_000)
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    call = rh.RsthosvdBatchedCall(dims_list, ranks_list, torch.float32, p=5, seed=3, clamp=True, streams=4)
    ref = call.run(Xs)
    torch.cuda.synchronize()
    snap = [(list(f.clone() for f in T.factors), T.core.clone()) for T in ref]
    for T in ref:
        T.core.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        call.run(Xs)                      # warm-up on the capture stream (function attributes, streams)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            call.run(Xs)
    for T in ref:
        T.core.zero_()
    g.replay()
    torch.cuda.synchronize()
    for T, (fs, c) in zip(ref, snap):
        assert torch.equal(T.core, c)
        for a, b in zip(T.factors, fs):
            assert torch.equal(a, b)


def test_batched_error_names_the_tensor(rh):
    batch = _small_batch(3, 400_000)
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [list(b[1]) for b in batch]
    ranks_list[1][0] = dims_list[1][0] + 1             # r + p > I_n without clamping
    with pytest.raises(rh.RhError, match="tensor 1"):
        rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5)
