"""Batched R-STHOSVD (Alg. 3 on each tensor of a batch of uneven shapes) through the C ABI.  Needs a GB300.

* Every tensor of a batch must equal, bit for bit, the single-tensor rsthosvd call with
  tensor_id = base + i, on both engines: the stream engine only changes which stream a tensor
  runs on; the grouped engine (streams = 0) runs each tensor's recorded launches inside grouped
  launches with the tensor's own grids and arguments, and every reduction of the single call is
  deterministic.  The grouped cases mix tensors whose truncation takes different routes (FP32
  Gram, double-float Gram, tall-skinny QR) and whose sketch QR takes the Householder branch, so
  the per-tensor device-side branches are exercised inside one grouped launch.
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


@pytest.mark.parametrize("form,streams", [(None, 0), (None, 3), ("f32_bf16x2", 8), ("f32_bf16x2", 0)])
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
    for streams in (4, 0):
        Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=1, clamp=True, streams=streams)
        torch.cuda.synchronize()
        _order5_check(rh, Ts, Xs, dims_list, ranks_list)


def _order5_check(rh, Ts, Xs, dims_list, ranks_list):
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=1, tensor_id=i, clamp=True)
        torch.cuda.synchronize()
        _same(Ts[i], T1)
        nx, ng = Ts[i].norms.cpu().numpy()
        assert ng <= nx * (1 + 1e-6)


@pytest.mark.parametrize("streams", [4, 0])
def test_batched_graph_capture(rh, streams):
    batch = _small_batch(16, 500_000)
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    call = rh.RsthosvdBatchedCall(dims_list, ranks_list, torch.float32, p=5, seed=3, clamp=True, streams=streams)
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


def _route_batch(dtype):
    """Recipe tensors plus tensors whose truncation or sketch QR leaves the default route."""
    batch = [(d, r, sd, None) for d, r, sd in _small_batch(6, 600_000)]
    batch.append(([90, 80, 70], [10, 10, 10], None, ([14] * 3, 0.4, 1e-7, 12)))      # double-float Gram
    batch.append(([300, 200, 130], [34, 34, 34], None, ([44] * 3, 0.55, 1e-7, 14)))  # Gram singular: QR
    batch.append(([50, 45, 40], [4, 4, 4], None, ([4] * 3, 0.8, 0.0, 13)))           # rank-deficient sketch
    Xs_np, Xs = [], []
    for dims, ranks, seed, spec in batch:
        if spec is None:
            X = lowrank_plus_noise_np(dims, ranks, 0.9, 1e-3, seed=seed)
        else:
            core, decay, noise, sd = spec
            X = lowrank_plus_noise_np(dims, core, decay, noise, seed=sd)
        X = X.astype(dtype)
        Xs_np.append(X.astype(np.float64))
        Xs.append(torch.from_numpy(np.ascontiguousarray(X.ravel(order="F"))).cuda())
    return [b[0] for b in batch], [b[1] for b in batch], Xs_np, Xs


def test_grouped_mixed_routes_equal_single_calls(rh):
    dims_list, ranks_list, _, Xs = _route_batch(np.float32)
    Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=4, seed=5, tensor_id=3, clamp=True, streams=0)
    torch.cuda.synchronize()
    bits = set()
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=4, seed=5, tensor_id=3 + i, clamp=True)
        torch.cuda.synchronize()
        _same(Ts[i], T1)
        assert torch.equal(Ts[i].info, T1.info)
        bits |= {v & 10 for v in Ts[i].info.cpu().numpy().tolist()}
    assert {2, 8, 0} <= bits, bits     # FP32 Gram, double-float Gram and QR routes all ran


def test_grouped_forced_qr_route(rh):
    batch = _small_batch(8, 1_000_000)
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=2, clamp=True, streams=0, svd_route=1)
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=2, tensor_id=i, clamp=True, svd_route=1)
        torch.cuda.synchronize()
        _same(Ts[i], T1)


def test_grouped_f64_equals_single_calls(rh):
    batch = _small_batch(8, 600_000)
    _, Xs = _make(batch, np.float64)
    dims_list = [b[0] for b in batch] + [[60, 50, 40]]
    ranks_list = [b[1] for b in batch] + [[8, 8, 8]]
    from workloads import hilbert

    Xh = hilbert([60, 50, 40], offset=1)
    Xs.append(torch.from_numpy(np.ascontiguousarray(Xh.ravel(order="F"))).cuda())
    Ts = rh.rsthosvd_batched(Xs, dims_list, ranks_list, p=5, seed=6, clamp=True, streams=0)
    for i, X in enumerate(Xs):
        T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=6, tensor_id=i, clamp=True)
        torch.cuda.synchronize()
        _same(Ts[i], T1)
        assert torch.equal(Ts[i].info, T1.info)
    assert Ts[-1].info.cpu().numpy().tolist() == [1, 1, 1]   # Householder branch of the sketch QR


def test_batched_plan_reruns_on_new_data(rh):
    batch = _small_batch(40, 3_000_000)
    _, Xs = _make(batch)
    dims_list = [b[0] for b in batch]
    ranks_list = [b[1] for b in batch]
    call = rh.RsthosvdBatchedCall(dims_list, ranks_list, torch.float32, p=5, seed=8, clamp=True, streams=0)
    plan = call.plan(Xs)
    assert 0 < plan.launches <= 60 * max(len(d) for d in dims_list)
    for rep in range(2):
        if rep == 1:
            for X in Xs:
                X.mul_(-0.5).add_(0.25)          # new contents in the same buffers
        Ts = plan.run()
        torch.cuda.synchronize()
        for i, X in enumerate(Xs):
            T1 = rh.rsthosvd(X, dims_list[i], ranks_list[i], p=5, seed=8, tensor_id=i, clamp=True)
            torch.cuda.synchronize()
            _same(Ts[i], T1)
    plan.close()
