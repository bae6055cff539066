"""R-STHOSVD through ``rsthosvd_host`` (host buffers: the copy of X to the device, the decomposition
and the copies of the factors, core and norms back, all enqueued on one stream).  Needs a GB300.

The device part runs the same plan and kernels as ``rsthosvd`` on a device-resident copy of the
input, so every output must be bit-identical to that call, for each storage form (FP64, FP32, FP32
split on the fly, BF16, block-scaled E4M3) and from pinned as well as pageable host memory; the
device call itself is pinned to the oracle by the parity tests.
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


from workloads import bf16_bits_np, fp8_quantize_np, lowrank_plus_noise_np  # noqa: E402


def _host_input(form, shape):
    X = lowrank_plus_noise_np(list(shape), [10] * len(shape), 0.8, 1e-3, seed=41)
    if form == "float64":
        return torch.from_numpy(np.ascontiguousarray(X.ravel(order="F")))
    if form in ("float32", "f32_bf16x2"):
        return torch.from_numpy(np.ascontiguousarray(X.astype(np.float32).ravel(order="F")))
    if form == "bf16":
        return torch.from_numpy(bf16_bits_np(X).view(np.int16).copy())
    return torch.from_numpy(fp8_quantize_np(X.astype(np.float32)))


@pytest.mark.parametrize("form,shape,ranks,p", [("float64", (60, 48, 40), (6, 5, 4), 4),
                                                ("float32", (60, 48, 40), (6, 5, 4), 4),
                                                ("f32_bf16x2", (128, 48, 40), (8, 6, 5), 6),
                                                ("bf16", (128, 48, 40), (8, 6, 5), 6),
                                                ("fp8_e4m3", (128, 48, 40), (8, 6, 5), 6)])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_call_equals_device_call(rh, form, shape, ranks, p, pinned):
    host = _host_input(form, shape)
    if pinned:
        host = host.pin_memory()
    dtype = {"float64": torch.float64, "float32": torch.float32}.get(form, form)
    hc = rh.RsthosvdHostCall(list(shape), dtype, list(ranks), p=p, seed=3)
    hc.run(host)
    torch.cuda.synchronize()
    T = rh.rsthosvd(host.cuda(), list(shape), list(ranks), p=p, seed=3,
                    form=None if form in ("float64", "float32") else form)
    torch.cuda.synchronize()
    assert hc.h2d_bytes == host.numel() * host.element_size()
    for fh, fd in zip(hc.factors, T.factors):
        assert torch.equal(fh, fd.cpu())
    assert torch.equal(hc.core, T.core.cpu())
    assert torch.equal(hc.norms, T.norms.cpu())


def test_host_call_rejects_a_device_tensor(rh):
    hc = rh.RsthosvdHostCall([60, 48, 40], torch.float32, [6, 5, 4], p=4)
    with pytest.raises(ValueError, match="host tensor"):
        hc.run(torch.zeros(60 * 48 * 40, dtype=torch.float32, device="cuda"))
