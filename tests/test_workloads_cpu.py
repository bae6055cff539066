"""The seeded input recipes (``workloads``) against their stated construction (CPU only).

The tests and the benchmark feed both the CUDA path and the oracle from these generators, so their
shapes and structure are checked here on small sizes: the Hilbert-type entries, the multilinear
rank and noise level of the low-rank + noise tensors (numpy and torch versions), the Zipf COO
tensor (distinct, in range, sorted, its value law and index skew), the batch recipe's ranges and
the E4M3 storage's layout.
"""

import numpy as np
import pytest

import workloads as wl
from oracle.tensor import unfold


def test_hilbert_entries():
    X = wl.hilbert([4, 3, 5], offset=3)
    assert X.shape == (4, 3, 5) and X.flags["F_CONTIGUOUS"]
    for i, j, k in [(0, 0, 0), (3, 2, 4), (1, 2, 0)]:
        assert X[i, j, k] == 1.0 / (i + j + k + 3)


@pytest.mark.parametrize("noise", [0.0, 1e-2])
def test_lowrank_plus_noise_structure(noise):
    dims, core, decay = [14, 12, 10], [4, 3, 5], 0.8
    X = wl.lowrank_plus_noise_np(dims, core, decay, noise, seed=3)
    assert X.shape == tuple(dims) and X.flags["F_CONTIGUOUS"]
    S = wl.lowrank_plus_noise_np(dims, core, decay, 0.0, seed=3)          # the same signal
    for n in range(3):
        s = np.linalg.svd(unfold(S, n), compute_uv=False)
        assert s[core[n] - 1] > 1e-3 * s[0] and np.all(s[core[n]:] < 1e-12 * s[0])   # rank r_n exactly
    if noise:
        assert abs(np.linalg.norm(X - S) / np.linalg.norm(S) - noise) < 1e-12
    else:
        assert np.array_equal(X, S)
    assert np.array_equal(X, wl.lowrank_plus_noise_np(dims, core, decay, noise, seed=3))   # seeded


def test_lowrank_plus_noise_torch_structure():
    torch = pytest.importorskip("torch")
    dims, core = [12, 10, 9], [3, 4, 2]
    flat = wl.lowrank_plus_noise_torch(dims, core, 0.9, 1e-3, 5, torch.float64, torch.device("cpu"))
    sig = wl.lowrank_plus_noise_torch(dims, core, 0.9, 0.0, 5, torch.float64, torch.device("cpu"))
    X = np.reshape(flat.numpy(), dims, order="F")
    S = np.reshape(sig.numpy(), dims, order="F")
    for n in range(3):
        s = np.linalg.svd(unfold(S, n), compute_uv=False)
        assert np.all(s[core[n]:] < 1e-12 * s[0]) and s[core[n] - 1] > 1e-4 * s[0]
    assert abs(np.linalg.norm(X - S) / np.linalg.norm(S) - 1e-3) < 1e-9


def test_zipf_coo_structure():
    dims, nnz = [40, 30, 20], 3000
    idx, vals = wl.zipf_coo(dims, nnz, 1.1, 3.0, seed=5)
    assert idx.shape == (nnz, 3) and idx.dtype == np.int32 and vals.shape == (nnz,) and vals.dtype == np.float32
    assert np.all(idx >= 0) and np.all(idx < np.array(dims))
    keys = (idx[:, 0].astype(np.int64) * dims[1] + idx[:, 1]) * dims[2] + idx[:, 2]
    assert np.all(np.diff(keys) > 0)                        # distinct and sorted, mode 1 slowest
    # values log(1 + Poisson + 1): at least log 2, and exp(v) - 2 a non-negative integer
    c = np.exp(vals.astype(np.float64)) - 2.0
    assert np.all(vals >= np.float32(np.log(2.0))) and np.allclose(c, np.round(c), atol=1e-4)
    # Zipf skew: index 0 is the most frequent coordinate of every mode
    for n in range(3):
        counts = np.bincount(idx[:, n], minlength=dims[n])
        assert counts[0] == counts.max() and counts[0] > 3 * counts[dims[n] // 2]


def test_batch_recipe_ranges():
    rec = wl.batch_recipe()
    assert len(rec) == 512
    assert {len(d) for d, _, _ in rec} == {3, 4, 5}
    for i, (d, r, sd) in enumerate(rec):
        assert all(16 <= v <= 96 for v in d)
        assert all(1 <= a <= min(16, v) for a, v in zip(r, d)) and all(a >= min(4, v) for a, v in zip(r, d))
        assert sd == 4 * 100003 + i
    assert rec == wl.batch_recipe()                         # seeded


def test_fp8_storage_layout_matches_the_oracle_layout():
    from oracle import storage

    for dims in ([16, 3, 2], [20, 7], [130, 5, 3]):
        ld, off, nscales, total = storage.fp8_layout(dims)
        buf = wl.fp8_quantize_np(np.random.default_rng(1).standard_normal(dims))
        assert np.asarray(buf).size == total
        X = storage.fp8_dequantize(buf, dims)
        assert X.shape == tuple(dims)
