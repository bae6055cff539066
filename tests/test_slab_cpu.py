"""The slab partition of R-STHOSVD (``paper_1905_07311_gb300.slab``) on CPU ranks (gloo, world sizes 2 and 3).

The partition and exchange logic -- global Omega rows per slab, the all-reduce of the sketches, the
all-gather of the tall-skinny triangles and of the last mode's row blocks, the all-reduce of the
last mode's partial products -- runs unchanged; the per-slab arithmetic comes from a stand-in
backend written with numpy for these host tensors (the library itself needs a GPU).  Checked:
  * the slabs' sketches with their global Omega rows add up to the whole tensor's sketch;
  * the left singular vectors of the stacked triangles [R_1^T R_2^T] are those of B itself;
  * the whole decomposition equals the oracle's R-STHOSVD (Alg. 3, modes in order) to 1e-12,
    with even and uneven slabs, with two slabs on one rank, and on three ranks for a 4-way tensor.
"""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class NumpyBackend:
    """The library's steps for FP64 host tensors, in the binding's layouts: a matrix (rows x cols,
    column-major) is the (cols, rows) tensor; a tensor is flat and column-major."""

    torch = torch

    def __init__(self):
        from oracle import rng, tucker
        from oracle.tensor import fold, unfold

        self.rng, self.tk, self.fold, self.unfold = rng, tucker, fold, unfold

    def _t(self, x, dims):
        return np.reshape(x.numpy(), dims, order="F")

    def _flat(self, X):
        return torch.from_numpy(np.ascontiguousarray(np.ravel(X, order="F")))

    def _mat(self, M):             # numpy rows x cols -> (cols, rows) tensor
        return torch.from_numpy(np.ascontiguousarray(M.T))

    def _np(self, t):              # (cols, rows) tensor -> numpy rows x cols
        return t.numpy().T

    def sketch(self, X, dims, mode, ell, row0, seed, tensor_id, Y=None, norm=None, first=False):
        Xm = self.unfold(self._t(X, dims), mode)
        M = Xm.shape[1]
        Om = self.rng.omega(seed, tensor_id, mode, np.arange(row0, row0 + M, dtype=np.int64), ell).astype(np.float64)
        Ys = self._mat(Xm @ Om)
        ns = torch.tensor([float(np.sum(Xm ** 2))], dtype=torch.float64)
        if Y is not None:
            Ys = Y + Ys
            ns = norm + ns
        return Ys, ns

    def orth(self, Y):
        return self._mat(self.tk.canon_qr(self._np(Y)))

    def mode_product(self, X, dims, mode, A, first=False, out64=False):
        T = self._t(X, dims)
        Am = self._np(A)                                   # I_mode x k
        out = list(dims)
        out[mode] = Am.shape[1]
        Y = self.fold(Am.T @ self.unfold(T, mode), mode, out)
        return self._flat(Y), out

    def tsqr_r(self, B, dims, mode):
        R = np.linalg.qr(self.unfold(self._t(B, dims), mode).T, mode="r")
        n = dims[mode]
        Rf = np.zeros((n, n))
        Rf[: R.shape[0], :] = R
        return self._mat(Rf)

    def left_svd(self, B, dims, mode):
        U, s, _ = np.linalg.svd(self.unfold(self._t(B, dims), mode), full_matrices=False)
        return self._mat(U), torch.from_numpy(s)

    def factor(self, Q, U, r):
        A = self._np(Q) @ self._np(U)[:, :r]
        sg = self.tk.canon_signs(A)
        return self._mat(A * sg), self._mat(self._np(U)[:, :r] * sg)


def _tensor(dims, seed):
    from workloads import lowrank_plus_noise_np

    return lowrank_plus_noise_np(dims, [5] * len(dims), 0.8, 1e-2, seed=seed)


def _slabs_of(X, bounds):
    from paper_1905_07311_gb300.slab import Slab

    return [Slab(k0, k1, torch.from_numpy(np.ascontiguousarray(np.ravel(X[..., k0:k1], order="F"))))
            for k0, k1 in bounds]


def _rank_main(rank, world, port, dims, ranks, p, seed, bounds_per_rank, out):
    sys.path.insert(0, ROOT)
    from paper_1905_07311_gb300 import slab

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        X = _tensor(dims, 3)
        be = NumpyBackend()
        comm = slab.TorchComm()
        # the slabs' sketches of mode 0 with global Omega rows, reduced across ranks
        ell = ranks[0] + p
        Y = nrm = None
        for s in _slabs_of(X, bounds_per_rank[rank]):
            sd = dims[:-1] + [s.k1 - s.k0]
            L, Rm = 1, int(np.prod(dims[1:-1]))
            Y, nrm = be.sketch(s.get(), sd, 0, ell, L * Rm * s.k0, seed, 0, Y=Y, norm=nrm)
        Y = comm.allreduce_sum(Y)
        # the triangles of mode 0's B from every rank
        res = slab.rsthosvd_slabs(_slabs_of(X, bounds_per_rank[rank]), dims, ranks, p=p, seed=seed, comm=comm,
                                  backend=be)
        out[rank] = {"Y": Y.numpy().copy(), "factors": [f.numpy().copy() for f in res.factors],
                     "core": res.core.numpy().copy(), "core_dims": list(res.core_dims),
                     "norm": float(res.norm_x2.item())}
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dims,ranks,bounds", [
    ([20, 18, 16], [4, 5, 3], [[(0, 8)], [(8, 16)]]),
    ([20, 18, 16], [4, 5, 3], [[(0, 5)], [(5, 16)]]),
    ([20, 18, 16], [4, 5, 3], [[(0, 3), (3, 9)], [(9, 16)]]),
    # three ranks on a 4-way tensor, uneven slabs, one rank with two slabs
    ([10, 9, 8, 12], [4, 3, 4, 3], [[(0, 2)], [(2, 5), (5, 9)], [(9, 12)]]),
])
def test_slab_partition_on_gloo_ranks_equals_one_tensor(dims, ranks, bounds):
    from oracle import rng, tucker
    from oracle.tensor import rel_error, unfold

    p, seed = 3, 11
    world = len(bounds)
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [mp.Process(target=_rank_main, args=(r, world, port, dims, ranks, p, seed, bounds, out))
                 for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=180)
            assert pr.exitcode == 0
        res = {k: dict(v) for k, v in out.items()}
    X = _tensor(dims, 3)
    # the slab sketches with global Omega rows sum to the whole tensor's sketch
    Xm = unfold(X, 0)
    Yfull = Xm @ rng.omega(seed, 0, 0, np.arange(Xm.shape[1]), ranks[0] + p).astype(np.float64)
    for r in range(world):
        assert np.allclose(res[r]["Y"].T, Yfull, rtol=0, atol=1e-12 * np.abs(Yfull).max())
    # every rank holds the same decomposition, equal to the oracle's
    ref = tucker.rsthosvd(X, ranks, p, seed, rho=list(range(len(dims))))
    for r in range(world):
        A = [f.T for f in res[r]["factors"]]
        G = np.reshape(res[r]["core"], res[r]["core_dims"], order="F")
        for n in range(len(dims)):
            assert np.allclose(A[n], ref["factors"][n], rtol=0, atol=1e-10)
        assert np.allclose(G, ref["core"], rtol=0, atol=1e-10 * np.abs(ref["core"]).max())
        assert abs(rel_error(X, G, A) - rel_error(X, ref["core"], ref["factors"])) <= 1e-12
        assert abs(res[r]["norm"] - float(np.sum(X ** 2))) <= 1e-12 * float(np.sum(X ** 2))


def test_stacked_triangles_give_the_left_singular_vectors_of_b():
    """B = [B_1 B_2] (columns split): with B_s^T = Q_s R_s, B and [R_1^T R_2^T] have the same left
    singular vectors and values (checked on a random ell x m matrix, as a pure identity)."""
    rs = np.random.default_rng(5)
    B = rs.standard_normal((9, 70)) * (0.7 ** np.arange(9))[:, None]
    R1 = np.linalg.qr(B[:, :30].T, mode="r")
    R2 = np.linalg.qr(B[:, 30:].T, mode="r")
    C = np.hstack([R1.T, R2.T])
    U, s, _ = np.linalg.svd(B, full_matrices=False)
    Uc, sc, _ = np.linalg.svd(C, full_matrices=False)
    assert np.allclose(s, sc, rtol=1e-12)
    assert np.allclose(np.abs(U.T @ Uc), np.eye(9), atol=1e-10)


def _bad_rank_main(rank, world, port, case, out):
    import datetime

    sys.path.insert(0, ROOT)
    from paper_1905_07311_gb300 import slab

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=60))
    try:
        dims, ranks, p = [12, 10, 8], [3, 3, 3], 2
        X = _tensor(dims, 4)
        bounds = {"good": [[(0, 4)], [(4, 8)]], "options": [[(0, 4)], [(4, 8)]], "gap": [[(0, 3)], [(4, 8)]],
                  "order": [[(4, 8)], [(0, 4)]], "short": [[(0, 4)], [(4, 7)]], "size": [[(0, 4)], [(4, 8)]],
                  "empty": [[(0, 8)], []]}[case][rank]
        slabs = _slabs_of(X, bounds)
        if case == "options" and rank == 1:
            p = 3
        if case == "size" and rank == 1:
            slabs[0] = slab.Slab(4, 8, slabs[0].data[:-1])
        try:
            slab.rsthosvd_slabs(slabs, dims, ranks, p=p, seed=1, comm=slab.TorchComm(), backend=NumpyBackend())
            out[rank] = "ok"
        except ValueError as e:
            out[rank] = "ValueError: " + str(e)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case,words", [("good", None), ("options", "disagree"), ("gap", "tile"),
                                        ("order", "tile"), ("short", "tile"), ("size", "rank(s) [1]"),
                                        ("empty", "rank(s) [1]")])
def test_misconfigured_ranks_all_raise_the_same_error(case, words):
    """A rank with other options, slabs that leave a gap, come out of rank order or stop short of the
    last mode, a slab of the wrong size, or no slab at all: every rank raises the same ValueError
    before the decomposition's first collective, so none is left waiting in it."""
    mp = torch.multiprocessing.get_context("spawn")
    with mp.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [mp.Process(target=_bad_rank_main, args=(r, 2, port, case, out)) for r in range(2)]
        for pr in procs:
            pr.start()
        try:
            for pr in procs:
                pr.join(timeout=120)
                assert pr.exitcode == 0
        finally:
            for pr in procs:
                if pr.is_alive():
                    pr.kill()
        res = dict(out)
    if words is None:
        assert res == {0: "ok", 1: "ok"}
    else:
        assert res[0] == res[1] and res[0].startswith("ValueError") and words in res[0], res
