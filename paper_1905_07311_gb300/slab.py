"""R-STHOSVD (Alg. 3 with RandSVD, Alg. 1) of a tensor cut along its last mode into slabs.

The slabs either live on different GPUs (one process per GPU, torch.distributed between them) or in
host memory and are streamed to one GPU (a tensor larger than the device memory it may use).  The
algorithm is Alg. 3 with the last mode processed last; what each step exchanges:

  mode n < d-1  Y_n = sum over slabs of X_(n),s Omega_n,s: each slab's columns are a contiguous
                block of Kolda columns, so its sketch uses the global Omega rows row0 = L R' k0
                (L, R' the sizes before and between, k0 the slab's first last-mode index) and the
                partial sketches add up -- an all-reduce of the I_n x ell matrix.  The QR runs on
                every rank on the same Y.  B_s = Q^T X_(n),s stays local.  The SVD of B = [B_1 ...]
                comes from the triangles of the local tall-skinny QRs, B_s^T = Q_s R_s: B has the
                left singular vectors of [R_1^T ... R_S^T], so the ell x ell triangles are all-gathered
                and every rank factors the same stack.  A_n, U_r on every rank; G_s <- U_r^T B_s local.
  mode d-1      each slab owns the rows k0 .. k1 - 1 of Y_{d-1} (Omega_{d-1} is indexed by the other
                modes only): the row blocks are all-gathered; QR on every rank; the partial mode
                products Q_s^T G_(d-1),s are all-reduced into B; its SVD, A_{d-1} and the core on
                every rank.

Every arithmetic step is a call of the C library (through ``Backend``); the communicator only moves
data (all-reduce sums, all-gathers).  ``Backend`` and ``Comm`` are small interfaces so that the
partition and exchange logic can be run with other implementations (a CPU test substitutes both).
"""

# ---------------------------------------------------------------------------------------------
# communicators
# ---------------------------------------------------------------------------------------------
class SelfComm:
    """One rank: every exchange is the identity."""

    rank, world = 0, 1

    def allreduce_sum(self, t):
        return t

    def allgather(self, t):
        return [t]

    def allgather_ints(self, values):
        return [[int(v) for v in values]]


class TorchComm:
    """torch.distributed (NCCL for CUDA tensors, gloo for host tensors) on the default group."""

    def __init__(self):
        import torch
        import torch.distributed as dist

        self.dist = dist
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()
        # where the small host-side exchanges live: NCCL moves device tensors only
        nccl = dist.get_backend() == "nccl"
        self.device = torch.device("cuda", torch.cuda.current_device()) if nccl else torch.device("cpu")

    def allgather_ints(self, values):
        """Every rank's list of integers (the lists have the same length on every rank)."""
        import torch

        t = torch.tensor([int(v) for v in values], dtype=torch.int64, device=self.device)
        out = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(out, t)
        return [[int(v) for v in o.tolist()] for o in out]

    def allreduce_sum(self, t):
        self.dist.all_reduce(t)
        return t

    def allgather(self, t):
        """Tensors of every rank (all of t's shape but the last dimension must agree)."""
        import torch

        n = torch.tensor([t.shape[-1]], dtype=torch.int64, device=t.device)
        sizes = [torch.empty_like(n) for _ in range(self.world)]
        self.dist.all_gather(sizes, n)
        sizes = [int(v.item()) for v in sizes]
        width = max(sizes)
        pad = t
        if t.shape[-1] < width:
            pad = torch.zeros(t.shape[:-1] + (width,), dtype=t.dtype, device=t.device)
            pad[..., : t.shape[-1]] = t
        out = [torch.empty_like(pad) for _ in range(self.world)]
        self.dist.all_gather(out, pad.contiguous())
        return [o[..., :w] for o, w in zip(out, sizes)]


# ---------------------------------------------------------------------------------------------
# the library's operations on device tensors
# ---------------------------------------------------------------------------------------------
class LibraryBackend:
    """Steps of the decomposition as calls of the C library on CUDA tensors.  Layouts follow the
    binding: a matrix M (rows x cols, column-major) is the tensor of shape (cols, rows); a tensor is
    flat and column-major."""

    def __init__(self, form="f32"):
        import paper_1905_07311_gb300 as rh
        import torch

        self.rh, self.torch = rh, torch
        self.form = form              # "f64", "f32" or "f32_bf16x2" (first mode on the tensor cores)

    def dtype(self):
        return self.torch.float64 if self.form == "f64" else self.torch.float32

    def sketch(self, X, dims, mode, ell, row0, seed, tensor_id, Y=None, norm=None, first=False):
        form = "f32_bf16x2" if (first and self.form == "f32_bf16x2") else None
        return self.rh.rhosvd_sketch_offset(X, dims, mode, ell, row0, seed=seed, tensor_id=tensor_id, with_norm=True,
                                            form=form, Y=Y, norm=norm)

    def orth(self, Y):
        return self.rh.orthonormalize(Y)[0]

    def mode_product(self, X, dims, mode, A, first=False, out64=False):
        """X x_mode A^T with A the (k, I_mode) tensor of an I_mode x k FP64 matrix; output in the data
        precision (FP64 with out64).  The first mode of an f32_bf16x2 decomposition runs on the
        tensor cores."""
        if first and self.form == "f32_bf16x2":
            Y = self.rh.mode_product_bf16(X, dims, A.contiguous(), pieces="f32")
            out = list(dims)
            out[0] = int(A.shape[0])
            return Y.reshape(-1), out
        Ac = A if X.dtype == self.torch.float64 else self.rh.cast_f64(A, self.torch.float32)
        return self.rh.mode_product(X, dims, mode, Ac, out_dtype=self.torch.float64 if out64 else None)

    def tsqr_r(self, B, dims, mode):
        return self.rh.tall_skinny_r(B, dims, mode)

    def left_svd(self, B, dims, mode):
        return self.rh.left_svd(B, dims, mode)

    def factor(self, Q, U, r):
        return self.rh.tucker_factor(Q, U, r)

    def norm2(self, X, dims):
        """||X||^2 by the library (the sketch's norm accumulation with one column)."""
        _, n2 = self.rh.rhosvd_sketch_offset(X, dims, 0, 1, 0, with_norm=True)
        return n2


# ---------------------------------------------------------------------------------------------
# slabs
# ---------------------------------------------------------------------------------------------
class Slab:
    """X[..., k0:k1] of the global tensor: a flat column-major tensor of sizes dims[:-1] + [k1 - k0],
    on the device, or in (pinned) host memory and copied to ``device`` each time it is used."""

    def __init__(self, k0, k1, data, device=None):
        self.k0, self.k1, self.data, self.device = int(k0), int(k1), data, device

    def resident(self):
        return self.device is None or self.data.device == self.device

    def get(self):
        if self.resident():
            return self.data
        return self.data.to(self.device, non_blocking=True)


def _streamed(slabs, torch):
    """The slabs' device tensors in order.  Host-resident slabs are copied on a side stream one slab
    ahead of their use (two slabs in flight at most), so the host-to-device copy of slab s + 1
    overlaps the kernels of slab s; each copy is ordered before its use by an event."""
    if all(s.resident() for s in slabs):
        for s in slabs:
            yield s.data
        return
    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=cur.device)

    def issue(s):
        if s.resident():
            return s.data, None
        side.wait_stream(cur)          # the slot the copy lands in is free once earlier work is done
        with torch.cuda.stream(side):
            t = s.data.to(s.device, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(side)
        return t, ev

    nxt = issue(slabs[0])
    for i in range(len(slabs)):
        t, ev = nxt
        if i + 1 < len(slabs):
            nxt = issue(slabs[i + 1])
        if ev is not None:
            cur.wait_event(ev)
            t.record_stream(cur)
        yield t


def _prod(v):
    out = 1
    for x in v:
        out *= int(x)
    return out


def _ell(r, p, I, M, clamp):
    ell = int(r) + int(p)
    if ell > min(I, M):
        if not clamp:
            raise ValueError(f"r + p = {ell} exceeds min(I_n, prod of the other sizes) = {min(I, M)}")
        ell = min(I, M)
    if ell > 64:
        raise ValueError("r + p must be <= 64")
    return ell


def _validate(slabs, dims, ranks, p, seed, tensor_id, clamp, comm):
    """Checks that every rank takes in the same order and answers the same way, before any collective
    of the decomposition, so that a misconfigured rank makes every rank raise the same error instead
    of leaving the others in a collective of another size: the same sizes, ranks and options on every
    rank; each rank's slabs consecutive, non-empty and of sizes dims[:-1] + [k1 - k0]; the ranks'
    ranges tiling 0 .. dims[-1] in rank order."""
    import hashlib

    per = _prod(dims[:-1])
    ok = 1 if slabs and len(ranks) == len(dims) else 0
    for a, b in zip(slabs, slabs[1:]):
        ok &= 1 if a.k1 == b.k0 else 0
    for sl in slabs:
        ok &= 1 if sl.k1 > sl.k0 and sl.data.numel() == per * (sl.k1 - sl.k0) else 0
    k_lo, k_hi = (slabs[0].k0, slabs[-1].k1) if slabs else (-1, -1)
    conf = repr(([int(v) for v in dims], [int(v) for v in ranks], int(p), int(seed), int(tensor_id), bool(clamp)))
    digest = int.from_bytes(hashlib.sha256(conf.encode()).digest()[:7], "little")
    rows = comm.allgather_ints([k_lo, k_hi, ok, digest])
    if any(r[3] != rows[0][3] for r in rows):
        raise ValueError("the ranks disagree on the sizes, ranks or options of the decomposition")
    bad = [i for i, r in enumerate(rows) if not r[2]]
    if bad:
        raise ValueError(f"rank(s) {bad}: slabs empty, not consecutive, or not of sizes dims[:-1] + [k1 - k0]")
    edges = [0] + [r[1] for r in rows]
    if any(r[0] != e for r, e in zip(rows, edges)) or edges[-1] != int(dims[-1]):
        raise ValueError("the ranks' slabs do not tile 0 .. dims[-1] in rank order: "
                         + ", ".join(f"[{r[0]}, {r[1]})" for r in rows))


class SlabResult:
    def __init__(self, factors, core, core_dims, norm_x2):
        self.factors, self.core, self.core_dims, self.norm_x2 = factors, core, core_dims, norm_x2


def rsthosvd_slabs(slabs, dims, ranks, p=5, seed=0, tensor_id=0, comm=None, backend=None, clamp=False,
                   validate=True):
    """R-STHOSVD of the global tensor of sizes ``dims`` whose slabs along the last mode are given by
    ``slabs`` (this rank's, consecutive, in increasing k0; together the ranks' slabs cover
    0 .. dims[-1] in rank order).  Modes 0 .. d-2 in increasing order, then the last mode.  Returns the
    factors (list of (r_n, I_n) FP64 tensors: column-major I_n x r_n), the FP64 core (flat,
    r_0 x ... x r_{d-1}) on every rank and ||X||^2.  ``validate`` first checks across the ranks that
    they agree on the problem and that their slabs tile the last mode (one small all-gather; every
    rank raises the same ValueError otherwise); a caller repeating the same call may skip it."""
    comm = comm or SelfComm()
    be = backend or LibraryBackend()
    torch = be.torch
    d = len(dims)
    if d < 2:
        raise ValueError("a slab partition needs at least two modes")
    if validate:
        _validate(slabs, dims, ranks, p, seed, tensor_id, clamp, comm)
    cur = [int(v) for v in dims]
    k_lo, k_hi = slabs[0].k0, slabs[-1].k1
    for a, b in zip(slabs, slabs[1:]):
        if a.k1 != b.k0:
            raise ValueError("a rank's slabs must be consecutive")
    K = k_hi - k_lo
    factors = [None] * d
    local, ldims = None, None     # this rank's current core: sizes cur[:-1] + [K]
    norm_x2 = None
    for n in range(d - 1):
        I = cur[n]
        M = _prod(cur) // I
        ell = _ell(ranks[n], p, I, M, clamp)
        r = min(int(ranks[n]), ell)
        L, Rm = _prod(cur[:n]), _prod(cur[n + 1:d - 1])
        first = n == 0
        # Y_n: the slabs' sketches with their global Omega rows, summed on the device, then across ranks
        Y = nrm = None
        if first:
            for s, Xs in zip(slabs, _streamed(slabs, torch)):
                sd = cur[:-1] + [s.k1 - s.k0]
                Y, nrm = be.sketch(Xs, sd, 0, ell, L * Rm * s.k0, seed, tensor_id, Y=Y, norm=nrm, first=True)
        else:
            Y, _ = be.sketch(local, ldims, n, ell, L * Rm * k_lo, seed, tensor_id)
        Y = comm.allreduce_sum(Y)
        if first:
            norm_x2 = comm.allreduce_sum(nrm)
        Q = be.orth(Y)
        # B_s = Q^T X_(n),s (local), stacked along the last mode
        if first:
            parts = []
            for s, Xs in zip(slabs, _streamed(slabs, torch)):
                sd = cur[:-1] + [s.k1 - s.k0]
                Bs, bd = be.mode_product(Xs, sd, 0, Q, first=True)
                parts.append(Bs)
            B = parts[0] if len(parts) == 1 else torch.cat(parts)
            bdims = [ell] + cur[1:-1] + [K]
        else:
            B, bdims = be.mode_product(local, ldims, n, Q)
        # SVD of the global B from the stacked triangles of the local tall-skinny QRs
        Rloc = be.tsqr_r(B, bdims, n)                       # (ell, ell) tensor: row c = column c of R
        Rs = comm.allgather(Rloc)
        # the ell x (W ell) matrix [R_1^T ... R_W^T] as its (W ell, ell) tensor: block s is R_s's tensor
        # transposed
        C = torch.cat([R.t() for R in Rs]).contiguous()
        U, _ = be.left_svd(C.reshape(-1), [ell, ell * len(Rs)], 0)
        A, Ur = be.factor(Q, U, r)
        factors[n] = A
        local, ldims = be.mode_product(B, bdims, n, Ur)
        cur[n] = r
    # the last mode: rows k_lo .. k_hi of Y are this rank's
    n = d - 1
    I = cur[n]
    M = _prod(cur) // I
    ell = _ell(ranks[n], p, I, M, clamp)
    r = min(int(ranks[n]), ell)
    Yloc, _ = be.sketch(local, ldims, n, ell, 0, seed, tensor_id)   # (ell, K)
    Y = torch.cat(comm.allgather(Yloc), dim=1).contiguous()          # (ell, I): ranks in slab order
    Q = be.orth(Y)
    Qloc = Q[:, k_lo:k_hi].contiguous()
    # the partial products in FP64 (the last mode's B is small): its SVD and the core in FP64
    Bp, bdims = be.mode_product(local, ldims, n, Qloc, out64=True)
    B = comm.allreduce_sum(Bp)
    U, _ = be.left_svd(B, bdims, n)
    A, Ur = be.factor(Q, U, r)
    factors[n] = A
    core, cdims = be.mode_product(B, bdims, n, Ur, out64=True)
    cur[n] = r
    return SlabResult(factors, core, cdims, norm_x2)


def even_slabs(K, parts):
    """Bounds of ``parts`` consecutive slabs covering 0 .. K as evenly as possible."""
    return [(K * i // parts, K * (i + 1) // parts) for i in range(parts)]


__all__ = ["SelfComm", "TorchComm", "LibraryBackend", "Slab", "rsthosvd_slabs", "even_slabs", "SlabResult"]
