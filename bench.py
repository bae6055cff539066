"""Benchmark: R-STHOSVD time-to-Tucker and TFLOP/s on the dense 1024^3 FP32 workload.

Workload (one step = one full R-STHOSVD, Alg. 3 with RandSVD on every mode):
  X = G x_1 U_1 x_2 U_2 x_3 U_3 + E, 1024 x 1024 x 1024 FP32, core 50^3 of N(0,1) entries
  scaled by 0.9^(i+j+k), U_n orthonormal (QR of N(0,1) 1024 x 50), E Gaussian with
  ||E||_F = 1e-3 ||signal||_F; ranks (50, 50, 50), p = 10, Omega seed 0, order 1 -> 2 -> 3.
  X (4.3 GB) is far larger than L2, so no flush is needed between steps.

``value`` is algorithmic TFLOP/s summed over ranks (each rank decomposes its own tensor,
weak scaling, no data-path collective).  Algorithmic flops per mode with current core
size N_c, M = N_c / I_n and ell = r + p: sketch 2 N_c ell + mode product 2 N_c ell +
tall-skinny QR of B^T 4 M ell^2 + truncated-core product 2 M ell r.

Forms (--form): ``f32_bf16x2`` (default) reads the FP32 tensor once per first-mode kernel on the
tensor cores, splitting every tile into its exact BF16 head and tail in shared memory (16
significant bits of X, Omega rounded to BF16, FP32 accumulation; later modes FP32); ``f32`` is
the FP32 form on the CUDA cores throughout.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--form F]
       python bench.py --workload hilbert200|lowp192|batched|sparse [--steps K] [--warmup W]
"""

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "R-STHOSVD time-to-Tucker & TFLOP/s at equal rel. error vs plain FP64 GPU"
DIMS = [1024, 1024, 1024]
RANKS = [50, 50, 50]
P = 10
SEED = 0
RHO = [0, 1, 2]
WORKLOAD = "dense 3-way FP32 1024x1024x1024, low-rank 50^3 (decay 0.9) + 1e-3 noise; R-STHOSVD rank (50,50,50), p=10"


def algorithmic_flops(dims, ranks, p, rho):
    cur = list(dims)
    total = 0.0
    for n in rho:
        Nc = float(np.prod(cur))
        I = cur[n]
        M = Nc / I
        ell = min(ranks[n] + p, I, int(M))
        r = min(ranks[n], ell)
        total += 4.0 * Nc * ell + 4.0 * M * ell * ell + 2.0 * M * ell * r
        cur[n] = r
    return total


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", f"rh_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                t = [x.strip() for x in line.split(",")]
                if len(t) < 9:
                    continue
                try:
                    sm.append(float(t[1]))
                    smax.append(float(t[2]))
                except ValueError:
                    continue
                for name, v in zip(names, t[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_time_and_value(torch, dist, ms_local, flops_per_rank, world, device):
    """Whole-job time and throughput over the ranks: every rank decomposes its own tensor (weak
    scaling), the job takes as long as its slowest rank (max over ranks), and the value counts the
    work of all ranks.  Returns (ms per step, TFLOP/s); ``dist`` is None for a single process."""
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return ms, world * flops_per_rank / (ms * 1e-3) / 1e12


def make_input(torch, device, seed_offset=0):
    from workloads import lowrank_plus_noise_torch

    return lowrank_plus_noise_torch(DIMS, [50] * len(DIMS), 0.9, 1e-3, 2 + seed_offset, torch.float32, device)


# ---------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands on a bounded sample of the workload
# ---------------------------------------------------------------------------------
def cpu_baseline(X_gpu, slab=96, repeats=1):
    """Oracle R-STHOSVD on the slab X[:, :, :slab] (same generator, same ranks and p)."""
    from oracle import tucker

    n0, n1 = DIMS[0], DIMS[1]
    sub = X_gpu[: n0 * n1 * slab].double().cpu().numpy()
    Xs = np.reshape(sub, (n0, n1, slab), order="F")
    ranks = [RANKS[0], RANKS[1], min(RANKS[2], slab - P)]
    rho = RHO
    t0 = time.perf_counter()
    for _ in range(repeats):
        tucker.rsthosvd(Xs, ranks, P, SEED, rho=rho)
    dt = (time.perf_counter() - t0) / repeats
    fl = algorithmic_flops([n0, n1, slab], ranks, P, rho)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    return {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"oracle R-STHOSVD (numpy FP64, BLAS on all host cores) on the {n0}x{n1}x{slab} slab "
                      f"X[:, :, :{slab}] of the same tensor, ranks {ranks}, p={P}; {dt:.2f} s per run"}, dt


# ---------------------------------------------------------------------------------
# plain FP64 GPU comparator (PyTorch FP64 matmul / QR / SVD on the device)
# ---------------------------------------------------------------------------------
def _unfold_rev(torch, T, n):
    """Kolda mode-n unfolding of a tensor stored with reversed axes (axis d-1-k holds mode k)."""
    d = T.dim()
    a = d - 1 - n
    perm = [a] + [x for x in range(d) if x != a]      # remaining modes from the highest down
    return T.permute(perm).reshape(T.shape[a], -1), perm


def _fold_rev(torch, Mt, perm, shape_rev):
    tmp = Mt.reshape([shape_rev[perm[0]]] + [shape_rev[x] for x in perm[1:]])
    inv = [0] * len(perm)
    for i, q in enumerate(perm):
        inv[q] = i
    return tmp.permute(inv).contiguous()


def fp64_gpu_rsthosvd(torch, rh, X64, dims, ranks, p, seed, rho, tensor_id=0, clamp=False):
    """Alg. 3 in plain PyTorch FP64 on the device (matmul, linalg.qr, linalg.svd);
    Omega columns from the library's stream, so both runs use the same test matrices."""
    d = len(dims)
    G = X64.reshape(list(reversed(dims)))
    factors = [None] * d
    for n in rho:
        Gm, perm = _unfold_rev(torch, G, n)
        I, M = Gm.shape
        ell = ranks[n] + p
        if clamp:
            ell = min(ell, I, M)
        Om = rh.omega(seed, tensor_id, n, 0, M, ell).double().T      # M x ell
        Q, _ = torch.linalg.qr(Gm @ Om)
        B = Q.T @ Gm
        Ub, s, Vt = torch.linalg.svd(B, full_matrices=False)
        r = min(ranks[n], ell)
        factors[n] = Q @ Ub[:, :r]
        shape_rev = list(G.shape)
        shape_rev[d - 1 - n] = r
        G = _fold_rev(torch, s[:r, None] * Vt[:r], perm, shape_rev)
    return factors, G


# ---------------------------------------------------------------------------------
def run_ours(args):
    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    from paper_1905_07311_gb300 import build

    if local == 0:          # one build per node; the other ranks wait for it at the barrier
        build.build()
    if world > 1:
        dist.barrier()
    import paper_1905_07311_gb300 as rh
    from paper_1905_07311_gb300 import _lib

    L = _lib.lib()
    if world > 1:
        return run_sharded(args, torch, dist, world, rank, local, device, rh, L)
    X = make_input(torch, device, seed_offset=rank)
    tc = args.form in ("f32_bf16x2", "f32_bf16x3")
    form = args.form if tc else torch.float32
    call = rh.RsthosvdCall(DIMS, form, RANKS, p=P, seed=SEED, rho=RHO, device=device)
    for _ in range(args.warmup):
        call.run(X)
    torch.cuda.synchronize()

    stream = torch.cuda.current_stream(device)
    # ---- per-stage breakdown and the dominant kernel's launch time: a separate profiled pass ----
    kprof = max(1, min(args.steps, 3))
    L.rh_profile_enable(1)
    launches0 = L.rh_kernel_launches()
    for _ in range(kprof):
        T = call.run(X)
    torch.cuda.synchronize()
    launches = (L.rh_kernel_launches() - launches0) / kprof
    L.rh_profile_enable(0)
    cap = 100000
    kinds = (ctypes.c_int32 * cap)()
    tags = (ctypes.c_int32 * cap)()
    ms = (ctypes.c_float * cap)()
    nrec = min(L.rh_profile_collect(kinds, tags, ms, cap), cap)

    # ---- eager (stream launches) time of a step, unprofiled ----
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        T = call.run(X)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_eager = e0.elapsed_time(e1) / args.steps

    # ---- the step as the user replays it: the decomposition captured once in a CUDA graph ----
    side = torch.cuda.Stream(device=device)
    side.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        call.run(X)
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=side):
            call.run(X)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        graph.replay()
    torch.cuda.synchronize()

    # ---- timed region (device events on the launching stream) ----
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    flops = algorithmic_flops(DIMS, RANKS, P, RHO)
    ms_step, value = job_time_and_value(torch, dist if world > 1 else None, e0.elapsed_time(e1) / args.steps, flops,
                                        world, device)

    # ---- dominant kernel and its roofline ----
    per = {}
    for i in range(nrec):
        per.setdefault((kinds[i], tags[i]), []).append(ms[i])
    names = {0: "sketch", 1: "mode_product", 2: "qr", 3: "trunc_svd", 4: "core_product", 5: "jacobi"}
    breakdown = {f"{names[k]}[{t_}]": round(sum(v) / len(v), 4) for (k, t_), v in sorted(per.items())}
    dom = max([(0, 0), (1, 0)], key=lambda key: sum(per.get(key, [0.0])))
    dom_ms = sum(per[dom]) / len(per[dom])
    N = float(np.prod(DIMS))
    ell = RANKS[0] + P
    # algorithmic bytes of one launch: X read once (+ B = Q^T X_(1) written by the mode product)
    dom_bytes = N * 4 + (N / DIMS[0]) * ell * 4 * (dom[0] == 1)
    dom_flops = 2.0 * N * ell
    peaks, src = measured_peaks()
    sm_mhz = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    hbm_gbs = dom_bytes / (dom_ms * 1e-3) / 1e9
    if tc:
        kname = "sketch_tc_kernel<FP32 in>" if dom[0] == 0 else "ttm_tc_kernel<FP32 in>"
        roofline = {"kernel": kname, "bound": "hbm", "achieved": round(hbm_gbs, 1), "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": round(hbm_gbs / peaks["hbm_gbs"], 4),
                    "traffic": traffic_for(dom[0], tc=True),
                    "peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)" if src == "measured"
                    else "fallback 6.8 TB/s", "algorithmic_bytes": dom_bytes, "avg_launch_ms": round(dom_ms, 4)}
    else:
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12     # FFMA lanes x 2 flops x clock
        roofline = {"kernel": "sketch_kernel<float>" if dom[0] == 0 else "ttm_kernel<float>", "bound": "alu",
                    "achieved": round(dom_flops / (dom_ms * 1e-3) / 1e12, 3),
                    "peak": round(fp32_peak, 2), "unit": "TFLOP/s",
                    "frac": round(dom_flops / (dom_ms * 1e-3) / 1e12 / fp32_peak, 4),
                    "traffic": traffic_for(dom[0]),
                    "peak_source": f"FP32 FFMA: 152 SMs x 128 lanes x 2 flops x {sm_mhz:.0f} MHz (median sampled "
                                   "SM clock)",
                    "hbm_frac_of_" + src: round(hbm_gbs / peaks["hbm_gbs"], 4), "avg_launch_ms": round(dom_ms, 4)}

    # ---- end to end through the C ABI with host buffers ----
    e2e = None
    if not args.no_e2e:
        hc = rh.RsthosvdHostCall(DIMS, form, RANKS, p=P, seed=SEED, rho=RHO, device=device)
        Xh = X.cpu().pin_memory()
        hc.run(Xh)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ke = max(1, min(args.steps, 3))
        f0.record(stream)
        for _ in range(ke):
            hc.run(Xh)
        f1.record(stream)
        torch.cuda.synchronize()
        ms_e2e, v_e2e = job_time_and_value(torch, dist if world > 1 else None, f0.elapsed_time(f1) / ke, flops,
                                           world, device)
        e2e = {"value": round(v_e2e, 3), "unit": "TFLOP/s",
               "ms_per_step": round(ms_e2e, 3), "h2d_bytes_per_step": hc.h2d_bytes,
               "d2h_bytes_per_step": hc.d2h_bytes}
        del Xh, hc

    # ---- accuracy of this run and the plain FP64 GPU comparator (rank 0, untimed for value) ----
    extra = {}
    if rank == 0 and not args.no_fp64:
        extra = fp64_comparison(torch, rh, X, T, device)
        ref = extra.get("fp64_gpu", {})
        if "ms_per_step" in ref:
            ref["speedup_of_ours"] = round(ref["ms_per_step"] / ms_step, 2)
            ref["error_ratio_ours_over_fp64"] = round(extra["rel_error"] / ref["rel_error"], 6)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu, _ = cpu_baseline(X, slab=args.cpu_slab)

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "time_to_tucker_ms": round(ms_step, 4),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"f32_bf16x2": "bf16x2", "f32_bf16x3": "bf16x3"}.get(args.form, "f32"),
                "form": {"f32_bf16x2": "FP32 X split on the fly into BF16 head + tail (16 significant bits) in every "
                                       "tensor-core sketch, mode product and core product, Omega in BF16, FP32 "
                                       "accumulation",
                         "f32_bf16x3": "FP32 X split on the fly exactly into three BF16 pieces (24 significant "
                                       "bits) in every tensor-core sketch, mode product and core product, Omega in "
                                       "BF16, FP32 accumulation"}.get(args.form, "FP32 on the CUDA cores"),
                "data": "synthetic (seeded generator, inputs resident in HBM before timing)",
                "config": {"workload": WORKLOAD, "dims": DIMS, "ranks": RANKS, "p": P, "seed": SEED,
                           "order": [n + 1 for n in RHO], "parallelism": f"independent tensor per GPU x{world}",
                           "l2": f"input ({np.prod(DIMS) * 4 / 1e9:.2f} GB) larger than L2 (129 MB); no flush",
                           "graph": True},
                "roofline": roofline, "e2e": e2e, "gpu_launches": int(round(launches * args.steps)), "clocks": clk,
                "cpu_baseline": cpu, "breakdown_ms": breakdown,
                "timing": "CUDA-graph replay of the whole decomposition (captured once; every kernel runs each "
                          "step); eager stream launches: " + f"{ms_eager:.4f} ms per step; breakdown and "
                          "the dominant kernel's launch time from a separate profiled eager pass"}
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_sharded(args, torch, dist, world, rank, local, device, rh, L):
    """N > 1: one R-STHOSVD of the global tensor 1024 x 1024 x (1024 N), cut along its last mode into
    one 1024^3 slab per GPU (this rank's slab is the benchmark construction with seed 2 + rank): the
    slab partition of Alg. 3 with NCCL all-reduces of the sketches and the last mode's partial
    products and all-gathers of the tall-skinny triangles and the last mode's row blocks.  Weak
    scaling: the work per GPU is one 1024^3 slab; value = the global algorithmic flops / the slowest
    rank's time."""
    from paper_1905_07311_gb300 import slab

    X = make_input(torch, device, seed_offset=rank)
    gdims = DIMS[:-1] + [DIMS[-1] * world]
    k0 = DIMS[-1] * rank
    slabs = [slab.Slab(k0, k0 + DIMS[-1], X)]
    comm = slab.TorchComm()
    be = slab.LibraryBackend(args.form)
    # the ranks' agreement on the problem and their slab tiling are checked once, in the first warm-up
    # call (a small all-gather); the timed calls repeat the same call without it
    def run(validate=False):
        return slab.rsthosvd_slabs(slabs, gdims, RANKS, p=P, seed=SEED, comm=comm, backend=be, validate=validate)

    for i in range(args.warmup):
        run(validate=i == 0)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(device)
    n0 = L.rh_kernel_launches()
    clocks = Clocks(local)
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        res = run()
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    launches = (L.rh_kernel_launches() - n0) / args.steps
    flops = algorithmic_flops(gdims, RANKS, P, list(range(len(gdims))))
    ms_step, value = job_time_and_value(torch, dist, e0.elapsed_time(e1) / args.steps, flops / world, world, device)
    nx = float(res.norm_x2.item())
    ng = float((res.core.double() ** 2).sum().item())
    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16x2" if args.form == "f32_bf16x2" else "f32",
                "data": "synthetic (seeded generator, inputs resident in HBM before timing)",
                "config": {"workload": f"dense 3-way FP32 {gdims[0]}x{gdims[1]}x{gdims[2]} cut into {world} slabs of "
                                       "1024^3 along the last mode; R-STHOSVD rank (50,50,50), p=10",
                           "dims": gdims, "ranks": RANKS, "p": P, "seed": SEED,
                           "parallelism": f"slab partition along the last mode x{world} (NCCL all-reduce / all-gather)",
                           "l2": "input larger than L2; no flush"},
                "rel_error_from_norms": max(nx - ng, 0.0) ** 0.5 / nx ** 0.5,
                "gpu_launches": int(round(launches * args.steps)), "clocks": clk, "e2e": None, "cpu_baseline": None}
        print(json.dumps(line))
    dist.barrier()
    dist.destroy_process_group()


def traffic_for(kind, tc=False):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current kernel source
    (the kernel's .cu file, and for the tensor-core kernels also the shared tc.cuh)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    import hashlib

    want = {0: "sketch", 1: "ttm"}[kind] + ("_tc" if tc else "")
    csrc = os.path.join(ROOT, "paper_1905_07311_gb300", "csrc")
    blob = open(os.path.join(csrc, f"{want}.cu"), "rb").read()
    if tc:
        blob += open(os.path.join(csrc, "tc.cuh"), "rb").read()
    h = hashlib.sha256(blob).hexdigest()[:16]
    with open(path) as f:
        for line in f:
            t = line.split()
            if len(t) >= 3 and t[0] == want and t[1] == h:
                return float(t[2])
    return None


def fp64_comparison(torch, rh, X, T, device):
    """Relative errors of this run and of a plain PyTorch FP64 R-STHOSVD, plus its time."""
    try:
        X64 = X.double()
        A = [f.T.contiguous() for f in T.factors]   # I_n x r_n
        core = T.core.reshape(list(reversed(T.core_dims)))
        nx = torch.linalg.vector_norm(X64)
        e_ours = float(torch.linalg.vector_norm(X64 - _reconstruct(torch, core, A)) / nx)
        for _ in range(1):
            fp64_gpu_rsthosvd(torch, rh, X64, DIMS, RANKS, P, SEED, RHO)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fac, G = fp64_gpu_rsthosvd(torch, rh, X64, DIMS, RANKS, P, SEED, RHO)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b)
        e_ref = float(torch.linalg.vector_norm(X64 - _reconstruct(torch, G, fac)) / nx)
        del X64
        return {"rel_error": e_ours, "fp64_gpu": {"ms_per_step": round(ms, 3), "rel_error": e_ref,
                                                  "what": "plain PyTorch FP64 (matmul, linalg.qr, linalg.svd) Alg. 3 "
                                                          "on the same device and Omega stream",
                                                  "speedup_of_ours": None}}
    except Exception as exc:  # comparator is informational
        return {"fp64_gpu": {"error": repr(exc)}}


def _reconstruct(torch, core_rev, factors):
    """X_hat = G x_1 A_1 ... x_d A_d for tensors stored with reversed axes (C order)."""
    T = core_rev
    d = len(factors)
    for n in range(d):
        ax = d - 1 - n
        T = torch.movedim(torch.tensordot(factors[n], T, dims=([1], [ax])), 0, ax)
    return T.reshape(-1)


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return
    import torch

    device = "cuda" if torch.cuda.is_available() else "cpu"
    X = make_input(torch, device)
    times = []
    info = None
    for i in range(args.warmup + args.steps):
        cpu, dt = cpu_baseline(X, slab=args.cpu_slab)
        if i >= args.warmup:
            times.append(dt)
            info = cpu
    dt = sum(times) / len(times)
    n0, n1 = DIMS[0], DIMS[1]
    fl = algorithmic_flops([n0, n1, args.cpu_slab], [RANKS[0], RANKS[1], min(RANKS[2], args.cpu_slab - P)], P, RHO)
    value = fl / dt / 1e12
    info["value"] = round(value, 6)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "dims": DIMS, "ranks": RANKS, "p": P,
                                            "sample": f"slab {n0}x{n1}x{args.cpu_slab}"},
            "cpu_baseline": info,
            "e2e": {"value": round(value, 6), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------
# Further workloads (--workload): the configurations the tests check for parity, measured with the
# same rules (inputs resident, CUDA events on the launching stream, clocks sampled, warm-up).
# ---------------------------------------------------------------------------------
NAMES = {0: "sketch", 1: "mode_product", 2: "qr", 3: "trunc_svd", 4: "core_product", 5: "jacobi", 6: "power_step",
         7: "sp_omega_table", 8: "sp_sort", 9: "sp_items", 10: "sp_row_reduce"}


def _timed(torch, L, fn, steps, warmup, device, profile=True):
    """Device timing of ``steps`` calls of fn after ``warmup`` (profiling off); returns (ms per call,
    {stage: ms per call} from a separate profiled pass when ``profile``, launches per call, clocks)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    clocks = Clocks(device.index or 0)
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = L.rh_kernel_launches()
    clocks.start()
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = (L.rh_kernel_launches() - n0) / steps
    per = {}
    kp = max(1, min(steps, 3))
    if profile:
        L.rh_profile_enable(1)
        for _ in range(kp):
            fn()
        torch.cuda.synchronize()
        L.rh_profile_enable(0)
        cap = 200000
        kinds, tags, ms = (ctypes.c_int32 * cap)(), (ctypes.c_int32 * cap)(), (ctypes.c_float * cap)()
        nrec = min(L.rh_profile_collect(kinds, tags, ms, cap), cap)
        for i in range(nrec):
            per.setdefault(f"{NAMES.get(kinds[i], kinds[i])}[{tags[i]}]", []).append(ms[i])
    breakdown = {k: round(sum(v) / kp, 4) for k, v in sorted(per.items())}
    return e0.elapsed_time(e1) / steps, breakdown, launches, clk


def _cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()


def _hbm_roof(kernel, nbytes, ms, peaks, src):
    gbs = nbytes / (ms * 1e-3) / 1e9
    return {"kernel": kernel, "bound": "hbm", "achieved": round(gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": None,
            "peak_source": f"{src} HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs)", "algorithmic_bytes": nbytes,
            "avg_launch_ms": round(ms, 4)}


def _fp64_matmul_tflops(torch, device, n=4096, reps=3):
    """FP64 dense matmul rate (TFLOP/s) of this GPU: the best of ``reps`` timed torch.matmul calls
    of n x n operands after one warm-up call, CUDA events on the current stream."""
    a = torch.randn(n, n, dtype=torch.float64, device=device)
    b = torch.randn(n, n, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        torch.matmul(a, b)
        e1.record(stream)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def wl_hilbert200(torch, rh, L, args, device, peaks, src):
    """200^3 FP64 tensor 1/(i+j+k+1), rank (20, 20, 20), p = 5, seed 0, order 1, 2, 3."""
    from workloads import hilbert

    dims, ranks = [200, 200, 200], [20, 20, 20]
    Xn = hilbert(dims, offset=1)
    X = torch.from_numpy(np.ascontiguousarray(Xn.ravel(order="F"))).to(device)
    call = rh.RsthosvdCall(dims, torch.float64, ranks, p=5, seed=0, rho=[0, 1, 2], device=device)
    ms, br, launches, clk = _timed(torch, L, lambda: call.run(X), args.steps, args.warmup, device)
    T = call.run(X)
    G = torch.from_numpy(np.reshape(T.core.cpu().numpy(), T.core_dims, order="F"))
    A = [f.cpu().double().T for f in T.factors]
    Xh = G
    for n in range(3):
        Xh = torch.movedim(torch.tensordot(A[n], Xh, dims=([1], [n])), 0, n)
    Xt = torch.from_numpy(Xn)
    err = float(torch.linalg.vector_norm(Xt - Xh) / torch.linalg.vector_norm(Xt))
    # the first-mode sketch on the CUDA cores is FP64-FMA bound: 2 N ell flops against the FP64
    # rate measured here (a 4096^3 FP64 matmul; the part's nominal rate is 1.25 TFLOP/s)
    sk = br.get("sketch[0]", ms)
    fl = 2.0 * 200 ** 3 * 25
    fp64 = _fp64_matmul_tflops(torch, device)
    roof = {"kernel": "sketch_kernel<double>", "bound": "alu", "achieved": round(fl / (sk * 1e-3) / 1e12, 4),
            "peak": round(fp64, 3), "unit": "TFLOP/s", "frac": round(fl / (sk * 1e-3) / 1e12 / fp64, 4),
            "traffic": None, "peak_source": "FP64 matmul measured in this run (torch.matmul 4096^3, best of 3)",
            "algorithmic_flops": fl, "avg_launch_ms": sk}
    cpu = None
    if not args.no_cpu:
        from oracle import tucker

        t0 = time.perf_counter()
        out = tucker.rsthosvd(Xn, ranks, 5, 0, rho=[0, 1, 2])
        dt = time.perf_counter() - t0
        Gd, Ad = tucker.sthosvd(Xn, ranks, rho=[0, 1, 2])
        from oracle.tensor import rel_error

        cpu = {"value": round(dt * 1e3, 3), "unit": "ms", "cores": _cores(), "kind": "oracle",
               "sample": "oracle R-STHOSVD (numpy FP64) on the whole 200^3 tensor",
               "oracle_rel_error": rel_error(Xn, out["core"], out["factors"]),
               "sthosvd_rel_error": rel_error(Xn, Gd, Ad)}
    return {"metric": "R-STHOSVD time-to-Tucker, 200^3 Hilbert-type FP64, rank 20", "value": round(ms, 4),
            "unit": "ms", "higher_is_better": False, "dtype": "f64", "rel_error": err,
            "config": {"workload": "dense 3-way FP64 200x200x200, X(i,j,k) = 1/(i+j+k+1), rank (20,20,20), p=5, "
                                   "seed 0, order 1,2,3", "l2": "input 64 MB (fits L2); no flush"},
            "roofline": roof, "breakdown_ms": br, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu}


def wl_lowp192(torch, rh, L, args, device, peaks, src):
    """192^4 with a 30^4 core (decay 0.8), noise 1e-3, stored in BF16 and E4M3 (block scales);
    R-STHOSVD rank 30, p = 10; adaptive Alg. 5 at 1e-2 (block 8, p = 10) on the BF16 storage."""
    from workloads import fp8_quantize_torch, lowrank_plus_noise_torch

    dims, ranks = [192] * 4, [30] * 4
    X = lowrank_plus_noise_torch(dims, ranks, 0.8, 1e-3, 3, torch.float32, device)
    N = X.numel()
    stored = {"fp8_e4m3": fp8_quantize_torch(X, dims), "bf16": X.to(torch.bfloat16).view(torch.int16),
              "f32_bf16x2": X}
    nbytes = {"fp8_e4m3": stored["fp8_e4m3"].numel(), "bf16": 2 * N, "f32_bf16x2": 4 * N}
    forms = {}
    for form, Xs in stored.items():
        call = rh.RsthosvdCall(dims, form, ranks, p=10, seed=0, device=device)
        ms, br, launches, clk = _timed(torch, L, lambda: call.run(Xs), args.steps, args.warmup, device)
        sk = br.get("sketch[0]", ms)
        forms[form] = {"ms": round(ms, 4), "sketch0_GBs": round(nbytes[form] / (sk * 1e-3) / 1e9, 1),
                       "breakdown_ms": br, "gpu_launches": launches, "clocks": clk,
                       "info": call.info.cpu().numpy().tolist()}
    # adaptive on the BF16 storage
    Xb = stored["bf16"]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    rh.adaptive(Xb, dims, 1e-2, variant="sthosvd", block=8, p=10, seed=0, form="bf16")
    torch.cuda.synchronize()
    t0.record()
    Ta = rh.adaptive(Xb, dims, 1e-2, variant="sthosvd", block=8, p=10, seed=0, form="bf16")
    t1.record()
    torch.cuda.synchronize()
    adapt = {"ms": round(t0.elapsed_time(t1), 3), "ranks": Ta.ranks, "eps": 1e-2,
             "note": "synchronous call (one host read of the sizes per mode)"}
    f8 = forms["fp8_e4m3"]
    roof = _hbm_roof("sketch_tc_kernel<E4M3 in>", nbytes["fp8_e4m3"], f8["breakdown_ms"].get("sketch[0]"), peaks,
                     src)
    cpu = None
    if not args.no_cpu:
        from oracle import tucker

        sub = X.view(192, 192, 192, 192)[:8].contiguous().view(-1)   # X[:, :, :, :8] in column-major terms
        Xs = np.reshape(sub.double().cpu().numpy(), [192, 192, 192, 8], order="F")
        t = time.perf_counter()
        tucker.rsthosvd(Xs, [30, 30, 30, 8], 10, 0, clamp=True)
        dt = time.perf_counter() - t
        cpu = {"value": round(dt * 1e3, 1), "unit": "ms", "cores": _cores(), "kind": "oracle",
               "sample": "oracle R-STHOSVD (numpy FP64) on the 192x192x192x8 slab X[:, :, :, :8] (1/24 of the "
                         "tensor), ranks (30, 30, 30, 8), p = 10, ell clamped to the slab"}
    return {"metric": "R-STHOSVD time-to-Tucker, 192^4 stored in BF16 (E4M3 and FP32 forms alongside)",
            "value": forms["bf16"]["ms"], "unit": "ms", "higher_is_better": False, "dtype": "bf16",
            "config": {"workload": "dense 4-way 192^4, core 30^4 decay 0.8, noise 1e-3, seed 3; rank (30,30,30,30), "
                                   "p=10; storage BF16 / E4M3 with per-128-byte FP32 scales / FP32 split on the fly",
                       "l2": "inputs 1.4-5.4 GB (larger than L2); no flush"},
            "forms": forms, "adaptive_bf16": adapt, "roofline": roof, "cpu_baseline": cpu}


def _batch_errors(torch, Ts, X64s):
    """Relative Tucker error ||X - G x_1 A_1 ... x_d A_d|| / ||X|| of every tensor (FP64 on the device)."""
    out = []
    for T, X in zip(Ts, X64s):
        A = [f.T.contiguous() for f in T.factors]
        core = T.core.reshape(list(reversed(T.core_dims)))
        nx = torch.linalg.vector_norm(X)
        out.append(float(torch.linalg.vector_norm(X - _reconstruct(torch, core, A).reshape(-1)) / nx))
    return out


def _graph_timed(torch, L, step, args, device):
    """CUDA-graph capture of ``step`` on a side stream, replayed ``steps`` times after ``warmup``."""
    step()
    torch.cuda.synchronize()
    s = torch.cuda.Stream(device=device)
    s.wait_stream(torch.cuda.current_stream(device))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        step()
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=s):
            step()
    ms, _, _, clk = _timed(torch, L, g.replay, args.steps, args.warmup, device, profile=False)
    n0 = L.rh_kernel_launches()
    step()
    torch.cuda.synchronize()
    return ms, clk, L.rh_kernel_launches() - n0, g


def wl_batched(torch, rh, L, args, device, peaks, src):
    """The batched workload's order-3 and order-4 tensors (339 of 512, 8.0 GB FP32).  Grouped engine
    (--streams 0): a batched plan (each tensor's launches recorded once, one grouped launch per stage)
    whose run is captured in a CUDA graph and replayed; stream engine (--streams N): one
    rsthosvd_batched call captured and replayed.  --batch-form: f32 (FP32 on the CUDA cores),
    f32_bf16x2 (FP32 split into BF16 head + tail on the fly) or bf16 (BF16 storage); the BF16 forms
    process mode 0 first, on the small-row tensor-core kernels.  Unless --no-fp64: the same batch as
    FP64 data on the library's FP64 path (grouped, graph-replayed) and as a plain PyTorch FP64 loop
    (matmul, linalg.qr, linalg.svd per tensor, same Omega), the relative errors of all three against
    the FP32 tensors, and for the bf16 form the smallest oversampling p (from 5 up) whose errors are
    all within 1.02 x the FP64 ones."""
    from workloads import batch_recipe, lowrank_plus_noise_torch

    orders = tuple(int(v) for v in args.batch_orders.split(","))
    rec = [b for b in batch_recipe() if len(b[0]) in orders]
    if args.batch_count > 0:
        rec = rec[:args.batch_count]
    if 5 in orders:
        return wl_batched_waves(torch, rh, L, args, device, peaks, src, orders)
    form = args.batch_form
    rho = "natural" if form != "f32" else None
    Xs = [lowrank_plus_noise_torch(d, r, 0.9, 1e-3, sd, torch.float32, device) for d, r, sd in rec]
    nel = sum(x.numel() for x in Xs)
    if form == "bf16":
        Xin = [x.to(torch.bfloat16).view(torch.int16) for x in Xs]   # ties to even
        esize, dt = 2, "bf16"
    else:
        Xin = Xs
        esize, dt = 4, ("f32_bf16x2" if form == "f32_bf16x2" else torch.float32)
    dims_list = [b[0] for b in rec]
    ranks_list = [b[1] for b in rec]
    nbytes = esize * nel

    def run_form(p):
        call = rh.RsthosvdBatchedCall(dims_list, ranks_list, dt, p=p, seed=4, clamp=True, streams=args.streams,
                                      device=device, rho=rho)
        plan = call.plan(Xin) if args.streams == 0 else None
        step = plan.run if plan is not None else (lambda: call.run(Xin))
        return call, plan, step

    fp64 = None
    e64 = None
    if not args.no_fp64:
        X64s = [x.double() for x in Xs]
        c64 = rh.RsthosvdBatchedCall(dims_list, ranks_list, torch.float64, p=5, seed=4, clamp=True, streams=0,
                                     device=device, rho=rho)
        pl64 = c64.plan(X64s)
        ms64, clk64, _, g64 = _graph_timed(torch, L, pl64.run, args, device)
        e64 = _batch_errors(torch, pl64.run(), X64s)
        torch.cuda.synchronize()
        del g64
        pl64.close()
        # plain PyTorch FP64, one tensor after another (same Omega stream and tensor ids)
        rr = list(range(max(orders)))
        for i in range(min(3, len(rec))):
            fp64_gpu_rsthosvd(torch, rh, X64s[i], dims_list[i], ranks_list[i], 5, 4,
                              rr[:len(dims_list[i])] if rho else _default_rho(dims_list[i]), tensor_id=i, clamp=True)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        tout = []
        for i in range(len(rec)):
            tout.append(fp64_gpu_rsthosvd(torch, rh, X64s[i], dims_list[i], ranks_list[i], 5, 4,
                                          rr[:len(dims_list[i])] if rho else _default_rho(dims_list[i]),
                                          tensor_id=i, clamp=True))
        b.record()
        torch.cuda.synchronize()
        ms_t = a.elapsed_time(b)
        et = []
        for (fac, G), X in zip(tout, X64s):
            nx = torch.linalg.vector_norm(X)
            et.append(float(torch.linalg.vector_norm(X - _reconstruct(torch, G, fac).reshape(-1)) / nx))
        del tout
        fp64 = {"library_fp64_grouped": {"ms_per_step": round(ms64, 3), "mean_rel_error": float(np.mean(e64)),
                                         "max_rel_error": float(np.max(e64))},
                "torch_fp64_loop": {"ms_per_step": round(ms_t, 3), "mean_rel_error": float(np.mean(et)),
                                    "max_rel_error": float(np.max(et)),
                                    "what": "plain PyTorch FP64 (matmul, linalg.qr, linalg.svd) Alg. 3 per tensor on "
                                            "the same device, Omega stream and processing order"}}
    p_used, search = 5, []
    if form == "bf16" and e64 is not None and not args.no_psearch:
        for pp in (5, 6, 7, 8, 10, 12, 16):
            call, plan, step = run_form(pp)
            Ts = step()
            torch.cuda.synchronize()
            eb = _batch_errors(torch, Ts, X64s)
            worst = max(x / y for x, y in zip(eb, e64))
            search.append({"p": pp, "max_error_ratio_vs_fp64": round(worst, 5)})
            if plan is not None:
                plan.close()
            del call, plan, step
            if worst <= 1.02:
                p_used = pp
                break
    call, plan, step = run_form(p_used)
    ms, clk, launches, g = _graph_timed(torch, L, step, args, device)
    Ts = step()
    torch.cuda.synchronize()
    tps = len(Xs) / (ms * 1e-3)
    res_err = None
    if e64 is not None:
        eo = _batch_errors(torch, Ts, X64s)
        ratios = [x / y for x, y in zip(eo, e64)]
        res_err = {"mean_rel_error": float(np.mean(eo)), "max_rel_error": float(np.max(eo)),
                   "max_error_ratio_vs_fp64": round(max(ratios), 5), "mean_error_ratio_vs_fp64": round(
                       float(np.mean(ratios)), 5)}
        fp64["speedup_vs_library_fp64"] = round(fp64["library_fp64_grouped"]["ms_per_step"] / ms, 2)
        fp64["speedup_vs_torch_fp64"] = round(fp64["torch_fp64_loop"]["ms_per_step"] / ms, 2)
        fp64["equal_error"] = max(ratios) <= 1.02
        del X64s
    # roofline of the whole call: each tensor is read twice (sketch and mode product of its first mode)
    roof = _hbm_roof("rsthosvd_batched (whole call)", 2 * nbytes, ms, peaks, src)
    cpu = None
    if not args.no_cpu:
        from oracle import tucker

        t = time.perf_counter()
        for (d, r, _), X in list(zip(rec, Xs))[:6]:
            Xn = np.reshape(X.double().cpu().numpy(), d, order="F")
            tucker.rsthosvd(Xn, r, 5, 4, clamp=True)
        dt_ = time.perf_counter() - t
        cpu = {"value": round(6 / dt_, 3), "unit": "tensors/s", "cores": _cores(), "kind": "oracle",
               "sample": "oracle R-STHOSVD (numpy FP64) of the first 6 tensors of the same set"}
    names = {"f32": "FP32 on the CUDA cores", "f32_bf16x2": "FP32 split into BF16 head + tail on the fly, first mode "
             "on the small-row tensor-core kernels", "bf16": "BF16 storage, first mode on the small-row tensor-core "
             "kernels"}
    out = {"metric": "batched R-STHOSVD throughput (order-3 and order-4 tensors of the batch)",
           "value": round(tps, 1), "unit": "tensors/s", "higher_is_better": True,
           "dtype": {"f32": "f32", "f32_bf16x2": "bf16x2", "bf16": "bf16"}[form], "form": names[form],
           "ms_per_step": round(ms, 3),
           "config": {"workload": f"{len(Xs)} tensors, order {args.batch_orders}, sizes U[16,96], ranks U[4,16] capped, "
                                  "low rank + "
                                  f"1e-3 noise, seed 4, p={p_used} clamped; {nbytes / 1e9:.2f} GB "
                                  f"{'BF16' if form == 'bf16' else 'FP32'}",
                      "processing_order": "mode 0 first (natural)" if rho else "decreasing sizes",
                      "engine": "grouped (batched plan)" if args.streams == 0 else f"{args.streams} streams",
                      "graph": True, "l2": f"inputs {nbytes / 1e9:.1f} GB (larger than L2); no flush"},
           "roofline": roof, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu}
    if res_err is not None:
        out["errors"] = res_err
        out["fp64_gpu"] = fp64
    if search:
        out["p_search"] = search
    if plan is not None:
        plan.close()
    return out


def _default_rho(dims):
    """The library's default processing order: decreasing sizes, ties to the lower mode."""
    return sorted(range(len(dims)), key=lambda k: (-dims[k], k))


def wl_batched_waves(torch, rh, L, args, device, peaks, src, orders):
    """The batched workload with its order-5 tensors (all 512: 438.6 GB FP32, more than HBM): tensors
    in recipe order are packed into waves whose data and workspace stay below --wave-gb; each wave
    is generated on the device (untimed), recorded as a batched plan (tensor i keeps tensor_id = its
    index in the recipe, as in one call over the whole batch) and timed like the other workloads;
    the batch time is the sum of the wave times."""
    from workloads import batch_recipe, lowrank_plus_noise_torch
    from paper_1905_07311_gb300 import i32_array, i64_array, make_options

    allrec = batch_recipe()
    idx = [i for i, b in enumerate(allrec) if len(b[0]) in orders]
    if args.batch_count > 0:
        idx = idx[:args.batch_count]
    opts = make_options(seed=4, p=5, clamp=True)
    need = []
    for i in idx:
        d, r, _ = allrec[i]
        ws = L.rsthosvd_workspace_size(len(d), i64_array(d), 1, i32_array(r), ctypes.byref(opts))
        need.append(4 * int(np.prod(d)) + int(ws) + 4096)
    limit = args.wave_gb * 1e9
    waves, cur, acc = [], [], 0
    for i, nb in zip(idx, need):
        # a wave is a run of consecutive recipe tensors, so tensor_id = first index + position
        if cur and (acc + nb > limit or i != cur[-1] + 1):
            waves.append(cur)
            cur, acc = [], 0
        cur.append(i)
        acc += nb
    if cur:
        waves.append(cur)
    total_ms, nbytes, launches, clks = 0.0, 0, 0, []
    for wv in waves:
        Xs = [lowrank_plus_noise_torch(allrec[i][0], allrec[i][1], 0.9, 1e-3, allrec[i][2], torch.float32, device)
              for i in wv]
        torch.cuda.synchronize()
        call = rh.RsthosvdBatchedCall([allrec[i][0] for i in wv], [allrec[i][1] for i in wv], torch.float32, p=5,
                                      seed=4, tensor_id=wv[0], clamp=True, streams=0, device=device)
        plan = call.plan(Xs)
        ms, _, nl, clk = _timed(torch, L, plan.run, args.steps, args.warmup, device, profile=False)
        total_ms += ms
        nbytes += sum(4 * x.numel() for x in Xs)
        launches += int(nl)
        clks.append(clk)
        plan.close()
        del plan, call, Xs
        torch.cuda.empty_cache()
    tps = len(idx) / (total_ms * 1e-3)
    roof = _hbm_roof("rsthosvd_batched (all waves)", 2 * nbytes, total_ms, peaks, src)
    clk = {"sm_mhz": min(c["sm_mhz"] for c in clks if c.get("sm_mhz") is not None) if any(
               c.get("sm_mhz") is not None for c in clks) else None,
           "sm_max_mhz": clks[0].get("sm_max_mhz"),
           "reasons": sorted({r for c in clks for r in c.get("reasons", [])}),
           "samples": sum(c.get("samples", 0) for c in clks)}
    cpu = None
    if not args.no_cpu:
        from oracle import tucker

        small = [i for i in idx if len(allrec[i][0]) <= 4][:6]
        dt = 0.0
        for i in small:
            d, r, sd = allrec[i]
            X = lowrank_plus_noise_torch(d, r, 0.9, 1e-3, sd, torch.float32, device)
            Xn = np.reshape(X.double().cpu().numpy(), d, order="F")
            t0 = time.perf_counter()
            tucker.rsthosvd(Xn, r, 5, 4, tensor_id=i, clamp=True)
            dt += time.perf_counter() - t0
        cpu = {"value": round(len(small) / dt, 3), "unit": "tensors/s", "cores": _cores(), "kind": "oracle",
               "sample": "oracle R-STHOSVD (numpy FP64) of the first 6 order-3/4 tensors of the set (the order-5 "
                         "ones are GBs each)"}
    return {"metric": "batched R-STHOSVD throughput (all tensors of the batch, in waves)",
            "value": round(tps, 1), "unit": "tensors/s", "higher_is_better": True, "dtype": "f32",
            "ms_per_step": round(total_ms, 3),
            "config": {"workload": f"{len(idx)} tensors, order {args.batch_orders}, sizes U[16,96], ranks U[4,16] "
                                   f"capped, low rank + 1e-3 noise, seed 4, p=5 clamped; {nbytes / 1e9:.1f} GB FP32 "
                                   f"in {len(waves)} waves of <= {args.wave_gb:g} GB (data + workspace), each "
                                   "generated on the device outside the timed region",
                       "engine": "grouped (batched plan per wave)", "graph": False,
                       "l2": "inputs far larger than L2; no flush"},
            "roofline": roof, "gpu_launches": launches, "clocks": clk, "cpu_baseline": cpu,
            "waves": len(waves)}


def wl_sparse(torch, rh, L, args, device, peaks, src):
    """COO 20000 x 20000 x 5000 with 5e7 nonzeros (Zipf 1.1, log-count values), SP-STHOSVD rank 30,
    p = 10, with FP32 Omega and with Omega rounded to BF16 (the two forms of the sparse sketch), and
    SP-HOSVD.  The sketch is not HBM- or tensor-bound: each distinct Omega row (a distinct pair of
    other-mode coordinates) is generated once, so its roof is max(COO bytes / HBM, distinct rows x ell
    normals / the measured rate of the library's Omega generator)."""
    from workloads import zipf_coo_torch

    dims, nnz = [20000, 20000, 5000], 50_000_000
    idx, vals = zipf_coo_torch(dims, nnz, 1.1, 3.0, 5, device)
    torch.cuda.synchronize()
    forms = {}
    for om in ("f32", "bf16"):
        ms, _, launches, clk = _timed(torch, L, lambda: rh.sp_sthosvd_coo(idx, vals, dims, [30] * 3, p=10, seed=0,
                                                                           omega=om),
                                      args.steps, args.warmup, device, profile=False)
        ms_sk, br_sk, _, _ = _timed(torch, L, lambda: rh.rhosvd_sketch_coo(idx, vals, dims, 0, 40, seed=0, omega=om),
                                    args.steps, args.warmup, device, profile=True)
        forms[om] = {"sp_sthosvd_ms": round(ms, 3), "sketch_mode1_ms": round(ms_sk, 4), "launches": launches,
                     "clocks": clk, "sketch_breakdown_ms": br_sk}
    ms_ho, _, _, _ = _timed(torch, L, lambda: rh.sp_hosvd_coo(idx, vals, dims, [30] * 3, p=10, seed=0),
                            args.steps, args.warmup, device, profile=False)
    # Omega generator rate (normals per second) on a long stream
    rows = 1 << 24
    out = torch.empty((40, rows), dtype=torch.float32, device=device)
    o_ms, _, _, _ = _timed(torch, L, lambda: L.rh_omega(0, 0, 0, 0, rows, 40, ctypes.c_void_p(out.data_ptr()),
                                                        ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)),
                           args.steps, args.warmup, device, profile=False)
    del out
    rate = 40.0 * rows / (o_ms * 1e-3)
    # distinct Omega rows of mode 1: distinct (i_2, i_3) pairs
    distinct = int(torch.unique(idx[1].long() + dims[1] * idx[2].long()).numel())
    sk_bytes = nnz * 16.0
    t_roof = max(sk_bytes / (peaks["hbm_gbs"] * 1e9), distinct * 40.0 / rate) * 1e3
    ms_sk = forms["f32"]["sketch_mode1_ms"]
    roof = {"kernel": "rhosvd_sketch_coo (mode 1, ell 40, FP32 Omega)", "bound": "alu",
            "achieved": round(t_roof / ms_sk, 4), "peak": 1.0,
            "unit": "fraction of max(COO bytes / HBM, distinct Omega rows x ell / Omega rate)",
            "frac": round(t_roof / ms_sk, 4), "traffic": None,
            "peak_source": f"Omega generator measured at {rate / 1e9:.1f} G normals/s (rh_omega, 2^24 x 40), "
                           f"HBM {peaks['hbm_gbs']} GB/s ({src})",
            "distinct_rows_mode1": distinct, "roof_ms": round(t_roof, 4), "avg_launch_ms": ms_sk}
    cpu = None
    if not args.no_cpu:
        from oracle import tucker

        m = 1_000_000
        sub = np.stack([t[:m].cpu().numpy().astype(np.int64) for t in idx], axis=1)
        v = vals[:m].double().cpu().numpy()
        t = time.perf_counter()
        tucker.coo_sketch(sub, v, dims, 0, 40, 0)
        dt = time.perf_counter() - t
        cpu = {"value": round(m / dt / 1e6, 3), "unit": "M nonzeros/s (sketch, ell 40)", "cores": _cores(),
               "kind": "oracle", "sample": "oracle COO sketch of the first 1e6 nonzeros, mode 1, ell 40"}
    return {"metric": "SP-STHOSVD time-to-Tucker, COO 20000x20000x5000, 5e7 nonzeros",
            "value": forms["f32"]["sp_sthosvd_ms"], "unit": "ms", "higher_is_better": False, "dtype": "f32",
            "sketch_mode1_ms": ms_sk, "forms": forms, "sp_hosvd_ms": round(ms_ho, 3),
            "config": {"workload": "COO 20000x20000x5000, 5e7 distinct Zipf(1.1) coordinates, values "
                                   "log(1+Poisson(3)+1), seed 5; rank (30,30,30), p=10", "l2": "800 MB of COO; no flush"},
            "roofline": roof, "gpu_launches": forms["f32"]["launches"], "clocks": forms["f32"]["clocks"],
            "cpu_baseline": cpu}


def _dense1024_error(torch, rh, X, T):
    """Relative Tucker error by direct residual (FP64 reconstruction on the device)."""
    A = [f.T.contiguous() for f in T.factors]
    core = T.core.reshape(list(reversed(T.core_dims)))
    X64 = X.double()
    e = float(torch.linalg.vector_norm(X64 - _reconstruct(torch, core, A)) / torch.linalg.vector_norm(X64))
    del X64
    return e


def wl_power1024(torch, rh, L, args, device, peaks, src):
    """The benchmark tensor (1024^3 FP32, rank 50, p = 10, form f32_bf16x2) with q = 0, 1, 2 steps of
    randomized subspace iteration in every range finder (Sec. 5 "Variants", Sec. 6): time-to-Tucker,
    relative error, and the cost of a step.  A step is a mode product (tensor cores), the basis of
    range(B^T) (tall-skinny QR + CholeskyQR), a sketch against that dense basis (CUDA cores, the
    same head + tail split of X) and a QR."""
    X = make_input(torch, device)
    out = {}
    for q in (0, 1, 2):
        call = rh.RsthosvdCall(DIMS, "f32_bf16x2", RANKS, p=P, seed=SEED, rho=RHO, device=device, power_iters=q)
        ms, br, launches, clk = _timed(torch, L, lambda: call.run(X), args.steps, args.warmup, device)
        T = call.run(X)
        torch.cuda.synchronize()
        out[f"q{q}"] = {"ms": round(ms, 3), "rel_error": _dense1024_error(torch, rh, X, T),
                        "launches": launches, "clocks": clk, "breakdown_ms": br}
        del call
    return {"metric": "R-STHOSVD time-to-Tucker with subspace iteration, 1024^3 FP32 rank 50 p 10",
            "value": out["q1"]["ms"], "unit": "ms", "higher_is_better": False, "dtype": "bf16x2",
            "power_iters": out, "config": {"workload": WORKLOAD, "form": "f32_bf16x2"}}


def wl_rhosvd1024(torch, rh, L, args, device, peaks, src):
    """R-HOSVD (Alg. 2) of the benchmark tensor (1024^3 FP32, rank 50, p = 10): every mode sketched
    on the input, then the core chain.  Algorithmic bytes: X read once per mode's sketch and mode
    product and once more for the core chain's first product."""
    X = make_input(torch, device)
    N = float(np.prod(DIMS))
    nbytes = N * 4 * 7            # three sketches, three mode products, the core chain's first product
    forms = {}
    for form in ("f32_bf16x2", "f32"):
        call = rh.RhosvdCall(DIMS, form if form != "f32" else torch.float32, RANKS, p=P, seed=SEED, device=device)
        ms, br, launches, clk = _timed(torch, L, lambda: call.run(X), args.steps, args.warmup, device)
        T = call.run(X)
        torch.cuda.synchronize()
        forms[form] = {"ms": round(ms, 3), "rel_error": _dense1024_error(torch, rh, X, T), "breakdown_ms": br,
                       "launches": launches, "clocks": clk, "tc_modes": [int(v) for v in T.info.cpu().tolist()]}
        del call
    ms = forms["f32_bf16x2"]["ms"]
    return {"metric": "R-HOSVD time-to-Tucker, 1024^3 FP32 rank 50 p 10", "value": ms, "unit": "ms",
            "higher_is_better": False, "dtype": "bf16x2", "rel_error": forms["f32_bf16x2"]["rel_error"],
            "forms": forms, "gpu_launches": forms["f32_bf16x2"]["launches"], "clocks": forms["f32_bf16x2"]["clocks"],
            "roofline": _hbm_roof("R-HOSVD (whole call: 7 passes over X)", nbytes, ms, peaks, src),
            "config": {"workload": WORKLOAD.replace("R-STHOSVD", "R-HOSVD"),
                       "form": "f32_bf16x2: every mode's sketch and mode product and the core chain's products on "
                               "the tensor cores over the on-the-fly BF16 split of X"}}


def wl_outofcore(torch, rh, L, args, device, peaks, src):
    """Out-of-core R-STHOSVD: a 1024 x 1024 x 2048 FP32 tensor (8.6 GB, the benchmark's construction)
    held in pinned host memory and streamed to the device in slabs of 128 last-mode planes (512 MB)
    -- twice, for the first mode's sketch and its mode product; after the first mode the truncated
    core (50 x 1024 x 2048) stays on the device.  The first mode runs on the tensor cores (BF16 head +
    tail split on the fly).  Its roof is the host link: 2 x 8.6 GB / the measured host-to-device copy
    bandwidth.  The relative error comes from ||X||^2 - ||G||^2 (orthonormal factors, Alg. 3)."""
    from paper_1905_07311_gb300 import slab

    dims = [1024, 1024, 2048]
    Xr = lowrank_plus_noise_torch_host(torch, dims, device)      # axes reversed: Xr[i_3, i_2, i_1]
    bounds = slab.even_slabs(dims[-1], dims[-1] // 128)
    # a slab X[:, :, k0:k1] is the contiguous block Xr[k0:k1], column-major in (i_1, i_2, i_3 - k0)
    slabs = [slab.Slab(k0, k1, Xr[k0:k1].reshape(-1).pin_memory(), device=device) for k0, k1 in bounds]
    del Xr
    be = slab.LibraryBackend("f32_bf16x2")
    run = lambda: slab.rsthosvd_slabs(slabs, dims, RANKS, p=P, seed=SEED, backend=be)   # noqa: E731
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(device.index or 0)
    clocks.start()
    e0.record(stream)
    for _ in range(args.steps):
        res = run()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    nx = float(res.norm_x2.item())
    ng = float((res.core.double() ** 2).sum().item())
    err = max(nx - ng, 0.0) ** 0.5 / nx ** 0.5
    # host link: one slab's pinned copy, timed alone
    buf = torch.empty(slabs[0].data.numel(), dtype=torch.float32, device=device)
    h2d = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        buf.copy_(slabs[0].data, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        h2d.append(slabs[0].data.numel() * 4 / (a.elapsed_time(b) * 1e-3) / 1e9)
    gbs = max(h2d)
    nbytes = float(np.prod(dims)) * 4
    roof_ms = 2 * nbytes / (gbs * 1e9) * 1e3
    return {"metric": "out-of-core R-STHOSVD time-to-Tucker, 1024x1024x2048 FP32 streamed from host memory",
            "value": round(ms, 3), "unit": "ms", "higher_is_better": False, "dtype": "bf16x2",
            "rel_error_from_norms": err, "clocks": clk,
            "roofline": {"kernel": "whole call (host link)", "bound": "host link", "achieved": round(2 * nbytes / (ms * 1e-3) / 1e9, 1),
                         "peak": round(gbs, 1), "unit": "GB/s", "frac": round(roof_ms / ms, 4), "traffic": None,
                         "peak_source": "measured pinned host-to-device copy of one 512 MB slab (best of 5)",
                         "roof_ms": round(roof_ms, 3)},
            "config": {"workload": "dense 3-way FP32 1024x1024x2048 (low rank 50^3, decay 0.9, 1e-3 noise) in pinned "
                                   "host memory, 16 slabs of 1024x1024x128; R-STHOSVD rank (50,50,50), p=10",
                       "device_resident_x": False}}


def lowrank_plus_noise_torch_host(torch, dims, device):
    """The benchmark construction at ``dims`` (generated on the device), in host memory as the tensor
    with reversed axes whose C-order buffer is the column-major flat tensor."""
    from workloads import lowrank_plus_noise_torch

    X = lowrank_plus_noise_torch(dims, [50] * len(dims), 0.9, 1e-3, 2, torch.float32, device)
    out = X.reshape(list(reversed(dims))).cpu()
    del X
    return out


def wl_peaks(torch, rh, L, args, device, peaks, src):
    """Rates the rooflines of the non-BF16 paths need, measured on this device: dense matmul in FP64,
    TF32 and FP32 (torch.matmul, 8192^3 for TF32 / FP32, 4096^3 for FP64: 2 n^3 flops, best of the
    timed steps) and the Omega generator (rh_omega: Philox4x32-10 + Box-Muller normals per second,
    2^24 rows x 64 columns per launch; the 4 GB it writes take ~0.6 ms of its time at HBM speed)."""
    out = {}
    steps = max(3, args.steps)

    def best_ms(fn, reps):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        best = float("inf")
        stream = torch.cuda.current_stream(device)
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    clocks = Clocks(device.index or 0)
    clocks.start()
    prev = torch.backends.cuda.matmul.allow_tf32
    for name, dt, n, tf32 in (("fp64", torch.float64, 4096, False), ("tf32", torch.float32, 8192, True),
                              ("fp32", torch.float32, 8192, False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        a = torch.randn(n, n, dtype=dt, device=device)
        b = torch.randn(n, n, dtype=dt, device=device)
        ms = best_ms(lambda: torch.matmul(a, b), steps)
        out[f"{name}_matmul_tflops"] = round(2.0 * n ** 3 / (ms * 1e-3) / 1e12, 2)
        del a, b
    torch.backends.cuda.matmul.allow_tf32 = prev
    nrows, ell = 1 << 24, 64
    om = torch.empty((ell, nrows), dtype=torch.float32, device=device)
    st = ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)
    ms = best_ms(lambda: rh._lib.check(L.rh_omega(0, 0, 0, 0, nrows, ell, ctypes.c_void_p(om.data_ptr()), st)), steps)
    out["omega_normals_per_s"] = round(nrows * ell / (ms * 1e-3), -6)
    out["omega_ms"] = round(ms, 4)
    out["clocks"] = clocks.stop()
    out["how"] = wl_peaks.__doc__.split("\n\n")[0].replace("\n", " ")
    return out


def run_workload(args):
    import torch

    torch.cuda.set_device(0)
    device = torch.device("cuda", 0)
    from paper_1905_07311_gb300 import build

    build.build()
    import paper_1905_07311_gb300 as rh
    from paper_1905_07311_gb300 import _lib

    L = _lib.lib()
    peaks, src = measured_peaks()
    fn = {"hilbert200": wl_hilbert200, "lowp192": wl_lowp192, "batched": wl_batched, "sparse": wl_sparse,
          "peaks": wl_peaks, "power1024": wl_power1024, "rhosvd1024": wl_rhosvd1024,
          "outofcore": wl_outofcore}[args.workload]
    line = {"workload": args.workload, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic"}
    line.update(fn(torch, rh, L, args, device, peaks, src))
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-slab", type=int, default=None,
                    help="mode-3 extent of the CPU sample (default 384 for the baseline, 128 per reference step)")
    ap.add_argument("--form", default="f32_bf16x2", choices=["f32_bf16x2", "f32_bf16x3", "f32"],
                    help="f32_bf16x2: tensor cores over the on-the-fly BF16 head + tail split of X (default); "
                         "f32_bf16x3: the exact three-piece split; f32: CUDA-core FP32 throughout")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--dims", type=int, nargs=3, default=None,
                    help="smaller cube for profiling captures (default 1024 1024 1024)")
    ap.add_argument("--workload", default="dense1024",
                    choices=["dense1024", "hilbert200", "lowp192", "batched", "sparse", "peaks", "power1024",
                             "rhosvd1024", "outofcore"],
                    help="dense1024: the benchmark line (default); the others measure the further configurations "
                         "and print one JSON line each")
    ap.add_argument("--batch-orders", default="3,4",
                    help="batched workload: tensor orders taken from the 512-tensor recipe (comma list)")
    ap.add_argument("--wave-gb", type=float, default=120.0,
                    help="batched workload with order-5 tensors: data + workspace per wave (GB)")
    ap.add_argument("--batch-form", default="f32", choices=["f32", "f32_bf16x2", "bf16"],
                    help="batched workload: input form (f32 on the CUDA cores; the BF16 forms take mode 0 first)")
    ap.add_argument("--no-psearch", action="store_true",
                    help="batched bf16 form: keep p = 5 (no search for the p that reaches the FP64 error)")
    ap.add_argument("--batch-count", type=int, default=0,
                    help="batched workload: first N tensors of those orders (0 = all)")
    ap.add_argument("--streams", type=int, default=0,
                    help="batched workload: 0 = grouped engine (one launch per stage for the batch), "
                         "N >= 1 = N internal streams")
    args = ap.parse_args()
    if args.workload != "dense1024":
        run_workload(args)
        return
    if args.dims:
        global DIMS, WORKLOAD
        DIMS = list(args.dims)
        WORKLOAD = WORKLOAD.replace("1024x1024x1024", "x".join(str(v) for v in DIMS))
    if args.impl == "reference":
        args.cpu_slab = args.cpu_slab or 128
        run_reference(args)
    else:
        args.cpu_slab = args.cpu_slab or 384
        run_ours(args)


if __name__ == "__main__":
    main()
