"""Launch-shape tuner of the small-tensor kernels (needs a GB300).

The knobs of ``csrc/tuning_table.inc`` set how many CTAs the small-row sketches and mode products
(CUDA-core and tensor-core forms) and the Gram matrix of B spread one tensor's work over.  This
module times the batched R-STHOSVD workload (the order-3 and order-4 tensors of the 512-tensor
recipe: sizes U[16, 96], ranks U[4, 16], p = 5, clamped) in two forms: FP32 on the CUDA cores
(decreasing-size processing order) and FP32 split into BF16 head + tail with mode 0 first (the
small-row tensor-core kernels).  Each form runs as a grouped batched plan replayed from a CUDA graph.
The Gram knob also shapes the dense 1024^3 R-STHOSVD (rank 50, p = 10), which is timed as a third
objective while that knob moves.

Coordinate descent: for each knob in turn, every candidate value is planned, captured and timed
(median of ``reps`` replays after 3 warm-up replays, CUDA events on the replay stream); the knob
keeps the value with the lowest sum over the objectives it affects of time / time at the current
table, and moves only when that sum drops by more than ``--min-gain``.  Passes repeat until a pass
changes nothing (at most ``--passes``).  The result is written back to ``csrc/tuning_table.inc``
(``--out``) and one JSON line per evaluation goes to stdout.

Single calls and batched calls use the same table, so that a batched call's results equal those of
single calls bit for bit.  The tuner therefore also reports, without optimising it, the latency of
single calls on small tensors (the first 24 tensors of the batch, FP32, one call after another in
one graph) at the starting and at the chosen table.

    python -m paper_1905_07311_gb300.tune [--passes 2] [--reps 10] [--count 0] [--no-dense] [--out PATH]
"""

import argparse
import json
import os
import statistics
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TABLE = os.path.join(HERE, "csrc", "tuning_table.inc")

CANDIDATES = {
    "ctas_per_sm": [1, 2, 3, 4, 6, 8, 12, 16],
    "min": [1, 2, 4, 8, 16, 32, 64, 128, 256],
}


def _candidates(name):
    return CANDIDATES["ctas_per_sm"] if name.endswith("ctas_per_sm") else CANDIDATES["min"]


def read_table(path=TABLE):
    """[(key, name, value)] in the file's order."""
    import re

    with open(path) as f:
        text = f.read()
    return [(k, n, int(v)) for k, n, v in re.findall(r'RH_TUNE\((\w+),\s*"([\w.]+)",\s*(\d+)\)', text)]


def write_table(rows, values, path=TABLE, note=""):
    lines = [
        "// Launch-shape knobs of the small-tensor kernels: RH_TUNE(key, name, value).",
        "// Written by `python -m paper_1905_07311_gb300.tune` (coordinate descent over measured times of",
        "// the batched R-STHOSVD workload and, for the Gram knob, the dense 1024^3 one).",
    ]
    if note:
        lines.append("// " + note)
    for k, n, _ in rows:
        lines.append(f'RH_TUNE({k}, "{n}", {values[n]})')
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


class Objective:
    """One timed workload: plan it under the current knobs, capture it, return ms per replay."""

    def __init__(self, name, make, reps):
        self.name, self.make, self.reps = name, make, reps

    def time(self):
        import torch

        close, step = self.make()
        try:
            step()
            torch.cuda.synchronize()
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(s):
                step()
                torch.cuda.synchronize()
                with torch.cuda.graph(g, stream=s):
                    step()
                for _ in range(3):
                    g.replay()
                torch.cuda.synchronize()
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(self.reps + 1)]
                ev[0].record(s)
                for i in range(self.reps):
                    g.replay()
                    ev[i + 1].record(s)
                torch.cuda.synchronize()
            del g
            return statistics.median(ev[i].elapsed_time(ev[i + 1]) for i in range(self.reps))
        finally:
            close()


def _objectives(args, device):
    import torch

    import paper_1905_07311_gb300 as rh

    sys.path.insert(0, ROOT)
    from workloads import batch_recipe, lowrank_plus_noise_torch

    rec = [b for b in batch_recipe() if len(b[0]) in (3, 4)]
    if args.count > 0:
        rec = rec[:args.count]
    Xs = [lowrank_plus_noise_torch(d, r, 0.9, 1e-3, sd, torch.float32, device) for d, r, sd in rec]
    dims_list = [b[0] for b in rec]
    ranks_list = [b[1] for b in rec]

    def batched(dt, rho):
        def make():
            call = rh.RsthosvdBatchedCall(dims_list, ranks_list, dt, p=5, seed=4, clamp=True, streams=0,
                                          device=device, rho=rho)
            plan = call.plan(Xs)
            return plan.close, plan.run
        return make

    def singles():
        calls = [rh.RsthosvdCall(d, torch.float32, r, p=5, seed=4, tensor_id=i, clamp=True, device=device)
                 for i, (d, r) in enumerate(zip(dims_list[:24], ranks_list[:24]))]

        def step():
            for c, X in zip(calls, Xs[:24]):
                c.run(X)
        return (lambda: None), step

    report = {"single_calls_f32_24": Objective("single_calls_f32_24", singles, args.reps)}
    objs = {"batched_f32": Objective("batched_f32", batched(torch.float32, None), args.reps),
            "batched_f32_bf16x2": Objective("batched_f32_bf16x2", batched("f32_bf16x2", "natural"), args.reps)}
    if not args.no_dense:
        dims = [1024, 1024, 1024]
        Xd = lowrank_plus_noise_torch(dims, [50, 50, 50], 0.9, 1e-3, 0, torch.float32, device)

        def dense():
            call = rh.RsthosvdCall(dims, "f32_bf16x2", [50, 50, 50], p=10, seed=0, rho=[0, 1, 2], device=device)
            return (lambda: None), (lambda: call.run(Xd))

        objs["dense_1024"] = Objective("dense_1024", dense, args.reps)
    return objs, report, len(Xs)


def _affects(name, objs):
    """Which objectives a knob can change: the Gram knob shapes every workload; the small-row knobs
    only the batched forms."""
    return [o for o in objs if name.startswith("gram") or o.startswith("batched")]


def coordinate_descent(rows, values, objectives, measure, apply, passes, min_gain, log=lambda rec: None):
    """Tune the knobs of ``rows`` one after another, in the table's order; return the chosen values.

    ``measure(names)`` returns {objective: ms} under the knobs as currently applied, and
    ``apply(name, value)`` sets one knob.  A candidate scores sum over the objectives the knob
    affects of ms / ms at the knob's current value, so the current value scores len(affected).  The
    knob moves to the best-scoring candidate only if that score is below len(affected) - min_gain,
    and it is applied again either way.  Passes repeat until one moves no knob, at most ``passes``.
    """
    values = dict(values)
    for it in range(passes):
        moved = False
        for _, name, _ in rows:
            on = _affects(name, objectives)
            ref = measure(on)
            best_v, best_s = values[name], float(len(on))
            for v in _candidates(name):
                if v == values[name]:
                    continue
                apply(name, v)
                ms = measure(on)
                score = sum(ms[o] / ref[o] for o in on)
                log({"pass": it, "knob": name, "value": v, "score": round(score / len(on), 4),
                     "ms": {k: round(x, 4) for k, x in ms.items()}})
                if score < best_s:
                    best_v, best_s = v, score
            if best_v != values[name] and best_s < len(on) - min_gain:
                values[name] = best_v
                moved = True
            apply(name, values[name])
            log({"pass": it, "knob": name, "chosen": values[name]})
        if not moved:
            break
    return values


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--passes", type=int, default=2)
    ap.add_argument("--reps", type=int, default=10)
    ap.add_argument("--count", type=int, default=0, help="first N tensors of the batch (0 = all 339)")
    ap.add_argument("--min-gain", type=float, default=0.003,
                    help="gain a move needs (in units of one objective's time)")
    ap.add_argument("--no-dense", action="store_true", help="leave the dense 1024^3 objective out")
    ap.add_argument("--out", default=TABLE)
    args = ap.parse_args(argv)

    import torch

    from . import _lib
    from . import build

    if not torch.cuda.is_available():
        raise SystemExit("the tuner times kernels: it needs a CUDA device")
    build.build()
    L = _lib.lib()
    device = torch.device("cuda", 0)
    rows = read_table()
    for _, n, v in rows:
        _lib.check(L.rh_tuning_set(n.encode(), v))
    values = {n: v for _, n, v in rows}
    objs, report, ntens = _objectives(args, device)
    t0 = time.time()

    def measure(names):
        return {o: objs[o].time() for o in names}

    base = measure(list(objs))
    base.update({k: o.time() for k, o in report.items()})
    print(json.dumps({"table": values, "ms": {k: round(v, 4) for k, v in base.items()}, "tensors": ntens}),
          flush=True)

    def apply(name, v):
        _lib.check(L.rh_tuning_set(name.encode(), v))

    def log(rec):
        print(json.dumps(rec), flush=True)

    values = coordinate_descent(rows, values, list(objs), measure, apply, args.passes, args.min_gain, log)
    final = measure(list(objs))
    final.update({k: o.time() for k, o in report.items()})
    print(json.dumps({"table": values, "ms": {k: round(v, 4) for k, v in final.items()},
                      "ms_at_start": {k: round(v, 4) for k, v in base.items()},
                      "seconds": round(time.time() - t0, 1)}), flush=True)
    write_table(rows, values, args.out)


if __name__ == "__main__":
    main()
