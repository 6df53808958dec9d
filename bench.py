"""Throughput of the GB300 machine code: leaf nodes per second for one forward plus
one adjoint volume-potential apply on the adaptive 20-Gaussian workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|split]
                    [--impl ours|reference]

Workload: root [-1,1]^2, p = 16, density = 20 Gaussians (centres U[-0.5,0.5]^2,
widths log-uniform in [1e-3, 1e-1], amplitudes N(0,1), seed 1), quadtree
refined by the library (Alg. 2 resolution criterion, eps = 1e-11) and 2:1
balanced.  A step is one forward apply u = A f and one adjoint apply
h = A^T g of the whole tree; value = leaf nodes / (time of a step).
With --gpus N every rank runs its own replica (the path does not shard; no
collective on the data path) and value is the total over ranks.
--impl reference times the CPU FP64 oracle (direct quadrature) on a bounded
sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "adaptive 20-Gaussian quadtree (widths 1e-3..1e-1), p=16, eps=1e-11"
METRIC = "leaf nodes/sec (p=16, <=1e-10 rel err) fwd+adjoint"
UNIT = "leaf nodes/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="split", choices=["fp64", "split"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--workload", default="adaptive20", choices=list(WORKLOADS),
                    help="adaptive20: the benchmark workload; adaptive200: 200 Gaussians, widths 1e-4..1e-1")
    ap.add_argument("--nterms", type=int, default=24,
                    help="far-field expansion terms P+1: 24 keeps the truncation near 1e-12, inside the "
                         "1e-10 target of the metric (30 reaches FP64 rounding)")
    ap.add_argument("--no-overlap", dest="overlap", action="store_false",
                    help="run the near-field tensor launch in line instead of beside the far-field passes "
                         "(the library's default, on an internal stream)")
    ap.add_argument("--profile-run", action="store_true",
                    help="only the warm-up and timed steps of the chosen precision (for profiler captures)")
    return ap.parse_args()


WORKLOADS = {
    "adaptive20": (2, "adaptive 20-Gaussian quadtree (widths 1e-3..1e-1), p=16, eps=1e-11"),
    "adaptive200": (3, "adaptive 200-Gaussian quadtree (widths 1e-4..1e-1), p=16, eps=1e-11"),
    "batch64": (None, "64 adaptive trees (about 2e2..2e4 leaves, log-uniform), p in {8,12,16}, batched"),
}


def density(workload="adaptive20"):
    from paper_2501_17967_gb300 import synth
    return synth.config_density(WORKLOADS[workload][0])


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for name, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- oracle arm
def oracle_rate(tree_leaves, fvals, seconds, seed=11):
    """Oracle forward throughput (target nodes/s) on sampled leaves, bounded in time.
    The oracle's transposed operator costs the same per entry, so a fwd+adjoint
    step is twice the forward cost."""
    import oracle
    from paper_2501_17967_gb300 import synth
    lv, ix, iy = tree_leaves
    p = 16
    geom = synth.leaf_geometry(lv, ix, iy)
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(lv))
    done, t_used, vals = 0, 0.0, {}
    k = 1
    while t_used < seconds and done < len(order):
        ids = order[done:done + k]
        t0 = time.perf_counter()
        u = oracle.potential_at_nodes(p, geom, fvals, leaf_ids=ids)
        t_used += time.perf_counter() - t0
        for i, b in enumerate(ids):
            vals[int(b)] = u[i]
        done += len(ids)
        k = min(2 * k, 64)
    nodes = done * p * p
    return nodes / t_used / 2.0, nodes, t_used, vals


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import paper_2501_17967_gb300 as bc
    import oracle
    from paper_2501_17967_gb300 import synth
    g = density(args.workload)
    hctx = bc.Context(p=16, device=-1, cache_dir=None, build_tables=False)
    tree = bc.Tree.refine(hctx, g, eps=1e-11, max_level=18)
    leaves = tree.leaves()
    geom = synth.leaf_geometry(*leaves)
    fvals = g(oracle.leaf_nodes(geom, 16)).reshape(-1, 16, 16)
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        oracle_rate(leaves, fvals, per_step / 4)
    rates, nodes_tot, t_tot = [], 0, 0.0
    for s in range(args.steps):
        r, n, t, _ = oracle_rate(leaves, fvals, per_step, seed=100 + s)
        rates.append(r)
        nodes_tot += n
        t_tot += t
    value = nodes_tot / t_tot / 2.0
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload][1], "nleaf": int(tree.nleaf), "leaf_nodes": int(tree.nleaf) * 256,
                       "parallelism": "host threads"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{nodes_tot} target nodes of randomly sampled leaves over {args.steps} steps "
                                       f"(~{per_step:.0f}s each), forward oracle rate halved for fwd+adjoint"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
STAGES = ("tensor_v", "clear", "upward", "m2l", "down_levels", "tensor_e", "leaf_output", "tensor_near")


STAGE_KERNELS = {
    "tensor_v": "k_split_vec + k_split_gemm<256> (leaf-to-expansion; X list and near field too with --no-overlap)",
    "clear": "k_clear_flags",
    "upward": "k_up_levels",
    "m2l": "k_split_exp + k_split_gemm<64> (M2L per V pair; FP64 path: k_m2l_pairs + k_x_entries)",
    "down_levels": "k_down_levels",
    "tensor_e": "k_split_exp + k_split_gemm<64>",
    "leaf_output": "k_leaf_out",
    "tensor_near": "k_split_gemm<256> (X list, then near field, on the internal stream beside stages 1-4)",
}
# ncu dram__bytes_read.sum + dram__bytes_write.sum of each stage's tensor or
# pass kernel (cold cache; tensor_near: its X-list and near-field launches
# together), keyed by (workload, nterms, split): the launch list of the bench
# configuration (profiles/launches_adaptive20_split.md)
TRAFFIC = {
    ("adaptive20", 24, True): {"tensor_v": 3.59e6, "tensor_near": 29.24e6, "upward": 0.57e6, "m2l": 2.95e6,
                               "down_levels": 13.68e6, "tensor_e": 5.27e6, "leaf_output": 32.39e6},
}


def stage_work(st, nleaf, nleaf_far, P1, NP, split):
    """Algorithmic work of each stage of one apply, counted from the tree's lists:
    (amount, kind) with kind "tensor" (BF16 flops of the 15 digit products,
    rows x K x columns of the real operators), "fp64" (FP64 flops: complex x
    real = 4 per term, complex x complex = 8) or "bytes" (leaf output of the
    split path: FP64 partial results read + result written)."""
    n_shift = st["n_down"]
    R = 2 * P1
    if split:
        return {
            "tensor_v": (15 * 2.0 * NP * R * (nleaf + st["n_x"]), "tensor"),
            "tensor_near": (15 * 2.0 * NP * NP * st["n_near"], "tensor"),
            "clear": (0.0, "fp64"),
            "upward": (32.0 * P1 * P1 * st["n_nonleaf"], "fp64"),
            "m2l": (15 * 2.0 * R * R * st["n_v"], "tensor"),
            "down_levels": (8.0 * P1 * P1 * n_shift + 2.0 * P1 * (st["n_v"] + st["n_x"]), "fp64"),
            "tensor_e": (15 * 2.0 * R * NP * (nleaf_far + st["n_w"]), "tensor"),
            "leaf_output": (8.0 * NP * (st["n_near"] + st["n_w"] + nleaf_far + nleaf), "bytes"),
        }
    return {
        "tensor_v": (0.0, "tensor"),
        "tensor_near": (0.0, "tensor"),
        "clear": (0.0, "fp64"),
        "upward": (4.0 * P1 * NP * nleaf + 32.0 * P1 * P1 * st["n_nonleaf"], "fp64"),
        "m2l": (4.0 * P1 * P1 * st["n_v"] + 4.0 * P1 * NP * st["n_x"], "fp64"),
        "down_levels": (8.0 * P1 * P1 * n_shift + 2.0 * P1 * (st["n_v"] + st["n_x"]), "fp64"),
        "tensor_e": (0.0, "tensor"),
        "leaf_output": (2.0 * NP * NP * st["n_near"] + 4.0 * P1 * NP * (nleaf_far + st["n_w"]), "fp64"),
    }


def run_batch64(args):
    """64 independent Gaussian-sum densities on their own adaptive trees, p in
    {8, 12, 16} round-robin; one batch (union of trees, CUDA graph, autotuned
    launch shapes) per order.  A step = forward + adjoint of all 64."""
    import torch

    import paper_2501_17967_gb300 as bc
    from paper_2501_17967_gb300 import synth
    dev = torch.cuda.current_device()
    ctxs = {p: bc.Context(p=p, nterms=args.nterms, device=dev) for p in (8, 12, 16)}
    groups = {8: [], 12: [], 16: []}
    t0 = time.perf_counter()
    for k in range(64):
        g, p, eps = synth.batch_density(k)
        tree = bc.Tree.refine(ctxs[p], g, eps=eps, max_level=16)
        groups[p].append((tree, torch.from_numpy(g(tree.nodes())).to(dev)))
    t_tree = time.perf_counter() - t0
    batches = {p: bc.Batch(ctxs[p], [t for t, _ in groups[p]]) for p in groups}
    prec = {p: (bc.SPLIT_BF16 if (p in bc.SPLIT_ORDERS and args.precision == "split") else bc.FP64) for p in groups}
    outs = {p: [torch.empty_like(f) for _, f in groups[p]] for p in groups}
    adjs = {p: [torch.empty_like(f) for _, f in groups[p]] for p in groups}
    for p in groups:
        batches[p].autotune(prec[p])
    stream = torch.cuda.current_stream()

    def step():
        for p in groups:
            ins = [f for _, f in groups[p]]
            batches[p].run(ins, outs[p], precision=prec[p], stream=stream)
            batches[p].run(outs[p], adjs[p], precision=prec[p], adjoint=True, stream=stream)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    nodes = sum(t.nleaf * p * p for p in groups for t, _ in groups[p])
    leaves = [t.nleaf for p in groups for t, _ in groups[p]]
    line = {"metric": METRIC + " (batched)", "value": nodes / (ms * 1e-3), "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 (p=8,12) / bf16 digits + f64 (p=16)" if args.precision == "split" else "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOADS["batch64"][1], "trees": 64, "leaves_min": min(leaves),
                       "leaves_max": max(leaves), "leaves_total": sum(leaves), "leaf_nodes": nodes,
                       "tree_build_s": round(t_tree, 2),
                       "launch_shapes": {str(p): batches[p].shape(prec[p], 0) for p in groups},
                       "l2": "flushed (256 MB write) between timed steps"},
            "clocks": clocks.summary()}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch64(args)
    import torch
    import torch.distributed as dist

    import paper_2501_17967_gb300 as bc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    head = bc.FP64 if args.precision == "fp64" else bc.SPLIT_BF16

    g = density(args.workload)
    workload_name = WORKLOADS[args.workload][1]
    ctx = bc.Context(p=16, nterms=args.nterms, device=dev)
    ctx.set_option("split_overlap", 1 if args.overlap else 0)
    P1 = ctx.nterms or 30
    t0 = time.perf_counter()
    tree = bc.Tree.refine(ctx, g, eps=1e-11, max_level=18)
    t_tree = time.perf_counter() - t0
    st = tree.stats()
    N = tree.nleaf * 256
    fvals = g(tree.nodes()).reshape(-1, 16, 16)
    f = torch.from_numpy(fvals).to(dev)
    gen = torch.Generator(device=dev).manual_seed(1)
    gin = torch.randn(f.shape, generator=gen, device=dev, dtype=torch.float64)
    u = torch.empty_like(f)
    h = torch.empty_like(f)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2 (129 MB)
    stream = torch.cuda.current_stream()

    def timed(precision, steps, sampler=None):
        def step():
            bc.apply(tree, f, out=u, precision=precision, stream=stream)
            bc.apply_adjoint(tree, gin, out=h, precision=precision, stream=stream)
        for _ in range(max(3, args.warmup)):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        if sampler:
            sampler.start()
            time.sleep(0.3)
        # the timed steps run as in production: no stage events, no host reads
        for k in range(steps):
            flush.zero_()
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        if sampler:
            sampler.stop()
        if world > 1:
            dist.barrier()
        bc._check(bc._load().bc_sync(ctx.handle, None))
        total = torch.tensor([float(sum(a.elapsed_time(b) for a, b in ev))], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(total, op=dist.ReduceOp.MAX)
        # the per-stage breakdown comes from a separate pass with the library's
        # stage events on (they separate the kernels of the launch chain and
        # are read back every step, so they are kept out of the timed steps)
        stages = np.zeros((2, len(STAGES)))
        ctx.debug(timing=True)
        for k in range(steps):
            flush.zero_()
            step()
            stages[0] += ctx.stage_times(adjoint=False)
            stages[1] += ctx.stage_times(adjoint=True)
        ctx.debug(timing=False)
        bc._check(bc._load().bc_sync(ctx.handle, None))
        return float(total.item()) / steps, stages / steps

    clocks = ClockSampler(dev)
    if args.profile_run:
        ms_step, _ = timed(head, args.steps)
        if rank == 0:
            print(json.dumps({"profile_run": True, "workload": workload_name, "nleaf": int(tree.nleaf),
                              "ms_per_step": ms_step}))
        if world > 1:
            dist.destroy_process_group()
        return
    ms_step, stage_ms = timed(head, args.steps, clocks)
    value = world * N / (ms_step * 1e-3)
    other = bc.FP64 if head == bc.SPLIT_BF16 else bc.SPLIT_BF16
    ms_other, stage_other = timed(other, max(3, args.steps // 2))

    # end to end through the public API with pinned host buffers (headline precision)
    fh = f.cpu().pin_memory()
    gh = gin.cpu().pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    hh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        bc.apply(tree, fh, out=uh, precision=head)
        bc.apply_adjoint(tree, gh, out=hh, precision=head)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        bc.apply(tree, fh, out=uh, precision=head)
        bc.apply_adjoint(tree, gh, out=hh, precision=head)
    e2e_s = (time.perf_counter() - t0) / args.steps
    e2e = {"value": world * N / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 2 * N * 8,
           "d2h_bytes_per_step": 2 * N * 8}

    # rooflines per stage (per apply, averaged over forward and adjoint)
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh_:
            peaks = json.load(fh_)
    except OSError:
        pass
    fp64_peak = bc.fp64_peak_tflops(dev)
    bf16_peak = peaks.get("bf16_tflops", 1900.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    lv = tree.leaves()[0]
    wk = stage_work(st, tree.nleaf, int((lv >= 2).sum()), P1, 256, head == bc.SPLIT_BF16)
    if not args.overlap:
        # one group-V tensor launch (near field included) in stage 0
        wk["tensor_v"] = (wk["tensor_v"][0] + wk["tensor_near"][0], "tensor")
        wk["tensor_near"] = (0.0, "tensor")
    elif head == bc.SPLIT_BF16:
        # the X-list tiles run on the internal stream, before the near field
        xw = 15 * 2.0 * 256 * 2 * P1 * st["n_x"]
        wk["tensor_v"] = (wk["tensor_v"][0] - xw, "tensor")
        wk["tensor_near"] = (wk["tensor_near"][0] + xw, "tensor")
    # DRAM bytes per launch (read + write) from the ncu capture of this
    # configuration (profiles/kernels_adaptive20_split.md); null elsewhere
    traffic = TRAFFIC.get((args.workload, P1, head == bc.SPLIT_BF16), {})
    per_stage = {}
    for i, name in enumerate(STAGES):
        ms = float(stage_ms[:, i].mean())
        amount, kind = wk[name]
        if ms <= 0 or amount == 0:
            continue
        if kind == "bytes":
            ach, pk, bound, unit = amount / (ms * 1e-3) / 1e9, hbm_peak, "hbm", "GB/s"
        else:
            ach = amount / (ms * 1e-3) / 1e12
            pk, bound, unit = (bf16_peak, "tensor", "TFLOP/s") if kind == "tensor" else (fp64_peak, "alu", "TFLOP/s")
        per_stage[name] = {"ms": round(ms, 4), "kernel": STAGE_KERNELS[name], "bound": bound,
                           "achieved": round(ach, 4), "unit": unit, "peak": round(pk, 2), "frac": round(ach / pk, 4),
                           "traffic": traffic.get(name)}
    # the dominant kernel: the one with the most GPU time per apply; the two
    # launches of the group-V kernel (far tiles in stage 0, near tiles beside
    # stages 1-4) count together
    cand = dict(per_stage)
    if "tensor_v" in cand and "tensor_near" in cand:
        a, b = cand.pop("tensor_v"), cand.pop("tensor_near")
        ms_vn = a["ms"] + b["ms"]
        ach = (wk["tensor_v"][0] + wk["tensor_near"][0]) / (ms_vn * 1e-3) / 1e12
        tr = a["traffic"] + b["traffic"] if a["traffic"] is not None and b["traffic"] is not None else None
        cand["tensor_v+tensor_near"] = {
            "ms": round(ms_vn, 4), "kernel": "k_split_gemm<256> (group V: far and near launches together)",
            "bound": "tensor", "achieved": round(ach, 4), "unit": "TFLOP/s", "peak": round(bf16_peak, 2),
            "frac": round(ach / bf16_peak, 4), "traffic": tr}
    dom = max(cand, key=lambda k: cand[k]["ms"])
    d = cand[dom]
    src = {"tensor": "MEASURED_PEAKS.json bf16_tflops (burst), of measured",
           "alu": "bc_debug_fp64_peak: measured FP64 FMA throughput, of measured",
           "hbm": "MEASURED_PEAKS.json hbm_gbs, of measured"}
    roofline = {"bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
                "frac": d["frac"], "traffic": d["traffic"], "kernel": d["kernel"], "stage": dom,
                "peak_source": src[d["bound"]],
                "stages": per_stage}

    nl = st["nlevels"]
    # kernels per apply (trees of more than three levels): flag clear, upward
    # pass, M2L, downward level pass, leaf output; FP64: M2L pairs + X-list products;
    # split: input digits, group-V tensor launch (two when the near field runs apart), M2L
    # digits + tensor launch, expansion digits + group-E tensor launch
    if head == bc.SPLIT_BF16:
        launches_per_apply = 2 + (2 if args.overlap else 0) + 1 + 1 + 2 + 1 + 2 + 1
    else:
        launches_per_apply = 1 + 1 + 1 + (1 if st["n_x"] > 0 else 0) + 1 + 1
    pname = {bc.FP64: "fp64", bc.SPLIT_BF16: "split-bf16"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if head == bc.FP64 else "bf16 digits (5 slices) + f64",
            "data": "synthetic",
            "config": {"workload": workload_name, "precision": pname[head], "nleaf": int(tree.nleaf), "leaf_nodes": int(N),
                       "nlevels": nl, "nterms": P1, "tree_build_s": round(t_tree, 3),
                       "l2": "flushed (256 MB write) between timed steps", "parallelism": f"replicas x{world}"},
            "clocks": clocks.summary(), "e2e": e2e, "gpu_launches": 2 * launches_per_apply * args.steps,
            "roofline": roofline,
            "other_precision": {"precision": pname[other], "value": world * N / (ms_other * 1e-3),
                                "ms_per_step": ms_other,
                                "stage_ms": {n: round(float(stage_other[:, i].mean()), 4)
                                             for i, n in enumerate(STAGES)}}}

    if rank == 0 and not args.no_cpu_baseline:
        bc.apply(tree, f, out=u, precision=head)
        torch.cuda.synchronize()
        rate, nn, tt, vals = oracle_rate(tree.leaves(), fvals, args.cpu_seconds)
        line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{nn} target nodes ({nn // 256} random leaves) of the same tree in "
                                          f"{tt:.1f}s; forward rate halved for fwd+adjoint"}
        uu = u.cpu().numpy().reshape(-1, 256)
        got = np.stack([uu[b] for b in vals])
        ref = np.stack([vals[b] for b in vals])
        line["rel_err_vs_oracle_sample"] = float(np.abs(got - ref).max() / np.abs(ref).max())
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
