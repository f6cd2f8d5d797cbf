"""Benchmark: j2d5pt on one GB300, GCells/s (interior cell updates per second).

Headline workload (one line of JSON): FP64, 16384 x 16384 interior cells plus
the one-cell ring, seeded uniform [0,1) data and normalised weights, 1000 time
steps per benchmark step (one benchmark step = one j2d5pt_run of 1000 time
steps).  The plan is autotuned first (one-step / resident / bands / tiles over
temporal depths and tile shapes), then timed.  The other workloads (FP64
2048 x 1536, FP32 16384^2, the paper's 8592 x 8328 domain, 256 batched grids,
the 4096^2 gradient, the 3x3 box stencil j2d9pt at 16384^2) are reported
under "extras", each with the one-step
kernel beside it and its own roofline record (median of 3 repetitions).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --workload NAME   # one named run for profiling (see WORKLOADS)

Timing: CUDA events on the launching stream; L2 flushed (256 MiB write)
between benchmark steps; synchronise before and after.  The roofline uses the
library's own CUDA events around its stencil kernels (j2d5pt_kernel_time).
`e2e` times j2d5pt_run_host (host buffers; copies inside the timed region).
With --gpus N > 1 (torchrun) every rank runs its own replica (the method is
single-GPU; replicas only): value = all ranks' cell updates / max rank time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCells/s (cell-updates/s) at 1 GB300, FP64 and FP32, and % of roofline vs 1-step kernel"
WORKLOAD = "j2d5pt_f64_16384x16384_1000"
HEAD_N, HEAD_T = 16384, 1000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=12)  # ~20 s timed at 1.65 s per step
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--workload", default=None, help="run one named workload once (profiling) and exit")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


class Clocks:
    """nvidia-smi sampling (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu, self.proc = gpu_index, None
        self.path = "/tmp/j2d_clocks_%d_%d.csv" % (os.getpid(), gpu_index)

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
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
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


class L2Flush:
    def __init__(self):
        import torch
        self.buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.buf.fill_(1.0)


def kernel_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_03336_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(key):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        ent = json.load(open(path)).get(key)
    except Exception:
        return None
    if not ent or ent.get("source_hash") != kernel_hash():
        return None
    return ent.get("bytes_per_launch")


def kernel_of(algo):
    """The stencil kernel a plan's algorithm launches."""
    return {"onestep": "onestep_kernel", "stream": "stream_kernel"}.get(algo, "dtb_kernel")


def algo_of(plan):
    return plan.describe().split("algo=")[1].split()[0]


def timed(plan, fn, steps, warmup, flush, stream):
    """Per-step event times (ms) of fn() and the library's kernel times (ms)."""
    import torch
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    total, kern = [], []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        total.append(e0.elapsed_time(e1))
        kern.append(plan.kernel_time() if plan.get("timing") else None)
    torch.cuda.synchronize()
    return total, kern


def gcells(cells, ms):
    return cells / (ms * 1e-3) / 1e9


def aggregate(total_ms, cells_per_rank, world, device="cuda"):
    """Whole-job throughput of `world` replicas: the slowest rank's time
    (MAX all-reduce) against the cell updates of all ranks.  Returns
    (max_ms, GCells/s)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return total_ms, cells_per_rank * world / (total_ms * 1e-3) / 1e9


# ---- peaks and roofline records ---------------------------------------------

def measure_peaks(j2d5pt):
    """Roofline denominators measured live on this GPU (and the driver's HBM copy figure)."""
    fma64 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F64)
    fma32 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F32)
    exact = j2d5pt.j2d5pt_measure_exact_rate()
    smem = j2d5pt.j2d5pt_measure_smem_bandwidth()
    mask, _ = j2d5pt.j2d5pt_arith_info()
    f = bin(mask & 0xFF).count("1") / 8.0
    # FP64 cell rate: half of the cells (the exact mask) run on the integer
    # pipes, the rest as 5 FP64 FMA instructions; the two pipes work in
    # parallel, so the peak is set by the slower share, each at its measured rate
    chain = fma64 / 5
    alu = 1.0 / max((1.0 - f) / chain, f / exact if f else 0.0)
    hbm = None
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] * 1e9
    except Exception:
        pass
    return {"fma64": fma64, "fma32": fma32, "exact": exact, "smem": smem, "share": f, "alu_cells": alu,
            "hbm": hbm}


def roof_f64(pk, kernel_gcells, traffic=None, kernel="dtb_kernel"):
    """FP64: arithmetic bound (FP64 pipe plus the integer path), 9 flops per cell update."""
    achieved = kernel_gcells * 9 / 1e3
    peak = pk["alu_cells"] / 1e9 * 9 / 1e3
    return {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": traffic, "kernel": kernel,
            "peak_source": ("of measured: FP64 pipe %.1f GFMA/s (j2d5pt_measure_fma_rate) / 5 per chain cell, "
                            "integer path %.1f Gcells/s (j2d5pt_measure_exact_rate), exact share %.3f; x 9 flops "
                            "per cell" % (pk["fma64"] / 1e9, pk["exact"] / 1e9, pk["share"])),
            "kernel_gcells": round(kernel_gcells, 3), "peak_gcells": round(pk["alu_cells"] / 1e9, 3),
            "fp64_pipe_only_gcells": round(pk["fma64"] / 5 / 1e9, 3)}


def roof_f32_dtb(pk, kernel_gcells, sweep):
    """FP32 blocked kernels: on chip.  Shared memory carries one 4-byte load
    and store per cell per sweep (a sweep advances `sweep` steps); the FP32
    pipe does 5 FMA instructions per cell update.  The bound reported is the
    shared-memory pipe (the busiest unit in the profile); the FP32-pipe
    fraction is given beside it."""
    bpc = 8.0 / sweep
    achieved = kernel_gcells * 1e9 * bpc / 1e9
    peak = pk["smem"] / 1e9
    return {"bound": "smem", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "GB/s",
            "frac": round(achieved / peak, 4), "bytes_per_cell_update": bpc,
            "frac_fp32_pipe": round(kernel_gcells * 1e9 * 5 / pk["fma32"], 4),
            "peak_source": "of measured: shared memory j2d5pt_measure_smem_bandwidth; FP32 FMA j2d5pt_measure_fma_rate",
            "kernel_gcells": round(kernel_gcells, 3)}


def roof_f32_stream(pk, kernel_gcells, depth):
    """FP32 stream schedule (temporal blocking in registers): no shared-memory
    sweep; each cell update is 5 FMA-pipe operations (paired two to an
    instruction), so the bound is the FP32 pipe.  HBM carries one read and
    one write of the grid per pass of `depth` steps, plus the bands'
    overlapped x halo (128 columns read per 128 - 2G stored, G = depth
    rounded up to a whole vector): reported beside it."""
    g = (depth + 3) // 4 * 4
    bpc = 4.0 * (128.0 / (128 - 2 * g) + 1.0) / depth
    achieved = kernel_gcells * 9 / 1e3
    peak = pk["fma32"] / 5 * 9 / 1e12
    return {"bound": "alu", "achieved": round(achieved, 3), "peak": round(peak, 3), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "kernel": "stream_kernel",
            "hbm_bytes_per_cell_update": round(bpc, 4),
            "frac_hbm": round(kernel_gcells * bpc / (pk["hbm"] / 1e9), 4) if pk["hbm"] else None,
            "peak_source": "of measured: FP32 FMA j2d5pt_measure_fma_rate / 5 per cell; x 9 flops per cell",
            "kernel_gcells": round(kernel_gcells, 3), "peak_gcells": round(pk["fma32"] / 5 / 1e9, 2)}


def roof_f32(pk, kernel_gcells, desc):
    """The FP32 roofline record of whichever blocked schedule a plan runs."""
    f = dict(kv.split("=") for kv in desc.split())
    if f["algo"] == "stream":
        return roof_f32_stream(pk, kernel_gcells, int(f["depth"]))
    if f["algo"] == "onestep":
        return roof_hbm(pk, kernel_gcells, 4)
    return roof_f32_dtb(pk, kernel_gcells, int(f.get("sweep", "1")))


def roof_hbm(pk, kernel_gcells, elem):
    """One-step kernel, HBM: one read and one write of the element per cell update."""
    if not pk["hbm"]:
        return None
    achieved = kernel_gcells * 2 * elem
    peak = pk["hbm"] / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": round(peak, 1), "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs",
            "kernel_gcells": round(kernel_gcells, 3)}


def reps(plan, fn, flush, stream, cells, n=3):
    """Median over n repetitions (after one warm-up) of the whole-call and kernel GCells/s."""
    total, kern = timed(plan, fn, n, 1, flush, stream)
    out = {"gcells": round(gcells(cells, statistics.median(total)), 2), "reps": n}
    if kern and kern[0] is not None:
        out["kernel_gcells"] = round(gcells(cells, statistics.median(kern)), 2)
    return out


# ---- the headline -----------------------------------------------------------

def run_ours(args):
    import torch
    import __graft_entry__
    from paper_2306_03336_gb300 import j2d5pt, synth
    __graft_entry__.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    flush = L2Flush()
    nx = ny = HEAD_N
    steps_t = HEAD_T
    u0 = synth.field(nx, ny, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    plan = j2d5pt.Plan(nx, ny, "f64", w)
    src = plan.to_device(u0)
    dst = plan.empty()
    plan.autotune(src, dst, steps_t)
    plan.set("timing", 1)
    algo = algo_of(plan)

    def fn():
        plan.run(src, dst, steps_t, stream)

    l0 = j2d5pt.j2d5pt_kernel_launches()
    fn()
    plan.sync()
    launches_per_step = j2d5pt.j2d5pt_kernel_launches() - l0
    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    total, kern = timed(plan, fn, args.steps, args.warmup, flush, stream)
    clk = clocks.stop()
    plan.sync()
    cells = nx * ny * steps_t
    total_ms, value = aggregate(sum(total), cells * args.steps, world)

    pk = measure_peaks(j2d5pt)
    kern_ms = statistics.mean(kern)
    roof = roof_f64(pk, gcells(cells, kern_ms), traffic_for("f64_16384x16384_1000_" + algo), kernel_of(algo))

    # end to end through the C ABI on host buffers (pinned input and output)
    host_in = torch.from_numpy(u0).pin_memory().numpy()
    host_out = torch.empty(u0.shape, dtype=torch.float64).pin_memory().numpy()
    t_e2e, k_e2e = [], []
    n_e2e = max(3, min(args.steps, 5))
    clocks_e2e = Clocks(local)
    clocks_e2e.start()
    for i in range(1 + n_e2e):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out_h = plan.run_host(host_in, steps_t, out=host_out)
        t1 = time.perf_counter()
        if i >= 1:
            t_e2e.append(t1 - t0)
            k_e2e.append(plan.kernel_time())
    clk_e2e = clocks_e2e.stop()
    e2e = {"value": round(cells * len(t_e2e) * world / sum(t_e2e) / 1e9, 3), "unit": "GCells/s",
           "h2d_bytes_per_step": int(host_in.nbytes), "d2h_bytes_per_step": int(out_h.nbytes),
           "reps": len(t_e2e), "rep_seconds": [round(t, 4) for t in t_e2e],
           "kernel_ms": [round(k, 1) for k in k_e2e], "clocks": clk_e2e}
    del host_in, host_out

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(j2d5pt, synth, flush, stream, pk, plan, src, dst)
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(u0, w)
    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GCells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform [0,1) field and normalised uniform weights)",
            "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "time_steps": steps_t, "plan": plan.describe(),
                       "l2": "inputs (2.15 GB per buffer) larger than L2, and L2 flushed (256 MiB write) between steps",
                       "parallelism": "replicas (single-GPU method)" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps), "clocks": clk, "extras": extras,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def oracle_blocks_err(u0_f64, w, steps, got_view, size=256):
    """Max relative error of a GPU result against the FP64 oracle on blocks
    (corners, middle) evaluated exactly on windows of radius steps+1."""
    import oracle
    oracle.build()
    H, W = u0_f64.shape
    blocks = [(0, size, 0, size), ((H - size) // 2, (H + size) // 2, (W - size) // 2, (W + size) // 2),
              (H - size, H, W - size, W)]
    worst = 0.0
    for (y0, y1, x0, x1) in blocks:
        r = steps + 1
        a0, a1, b0, b1 = max(0, y0 - r), min(H, y1 + r), max(0, x0 - r), min(W, x1 + r)
        ref = oracle.run(np.ascontiguousarray(u0_f64[a0:a1, b0:b1]), w, steps, threads=oracle.max_threads())
        ref = ref[y0 - a0:y1 - a0, x0 - b0:x1 - b0]
        got = got_view[y0:y1, x0:x1].double().cpu().numpy()
        worst = max(worst, float((np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)).max()))
    return worst, "FP64 oracle on %d blocks of %dx%d cells (corners, middle), exact windows of radius %d" % (
        len(blocks), size, size, steps + 1)


def same_choice(p, desc):
    """Give plan p the algorithm, depth and tile shape another plan's description names."""
    f = dict(kv.split("=") for kv in desc.split())
    p.set("algo", f["algo"])
    if f["algo"] not in ("resident", "onestep"):
        p.set("depth", int(f["depth"])).set("tile_wx", int(f["tile_wx"]))
    return p


def run_extras(j2d5pt, synth, flush, stream, pk, head_plan, head_src, head_dst):
    """Secondary workloads, each beside the one-step kernel, each with its roofline record."""
    import torch
    out = {"peaks": {"fp64_gfma_s": round(pk["fma64"] / 1e9, 1), "fp32_gfma_s": round(pk["fma32"] / 1e9, 1),
                     "hbm_gbs": round(pk["hbm"] / 1e9, 1) if pk["hbm"] else None,
                     "fp64_alu_gcells": round(pk["alu_cells"] / 1e9, 2), "exact_gcells": round(pk["exact"] / 1e9, 2),
                     "smem_gbs": round(pk["smem"] / 1e9, 1)}}
    w = head_plan.weights[0]

    # 1) the headline grid (16384^2 FP64): one-step kernel, the FMA chain alone
    n, T = HEAD_N, HEAD_T
    cells = n * n * T
    p = j2d5pt.Plan(n, n, "f64", w).set("algo", "onestep").set("timing", 1)
    r = reps(p, lambda: p.run(head_src, head_dst, T, stream), flush, stream, cells)
    r["roofline"] = roof_f64(pk, r["kernel_gcells"], kernel="onestep_kernel")
    p.close()
    ent = {"onestep": r}
    p = same_choice(j2d5pt.Plan(n, n, "f64", w), head_plan.describe()).set("timing", 1).set("int_path", 0)
    r = reps(p, lambda: p.run(head_src, head_dst, T, stream), flush, stream, cells)
    r["frac_fp64_pipe"] = round(r["kernel_gcells"] / (pk["fma64"] / 5 / 1e9), 4)
    r["plan"] = p.describe()
    p.close()
    ent["fma_chain_only"] = r
    out["f64_16384x16384_1000"] = ent

    # 2) FP64 2048 x 1536, 1000 steps (fits on chip): every kernel family
    nx, ny, T = 2048, 1536, 1000
    u0 = synth.field(nx, ny, synth.data_seed(1))
    w1 = synth.weights(synth.weight_seed(1))
    cells = nx * ny * T
    fam = {}
    pa = j2d5pt.Plan(nx, ny, "f64", w1)
    a, b = pa.to_device(u0), pa.empty()
    pa.autotune(a, b, T)
    pa.set("timing", 1)
    r = reps(pa, lambda: pa.run(a, b, T, stream), flush, stream, cells)
    r["roofline"] = roof_f64(pk, r["kernel_gcells"], kernel=kernel_of(algo_of(pa)))
    r["plan"] = pa.describe()
    fam["autotuned"] = r
    pa.close()
    for algo, depth in (("onestep", 0), ("resident", 0), ("bands", 16), ("tiles", 8)):
        p = j2d5pt.Plan(nx, ny, "f64", w1).set("algo", algo).set("timing", 1)
        if depth:
            p.set("depth", depth)
        r = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
        r["frac_alu"] = round(r["kernel_gcells"] * 1e9 / pk["alu_cells"], 4)
        fam[algo] = r
        p.close()
    p = j2d5pt.Plan(nx, ny, "f64", w1).set("algo", "onestep").set("graph", 1)
    p.run(a, b, T, stream)
    r = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
    r["frac_alu"] = round(r["gcells"] * 1e9 / pk["alu_cells"], 4)
    fam["onestep_graph"] = r
    p.close()
    p = j2d5pt.Plan(nx, ny, "f64", w1).set("algo", "resident").set("timing", 1).set("int_path", 0)
    r = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
    r["frac_fp64_pipe"] = round(r["kernel_gcells"] / (pk["fma64"] / 5 / 1e9), 4)
    fam["resident_fma_chain_only"] = r
    p.close()
    out["f64_2048x1536_1000"] = fam
    del a, b

    # 3) FP32 16384^2, 1000 steps, same seeded data as the headline; error
    #    against the FP64 oracle (exact windows around blocks of cells)
    n, T = HEAD_N, HEAD_T
    cells = n * n * T
    u0 = synth.field(n, n, synth.data_seed(1))
    p = j2d5pt.Plan(n, n, "f32", w)
    a, b = p.to_device(u0.astype(np.float32)), p.empty()
    p.set("algo", "onestep").set("timing", 1)
    r1 = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
    r1["roofline"] = roof_hbm(pk, r1["kernel_gcells"], 4)
    p.set("algo", "auto")
    p.autotune(a, b, T)
    p.set("timing", 1)
    r2 = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
    r2["roofline"] = roof_f32(pk, r2["kernel_gcells"], p.describe())
    r2["plan"] = p.describe()
    err, how = oracle_blocks_err(u0.astype(np.float32).astype(np.float64), w, T, p.view(b))
    out["f32_16384x16384_1000"] = {"onestep": r1, "autotuned": r2, "max_rel_err_vs_fp64_oracle": err,
                                   "error_sample": how}
    p.close()
    del a, b
    torch.cuda.empty_cache()

    # 4) the paper's evaluation domain (Section 4, Figure 2): 8592 x 8328 run,
    #    8192^2 counted as the valid domain ("pruned"), FP64 and FP32, autotuned
    pd = {}
    nx_, ny_ = 8592, 8328
    uu = synth.field(nx_, ny_, synth.data_seed(1) + 20)
    for dt in ("f64", "f32"):
        p = j2d5pt.Plan(nx_, ny_, dt, w)
        a = p.to_device(uu if dt == "f64" else uu.astype(np.float32))
        b = p.empty()
        p.autotune(a, b, 1000)
        p.set("timing", 1)
        r = reps(p, lambda: p.run(a, b, 1000, stream), flush, stream, nx_ * ny_ * 1000)
        r["gcells_valid_8192sq"] = round(r["gcells"] * 8192 * 8192 / (nx_ * ny_), 2)
        if dt == "f64":
            r["roofline"] = roof_f64(pk, r["kernel_gcells"], kernel=kernel_of(algo_of(p)))
        else:
            r["roofline"] = roof_f32(pk, r["kernel_gcells"], p.describe())
        r["plan"] = p.describe()
        pd[dt] = r
        p.close()
        del a, b
        torch.cuda.empty_cache()
    out["paper_domain_8592x8328_1000"] = pd

    # 5) 256 batched FP64 grids, sides uniform in [64, 1024], 200 steps, CUDA graph
    cfg = synth.WORKLOADS["j2d5pt_f64_batch256_200"]
    sizes = synth.batch_sizes(cfg["count"], synth.data_seed(cfg["index"]), cfg["lo"], cfg["hi"])
    ws = np.stack([synth.weights(synth.weight_seed(cfg["index"]) + i) for i in range(len(sizes))])
    p = j2d5pt.Plan.batch(sizes, "f64", ws)
    srcs = [p.to_device(synth.field(a_, b_, synth.data_seed(cfg["index"]) + 10 + i), i) for i, (a_, b_) in enumerate(sizes)]
    dsts = [p.empty(i) for i in range(len(sizes))]
    p.autotune_batched(srcs, dsts, cfg["steps"])
    p.set("graph", 1)
    cells = sum(a_ * b_ for a_, b_ in sizes) * cfg["steps"]
    p.run_batched(srcs, dsts, cfg["steps"], stream)
    r = reps(p, lambda: p.run_batched(srcs, dsts, cfg["steps"], stream), flush, stream, cells)
    r["roofline"] = roof_f64(pk, r["gcells"])
    r["plan"] = p.describe()
    r["cells_per_step"] = int(cells / cfg["steps"])
    out["f64_batch256_200"] = r
    p.close()
    del srcs, dsts
    torch.cuda.empty_cache()

    # 6) the second stencil shape, the 3x3 box (j2d9pt): FP64 and FP32 16384^2,
    #    1000 steps, autotuned, beside its one-step kernel; FP64 against the
    #    arithmetic peak of the nine-term cell (FP64 pipe: 9 FMA instructions
    #    per chain cell; integer path: the measured nine-term rate; 17 flops per cell)
    n, T = HEAD_N, HEAD_T
    cells = n * n * T
    u0 = synth.field(n, n, synth.data_seed(1))
    wb = synth.box_weights(synth.weight_seed(1))
    exact9 = j2d5pt.j2d9pt_measure_exact_rate()
    f = pk["share"]
    alu9 = 1.0 / max((1.0 - f) / (pk["fma64"] / 9), f / exact9 if f else 0.0)
    box = {"exact9_gcells": round(exact9 / 1e9, 2), "peak_gcells": round(alu9 / 1e9, 2)}
    for dt in ("f64", "f32"):
        p = j2d5pt.Plan.box9(n, n, dt, wb)
        a, b = p.to_device(u0 if dt == "f64" else u0.astype(np.float32)), p.empty()
        p.set("algo", "onestep").set("timing", 1)
        r1 = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
        p.set("algo", "auto")
        p.autotune(a, b, T)
        p.set("timing", 1)
        r2 = reps(p, lambda: p.run(a, b, T, stream), flush, stream, cells)
        r2["plan"] = p.describe()
        if dt == "f64":
            for r in (r1, r2):
                g = r["kernel_gcells"]
                r["roofline"] = {"bound": "alu", "achieved": round(g * 17 / 1e3, 4),
                                 "peak": round(alu9 / 1e9 * 17 / 1e3, 4), "unit": "TFLOP/s",
                                 "frac": round(g * 1e9 / alu9, 4),
                                 "peak_source": "of measured: FP64 pipe / 9 per chain cell, nine-term integer path "
                                                "(j2d9pt_measure_exact_rate), exact share %.3f; x 17 flops" % f}
        else:
            r1["roofline"] = roof_hbm(pk, r1["kernel_gcells"], 4)
            f2 = dict(kv.split("=") for kv in p.describe().split())
            if f2["algo"] == "stream":
                # nine FMA-pipe operations per box cell (17 flops); HBM beside it
                k = int(f2["depth"])
                g9 = (k + 3) // 4 * 4
                bpc = 4.0 * (128.0 / (128 - 2 * g9) + 1.0) / k
                gk = r2["kernel_gcells"]
                r2["roofline"] = {"bound": "alu", "achieved": round(gk * 17 / 1e3, 3),
                                  "peak": round(pk["fma32"] / 9 * 17 / 1e12, 3), "unit": "TFLOP/s",
                                  "frac": round(gk * 1e9 * 9 / pk["fma32"], 4), "kernel": "stream_kernel",
                                  "hbm_bytes_per_cell_update": round(bpc, 4),
                                  "frac_hbm": round(gk * bpc / (pk["hbm"] / 1e9), 4) if pk["hbm"] else None,
                                  "peak_source": "of measured: FP32 FMA j2d5pt_measure_fma_rate / 9 per box cell; "
                                                 "x 17 flops per cell"}
            else:
                r2["roofline"] = roof_f32_dtb(pk, r2["kernel_gcells"], 1)
        box[dt] = {"onestep": r1, "autotuned": r2}
        p.close()
        del a, b
        torch.cuda.empty_cache()
    out["box9_16384x16384_1000"] = box

    # 7) gradient of L = <g, u_T>, 4096^2 FP64, 500 steps, checkpoints every 50
    from paper_2306_03336_gb300.autograd import J2D5PT
    cfg = synth.WORKLOADS["j2d5pt_f64_4096x4096_500_adjoint"]
    n, T = cfg["nx"], cfg["steps"]
    op = J2D5PT(n, n, "f64", cfg["checkpoint"])
    ut = torch.tensor(synth.field(n, n, synth.data_seed(cfg["index"])), device="cuda", requires_grad=True)
    wt = torch.tensor(synth.weights(synth.weight_seed(cfg["index"])), device="cuda", requires_grad=True)
    G = torch.tensor(synth.field(n, n, synth.data_seed(cfg["index"]) + 7), device="cuda")
    times = []
    for rep in range(4):
        ut.grad = None
        wt.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (op(ut, wt, T) * G).sum().backward()
        torch.cuda.synchronize()
        if rep:
            times.append(time.perf_counter() - t0)
    dt_ = statistics.median(times)
    p = j2d5pt.Plan(n, n, "f64", wt.detach().cpu().numpy()).set("timing", 1)
    a, b = p.to_device(G.cpu().numpy()), p.empty()
    ra = reps(p, lambda: p.run_adjoint(a, b, T, stream), flush, stream, n * n * T)
    ra["roofline"] = roof_f64(pk, ra["kernel_gcells"])
    ra["plan"] = p.describe()
    out["f64_4096x4096_500_grad"] = {"fwd_bwd_seconds": round(dt_, 4), "reps": len(times),
                                    "fwd_bwd_gcells": round(n * n * T / dt_ / 1e9, 2),
                                    "adjoint_only": ra, "checkpoint": cfg["checkpoint"]}
    p.close()
    op.close()
    return out


def cpu_baseline(u0, w, budget_s=12.0):
    """The oracle, as it stands, on the host cores, for a bounded number of steps."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    oracle.build()
    t0 = time.perf_counter()
    oracle.run(u0, w, 2, threads=threads)
    per = max((time.perf_counter() - t0) / 2, 1e-4)
    steps = int(max(2, min(1000, budget_s / per)))
    t0 = time.perf_counter()
    oracle.run(u0, w, steps, threads=threads)
    dt = time.perf_counter() - t0
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    return {"value": round(nx * ny * steps / dt / 1e9, 4), "unit": "GCells/s", "cores": threads, "kind": "oracle",
            "sample": "%dx%d FP64, %d of the 1000 time steps (%.2f s)" % (nx, ny, steps, dt)}


def run_reference(args):
    """The oracle (plain CPU FP64 code) on this workload: each step a bounded sample."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2306_03336_gb300 import synth
    oracle.build()
    nx = ny = HEAD_N
    u0 = synth.field(nx, ny, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    threads = len(os.sched_getaffinity(0))
    sample_steps = 4
    for _ in range(args.warmup):
        oracle.run(u0, w, 1, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(u0, w, sample_steps, threads=threads)
    dt = time.perf_counter() - t0
    value = nx * ny * sample_steps * args.steps / dt / 1e9
    sample = "%dx%d FP64, %d of the 1000 time steps per benchmark step" % (nx, ny, sample_steps)
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GCells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform [0,1) field and normalised uniform weights)",
            "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "time_steps": HEAD_T, "sample": sample},
            "cpu_baseline": {"value": round(value, 4), "unit": "GCells/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GCells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---- named runs for profiling --------------------------------------------------
# name: (nx, ny, dtype, algo, depth, tile_wx, steps, runs); algo "auto" = autotuned,
# "box:ALGO" = the 3x3 box stencil with that algorithm, "batch:ALGO" = the first
# nx grids of the 256-grid batch workload with that algorithm
WORKLOADS = {
    "headline": (HEAD_N, HEAD_N, "f64", "auto", 0, 0, HEAD_T, 2),
    "f64tiles": (8192, 8192, "f64", "tiles", 4, 4, 8, 1),
    "f64resident": (2048, 1536, "f64", "resident", 0, 0, 1000, 1),
    "f64onestep": (2048, 1536, "f64", "onestep", 0, 0, 8, 1),
    "f64skewed": (8192, 8192, "f64", "skewed", 4, 4, 8, 1),
    "f32tiles": (8192, 8192, "f32", "tiles", 16, 2, 16, 1),
    "f32skewed": (8192, 8192, "f32", "skewed", 16, 8, 32, 1),
    "f32onestep": (8192, 8192, "f32", "onestep", 0, 0, 4, 1),
    "f32stream": (8192, 8192, "f32", "stream", 8, 0, 16, 1),
    "f64stream": (8192, 8192, "f64", "stream", 2, 0, 4, 1),
    "f32boxstream": (8192, 8192, "f32", "box:stream", 8, 0, 16, 1),
    "f64box": (8192, 8192, "f64", "box:skewed", 4, 4, 8, 1),
    "f64batch": (64, 0, "f64", "batch:resident", 0, 0, 20, 1),
}


def run_workload(name):
    """One named workload on the seeded inputs, for ncu; prints the plan and exits."""
    import torch
    import __graft_entry__
    from paper_2306_03336_gb300 import j2d5pt, synth
    if name not in WORKLOADS:
        raise SystemExit("unknown workload %r (one of %s)" % (name, ", ".join(sorted(WORKLOADS))))
    nx, ny, dt, algo, depth, wx, steps, runs = WORKLOADS[name]
    __graft_entry__.build()
    torch.cuda.set_device(0)
    if algo.startswith("batch:"):
        cfg = synth.WORKLOADS["j2d5pt_f64_batch256_200"]
        sizes = synth.batch_sizes(cfg["count"], synth.data_seed(cfg["index"]), cfg["lo"], cfg["hi"])[:nx]
        ws = np.stack([synth.weights(synth.weight_seed(cfg["index"]) + i) for i in range(len(sizes))])
        p = j2d5pt.Plan.batch(sizes, dt, ws).set("algo", algo[6:])
        srcs = [p.to_device(synth.field(a, b, synth.data_seed(cfg["index"]) + 10 + i), i) for i, (a, b) in enumerate(sizes)]
        dsts = [p.empty(i) for i in range(len(sizes))]
        for _ in range(runs):
            p.run_batched(srcs, dsts, steps)
        p.sync()
        print(name, p.describe(), flush=True)
        p.close()
        return
    if algo.startswith("box:"):
        algo = algo[4:]
        p = j2d5pt.Plan.box9(nx, ny, dt, synth.box_weights(synth.weight_seed(1)))
    else:
        p = j2d5pt.Plan(nx, ny, dt, synth.weights(synth.weight_seed(1)))
    u0 = synth.field(nx, ny, synth.data_seed(1))
    src = p.to_device(u0 if dt == "f64" else u0.astype(np.float32))
    dst = p.empty()
    if algo == "auto":
        p.autotune(src, dst, steps)
    else:
        p.set("algo", algo)
        if depth:
            p.set("depth", depth)
        if wx:
            p.set("tile_wx", wx)
    for _ in range(runs):
        p.run(src, dst, steps)
    p.sync()
    print(name, p.describe(), flush=True)
    p.close()


def main():
    args = parse()
    if args.workload:
        run_workload(args.workload)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
