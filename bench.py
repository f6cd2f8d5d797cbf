"""Benchmark: j2d5pt on one GB300, GCells/s (interior cell updates per second).

Headline workload (one line of JSON): FP64, 2048 x 1536 interior cells plus
the one-cell ring, seeded uniform [0,1) data and normalised weights, 1000 time
steps per benchmark step (one benchmark step = one j2d5pt_run of 1000 time
steps).  The plan is autotuned first (one-step / resident / bands / tiles over
temporal depths), then timed.  The other workloads (FP64 and FP32 16384^2 with
1000 steps, 256 batched grids with 200 steps, the 4096^2 gradient with 500
steps) are reported under "extras", each against the one-step kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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
WORKLOAD = "j2d5pt_f64_2048x1536_1000"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)  # ~1 s timed: several clock samples
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
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
    nx, ny, steps_t = 2048, 1536, 1000
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

    # roofline of the dominant kernel: arithmetic.  An FP64 cell update is 9
    # flops (5 multiplies, 4 adds).  Half the cells (the exact mask) run on
    # the integer pipes, the rest as 5 FP64 FMA instructions on the FP64 pipe;
    # the two pipes work in parallel, so the peak cell rate is set by the
    # slower of the two shares, each at its measured rate.
    fma64 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F64)
    alu = alu_peak(j2d5pt, fma64)
    kern_ms = statistics.mean(kern)
    achieved = cells * 9 / (kern_ms * 1e-3) / 1e12
    peak = alu["peak_gcells"] * 9 / 1e3
    roof = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "traffic": traffic_for("f64_2048x1536_1000_" + algo),
            "kernel": "dtb_kernel" if algo != "onestep" else "onestep_kernel",
            "peak_source": ("measured: FP64 pipe %.1f GFMA/s (j2d5pt_measure_fma_rate) / 5 per chain cell, integer "
                            "path %.1f Gcells/s (j2d5pt_measure_exact_rate), exact share %.3f; x 9 flops per cell"
                            % (fma64 / 1e9, alu["exact_gcells"], alu["exact_share"])),
            "kernel_gcells": round(gcells(cells, kern_ms), 3), "peak_gcells": alu["peak_gcells"],
            "fp64_pipe_only_gcells": round(fma64 / 5 / 1e9, 3)}

    # end to end through the C ABI on host buffers (pinned input and output)
    host_in = torch.from_numpy(u0).pin_memory().numpy()
    host_out = torch.empty(u0.shape, dtype=torch.float64).pin_memory().numpy()
    t_e2e = []
    for i in range(args.warmup + args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out_h = plan.run_host(host_in, steps_t, out=host_out)
        t1 = time.perf_counter()
        if i >= args.warmup:
            t_e2e.append(t1 - t0)
    e2e = {"value": round(cells * len(t_e2e) * world / sum(t_e2e) / 1e9, 3), "unit": "GCells/s",
           "h2d_bytes_per_step": int(host_in.nbytes), "d2h_bytes_per_step": int(out_h.nbytes)}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(j2d5pt, synth, flush, stream, src, dst, w, fma64, alu["peak_gcells"])
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
                       "l2": "flushed (256 MiB write) between steps",
                       "parallelism": "replicas (single-GPU method)" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps), "clocks": clk, "extras": extras,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def alu_peak(j2d5pt, fma64):
    """Arithmetic peak of the FP64 kernels in cells/s (see run_ours)."""
    exact = j2d5pt.j2d5pt_measure_exact_rate()
    mask, _ = j2d5pt.j2d5pt_arith_info()
    f = bin(mask & 0xFF).count("1") / 8.0
    chain = fma64 / 5
    peak = 1.0 / max((1.0 - f) / chain, f / exact if f else 0.0)
    return {"peak_gcells": round(peak / 1e9, 3), "exact_gcells": round(exact / 1e9, 3), "exact_share": f}


def one(plan, fn, flush, stream, cells, reps=1):
    total, kern = timed(plan, fn, reps, 1, flush, stream)
    return round(gcells(cells, min(total)), 2), round(gcells(cells, min(kern)), 2)


def run_extras(j2d5pt, synth, flush, stream, src, dst, w, fma64, alu64):
    """Secondary workloads, each beside the one-step kernel."""
    import torch
    out = {}
    hbm = None
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        pass
    fma32 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F32)
    smem = j2d5pt.j2d5pt_measure_smem_bandwidth() / 1e9  # GB/s
    out["peaks"] = {"fp64_gfma_s": round(fma64 / 1e9, 1), "fp32_gfma_s": round(fma32 / 1e9, 1), "hbm_gbs": hbm,
                    "fp64_alu_gcells": alu64, "smem_gbs": round(smem, 1)}
    # DTB shared-memory traffic per cell update: one read and one write of the
    # element (the in-place row sweep); frac_smem = that rate / measured peak

    # 1) the headline grid through each kernel family
    nx, ny, T = 2048, 1536, 1000
    fam = {}
    for algo, depth in (("onestep", 0), ("resident", 0), ("bands", 16), ("tiles", 8)):
        p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", algo).set("timing", 1)
        if depth:
            p.set("depth", depth)
        run, kern = one(p, lambda: p.run(src, dst, T, stream), flush, stream, nx * ny * T)
        fam[algo] = {"gcells": run, "kernel_gcells": kern, "frac_alu": round(kern / alu64, 3)}
        if algo != "onestep":
            fam[algo]["frac_smem"] = round(kern * 16 / smem, 3)
        p.close()
    # the one-step baseline with its 1000 launches replayed from a CUDA graph
    p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", "onestep").set("graph", 1)
    p.run(src, dst, T, stream)
    total, _ = timed(p, lambda: p.run(src, dst, T, stream), 1, 1, flush, stream)
    run = round(gcells(nx * ny * T, min(total)), 2)
    fam["onestep_graph"] = {"gcells": run, "frac_alu": round(run / alu64, 3)}
    p.close()
    # the same resident kernel with every cell on the FMA chain (integer path off)
    p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", "resident").set("timing", 1).set("int_path", 0)
    run, kern = one(p, lambda: p.run(src, dst, T, stream), flush, stream, nx * ny * T)
    fam["resident_fma_chain_only"] = {"gcells": run, "kernel_gcells": kern,
                                      "frac_fp64_pipe": round(kern / (fma64 / 5 / 1e9), 3)}
    p.close()
    out["f64_2048x1536_1000"] = fam

    # 2) 16384^2, FP64 and FP32 from the same seeded data, 1000 steps
    n, T = 16384, 1000
    u0 = synth.field(n, n, synth.data_seed(1))
    res = {}
    for dt in ("f64", "f32"):
        p = j2d5pt.Plan(n, n, dt, w)
        a = p.to_device(u0 if dt == "f64" else u0.astype(np.float32))
        b = p.empty()
        p.set("algo", "onestep").set("timing", 1)
        r1, k1 = one(p, lambda: p.run(a, b, T, stream), flush, stream, n * n * T)
        p.autotune(a, b, T)
        best = p.describe()
        r2, k2 = one(p, lambda: p.run(a, b, T, stream), flush, stream, n * n * T)
        ent = {"onestep_gcells": r1, "best_gcells": r2, "best_kernel_gcells": k2, "best_plan": best}
        if dt == "f64":
            ent["onestep_frac_alu"] = round(k1 / alu64, 3)
            ent["best_frac_alu"] = round(k2 / alu64, 3)
            ent["best_frac_smem"] = round(k2 * 16 / smem, 3)
            ref64 = p.view(b).clone()
        else:
            if hbm:
                ent["onestep_frac_hbm"] = round(k1 * 8 / hbm, 3)
            ent["best_frac_fp32_pipe"] = round(k2 / (fma32 / 5 / 1e9), 3)
            # one 4-byte load and store per cell per sweep; a sweep advances `sweep` steps
            sweep = int(dict(kv.split("=") for kv in best.split()).get("sweep", "1"))
            ent["best_frac_smem"] = round(k2 * 8 / sweep / smem, 3)
            got = p.view(b).double()
            ent["max_rel_err_vs_fp64"] = float(((got - ref64).abs().max() / ref64.abs().max()).item())
            del ref64
        res[dt] = ent
        del a, b
        p.close()
        torch.cuda.empty_cache()
    out["16384x16384_1000"] = res

    # 2b) the paper's evaluation domain (Figure 2): 8592 x 8328 run, 8192^2 counted
    #     as the valid domain ("pruned"), FP64 and FP32, 1000 steps, autotuned
    pd = {}
    for dt in ("f64", "f32"):
        nx_, ny_ = 8592, 8328
        p = j2d5pt.Plan(nx_, ny_, dt, w)
        uu = synth.field(nx_, ny_, synth.data_seed(1) + 20)
        a = p.to_device(uu if dt == "f64" else uu.astype(np.float32))
        b = p.empty()
        p.autotune(a, b, 1000)
        p.set("timing", 1)
        total, kern = timed(p, lambda: p.run(a, b, 1000, stream), 1, 1, flush, stream)
        t = min(total)
        pd[dt] = {"gcells_full_domain": round(gcells(nx_ * ny_ * 1000, t), 2),
                  "gcells_valid_8192sq": round(gcells(8192 * 8192 * 1000, t), 2), "plan": p.describe()}
        p.close()
        del a, b
        torch.cuda.empty_cache()
    out["paper_domain_8592x8328_1000"] = pd

    # 3) 256 batched FP64 grids, sides uniform in [64, 1024], 200 steps, CUDA graph
    cfg = synth.WORKLOADS["j2d5pt_f64_batch256_200"]
    sizes = synth.batch_sizes(cfg["count"], synth.data_seed(cfg["index"]), cfg["lo"], cfg["hi"])
    ws = np.stack([synth.weights(synth.weight_seed(cfg["index"]) + i) for i in range(len(sizes))])
    p = j2d5pt.Plan.batch(sizes, "f64", ws)
    srcs = [p.to_device(synth.field(a_, b_, synth.data_seed(cfg["index"]) + 10 + i), i) for i, (a_, b_) in enumerate(sizes)]
    dsts = [p.empty(i) for i in range(len(sizes))]
    p.autotune_batched(srcs, dsts, cfg["steps"])
    p.set("graph", 1).set("timing", 1)
    cells = sum(a_ * b_ for a_, b_ in sizes) * cfg["steps"]
    rb, kb = one(p, lambda: p.run_batched(srcs, dsts, cfg["steps"], stream), flush, stream, cells, reps=2)
    out["f64_batch256_200"] = {"gcells": rb, "plan": p.describe(), "cells_per_step": int(cells / cfg["steps"])}
    p.close()
    del srcs, dsts
    torch.cuda.empty_cache()

    # 4) gradient of L = <g, u_T>, 4096^2 FP64, 500 steps, checkpoints every 50
    from paper_2306_03336_gb300.autograd import J2D5PT
    cfg = synth.WORKLOADS["j2d5pt_f64_4096x4096_500_adjoint"]
    n, T = cfg["nx"], cfg["steps"]
    op = J2D5PT(n, n, "f64", cfg["checkpoint"])
    ut = torch.tensor(synth.field(n, n, synth.data_seed(cfg["index"])), device="cuda", requires_grad=True)
    wt = torch.tensor(synth.weights(synth.weight_seed(cfg["index"])), device="cuda", requires_grad=True)
    G = torch.tensor(synth.field(n, n, synth.data_seed(cfg["index"]) + 7), device="cuda")
    for rep in range(2):
        ut.grad = None
        wt.grad = None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (op(ut, wt, T) * G).sum().backward()
        torch.cuda.synchronize()
        dt_ = time.perf_counter() - t0
    p = j2d5pt.Plan(n, n, "f64", wt.detach().cpu().numpy()).set("timing", 1)
    a, b = p.to_device(G.cpu().numpy()), p.empty()
    radj, kadj = one(p, lambda: p.run_adjoint(a, b, T, stream), flush, stream, n * n * T)
    out["f64_4096x4096_500_grad"] = {"fwd_bwd_seconds": round(dt_, 4),
                                    "fwd_bwd_gcells": round(n * n * T / dt_ / 1e9, 2),
                                    "adjoint_only_gcells": radj, "checkpoint": cfg["checkpoint"]}
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
    nx, ny = 2048, 1536
    u0 = synth.field(nx, ny, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    threads = len(os.sched_getaffinity(0))
    sample_steps = 200
    for _ in range(args.warmup):
        oracle.run(u0, w, 2, threads=threads)
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
            "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "time_steps": 1000, "sample": sample},
            "cpu_baseline": {"value": round(value, 4), "unit": "GCells/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GCells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
