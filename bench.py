"""Benchmark: j2d5pt on one GB300, GCells/s (interior cell updates per second).

Default workload: FP64, 2048 x 1536 interior cells plus the one-cell ring,
seeded uniform [0,1) data and normalised weights, 1000 time steps per step of
the benchmark (one "step" here = one full j2d5pt_run of 1000 time steps).
The library's AUTO configuration is timed (the tuned temporally blocked
kernel); the one-step kernel and the other workloads are reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: CUDA events on the launching stream, one event pair per benchmark
step, L2 flushed (256 MiB write) between steps, synchronise before and after.
`e2e` times j2d5pt_run_host (host buffers, copies inside the timed region).
With --gpus N > 1 (torchrun) every rank runs its own replica (the method is
single-GPU): value = all ranks' cell updates / max rank time, scaling "weak".
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
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---- clocks --------------------------------------------------------------

class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "j2d_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

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
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- workloads -----------------------------------------------------------

def make_inputs(nx, ny, index, dtype):
    from paper_2306_03336_gb300 import synth
    u0 = synth.field(nx, ny, synth.data_seed(index))
    w = synth.weights(synth.weight_seed(index))
    return (u0 if dtype == "f64" else u0.astype(np.float32)), w


class L2Flush:
    def __init__(self):
        import torch
        self.buf = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def __call__(self):
        self.buf.fill_(1.0)


def time_runs(fn, steps, warmup, flush, stream):
    """Per-step CUDA-event times (ms) of fn() on `stream`, L2 flushed between steps."""
    import torch
    for _ in range(warmup):
        flush()
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    return times


def kernel_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_03336_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it matches the current sources."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except Exception:
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("source_hash") != kernel_hash():
        return None
    return ent.get("bytes_per_launch")


def cpu_baseline(u0, w, budget_s=12.0):
    """The oracle, as it stands, on the host cores, for a bounded number of steps."""
    import oracle
    threads = len(os.sched_getaffinity(0))
    t0 = time.perf_counter()
    oracle.run(u0, w, 2, threads=threads)
    t1 = time.perf_counter()
    per = max((t1 - t0) / 2, 1e-4)
    steps = int(max(2, min(1000, budget_s / per)))
    t0 = time.perf_counter()
    oracle.run(u0, w, steps, threads=threads)
    dt = time.perf_counter() - t0
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    return {"value": nx * ny * steps / dt / 1e9, "unit": "GCells/s", "cores": threads, "kind": "oracle",
            "sample": "%dx%d FP64, %d of the 1000 steps (%.1f s)" % (nx, ny, steps, dt)}


def run_ours(args):
    import torch
    from paper_2306_03336_gb300 import j2d5pt
    import __graft_entry__
    __graft_entry__.build()
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.current_stream()
    flush = L2Flush()
    nx, ny, steps_t = 2048, 1536, 1000
    u0, w = make_inputs(nx, ny, 1, "f64")
    plan = j2d5pt.Plan(nx, ny, "f64", w)
    src = plan.to_device(u0)
    dst = plan.empty()
    plan.autotune(src, dst, steps_t)
    config_desc = plan.describe()

    def fn():
        plan.run(src, dst, steps_t, stream)

    launches0 = j2d5pt.j2d5pt_kernel_launches()
    fn()
    plan.sync()
    launches_per_step = j2d5pt.j2d5pt_kernel_launches() - launches0

    clocks = Clocks(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = time_runs(fn, args.steps, args.warmup, flush, stream)
    clk = clocks.stop()
    plan.sync()
    total_ms = sum(times)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    cells = nx * ny * steps_t
    value = cells * args.steps * world / (total_ms * 1e-3) / 1e9
    kernel_gcells = cells / (min(times) * 1e-3) / 1e9

    # roofline of the dominant kernel: FP64 pipe (5 FP64 instructions per cell update)
    fma64 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F64)
    peak_cells = fma64 / 5 / 1e9
    achieved_tflops = kernel_gcells * 9 / 1e3
    peak_tflops = fma64 / 5 * 9 / 1e12
    algo = config_desc.split("algo=")[1].split()[0]
    roof = {"bound": "alu", "achieved": round(achieved_tflops, 4), "peak": round(peak_tflops, 4),
            "unit": "TFLOP/s", "frac": round(achieved_tflops / peak_tflops, 4),
            "traffic": traffic_for("f64_2048x1536_" + algo),
            "kernel": algo, "peak_source": "measured FP64 FMA rate %.1f GFMA/s x 9 flops / 5 instructions" % (fma64 / 1e9),
            "peak_gcells": round(peak_cells, 2)}

    # e2e through the C ABI on host buffers
    host_in = torch.from_numpy(u0).pin_memory().numpy()
    h2d = host_in.nbytes
    t_e2e = []
    for i in range(args.warmup + args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out_h = plan.run_host(host_in, steps_t)
        t1 = time.perf_counter()
        if i >= args.warmup:
            t_e2e.append(t1 - t0)
    e2e = {"value": round(cells * len(t_e2e) * world / sum(t_e2e) / 1e9, 3), "unit": "GCells/s",
           "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(out_h.nbytes)}

    extras = {}
    if not args.no_extras and rank == 0:
        extras = run_extras(plan, src, dst, stream, flush, u0, w)

    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        cpu = cpu_baseline(u0, w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 3), "unit": "GCells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded uniform [0,1) field, normalised uniform weights)",
            "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "time_steps": steps_t,
                       "plan": config_desc, "l2": "flushed (256 MiB write) between steps",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches_per_step * args.steps),
            "clocks": clk, "extras": extras,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def gcells(nx, ny, steps, ms):
    return nx * ny * steps / (ms * 1e-3) / 1e9


def run_extras(plan, src, dst, stream, flush, u0, w):
    """Secondary measurements (one-step kernel on the main workload, other workloads)."""
    import torch
    from paper_2306_03336_gb300 import j2d5pt
    out = {}
    nx, ny = 2048, 1536
    p1 = j2d5pt.Plan(nx, ny, "f64", w).set("algo", "onestep")
    t = time_runs(lambda: p1.run(src, dst, 1000, stream), 2, 1, flush, stream)
    out["f64_2048x1536_onestep_gcells"] = round(gcells(nx, ny, 1000, min(t)), 3)
    p1.close()
    return out


def run_reference(args):
    """The oracle (plain CPU FP64 code) on this workload: each step a bounded sample."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    nx, ny = 2048, 1536
    u0, w = make_inputs(nx, ny, 1, "f64")
    threads = len(os.sched_getaffinity(0))
    sample_steps = 20
    for _ in range(args.warmup):
        oracle.run(u0, w, 2, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(u0, w, sample_steps, threads=threads)
    dt = time.perf_counter() - t0
    value = nx * ny * sample_steps * args.steps / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GCells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "nx": nx, "ny": ny,
                                            "sample": "%d of the 1000 time steps per benchmark step" % sample_steps},
            "cpu_baseline": {"value": round(value, 4), "unit": "GCells/s", "cores": threads, "kind": "oracle",
                             "sample": "%dx%d FP64, %d time steps per benchmark step" % (nx, ny, sample_steps)},
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
