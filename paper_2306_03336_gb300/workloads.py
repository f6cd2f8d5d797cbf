"""Run one named workload once, for profiling (e.g. under ncu):

  python -m paper_2306_03336_gb300.workloads headline   # FP64 2048x1536, 1000 steps: resident, then bands k=32 (4 runs each)
  python -m paper_2306_03336_gb300.workloads f32tiles   # FP32 8192^2, tiles k=16, 16 steps (one launch)
  python -m paper_2306_03336_gb300.workloads f32onestep # FP32 8192^2, one-step kernel, 4 steps
  python -m paper_2306_03336_gb300.workloads f64onestep # FP64 2048x1536, one-step kernel, 8 steps
  python -m paper_2306_03336_gb300.workloads f64tiles   # FP64 8192^2, tiles k=4, 4 strips wide, 8 steps (one launch)

Inputs are the seeded synthetic fields of paper_2306_03336_gb300.synth.
"""
import sys

import torch

from . import build as _build
from . import j2d5pt, synth


def _plan(nx, ny, dt, algo, depth=0, wx=0, index=1):
    p = j2d5pt.Plan(nx, ny, dt, synth.weights(synth.weight_seed(index))).set("algo", algo)
    if depth:
        p.set("depth", depth)
    if wx:
        p.set("tile_wx", wx)
    u0 = synth.field(nx, ny, synth.data_seed(index))
    src = p.to_device(u0 if dt == "f64" else u0.astype("float32"))
    return p, src, p.empty()


def main(which):
    _build.build()
    torch.cuda.set_device(0)
    if which == "headline":
        for algo, depth in (("resident", 0), ("bands", 32)):
            p, src, dst = _plan(2048, 1536, "f64", algo, depth)
            for _ in range(4):
                p.run(src, dst, 1000)
            p.sync()
            p.close()
    elif which == "f32tiles":
        p, src, dst = _plan(8192, 8192, "f32", "tiles", 16, 2)
        p.run(src, dst, 16)
        p.sync()
        p.close()
    elif which == "f32onestep":
        p, src, dst = _plan(8192, 8192, "f32", "onestep")
        p.run(src, dst, 4)
        p.sync()
        p.close()
    elif which == "f64tiles":
        p, src, dst = _plan(8192, 8192, "f64", "tiles", 4, 4)
        p.run(src, dst, 8)
        p.sync()
        p.close()
    elif which == "f64onestep":
        p, src, dst = _plan(2048, 1536, "f64", "onestep")
        p.run(src, dst, 8)
        p.sync()
        p.close()
    else:
        raise SystemExit("unknown workload %r" % which)
    print("done")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "headline")
