"""Build step for libj2d5pt.so: nvcc for sm_103a, one object per translation
unit compiled in parallel, then a shared-library link.  Also builds the
bounds-checked variant libj2d5pt_checked.so (-DJ2D_BOUNDS_CHECK: every memory
access of the blocked kernels tested against its buffer, a failure reported
as J2D_ERR_BOUNDS).  Output stays in the package directory (git-ignored)."""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libj2d5pt.so")
LIB_CHECKED = os.path.join(HERE, "libj2d5pt_checked.so")
UNITS = ["api.cu", "onestep.cu", "dtb.cu", "stream.cu", "noalloc.cu"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
         "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall", "--expt-relaxed-constexpr"]
VARIANTS = {LIB: ("regular", []), LIB_CHECKED: ("checked", ["-DJ2D_BOUNDS_CHECK"])}


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "j2d5pt.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _compile(job):
    unit, sub, extra = job
    src = os.path.join(CSRC, unit)
    os.makedirs(os.path.join(BUILD, sub), exist_ok=True)
    obj = os.path.join(BUILD, sub, unit.replace(".cu", ".o"))
    cmd = [NVCC] + FLAGS + list(extra) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (unit, " ".join(cmd), r.stderr))
    return obj, r.stderr


def _link(lib, objs):
    tmp = lib + ".tmp"
    r = subprocess.run([NVCC, "-shared", "-o", tmp] + objs, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)


def build(force=False, verbose=False, extra=(), checked=True):
    """Compile the CUDA libraries whose sources are newer than them (the
    regular one, and with checked=True also the bounds-checked one); return
    the path of the regular library."""
    deps = _deps_mtime()
    libs = [LIB] + ([LIB_CHECKED] if checked else [])
    stale = [l for l in libs if force or not os.path.exists(l) or os.path.getmtime(l) < deps]
    if not stale:
        return LIB
    jobs = [(u, VARIANTS[l][0], list(VARIANTS[l][1]) + list(extra)) for l in stale for u in UNITS]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(_compile, jobs))
    if verbose:
        for _, err in results:
            if err.strip():
                sys.stderr.write(err)
    for i, l in enumerate(stale):
        _link(l, [o for o, _ in results[i * len(UNITS):(i + 1) * len(UNITS)]])
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
