"""Build libakra.so (sm_103a) in-tree: one nvcc process per translation unit, then link.

Two variants are built side by side: libakra.so (release) and libakra_debug.so, the same
sources compiled with -DAKRA_DEBUG (bounds checks on the global-memory indices of the operator
kernels, see akra_debug_violations in include/akra.h).
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "libakra.so")
OUT_DEBUG = os.path.join(HERE, "libakra_debug.so")
TUS = ["akra_plan", "akra_legendre", "akra_legendre_tc", "akra_ringfft", "akra_ringfft32", "akra_cg", "akra_grad", "akra_batch",
       "akra_static", "akra_diag", "akra_spectra", "akra_flat"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "-diag-suppress", "128", "-Wno-deprecated-gpu-targets"]
VARIANTS = {OUT: ("release", []), OUT_DEBUG: ("debug", ["-DAKRA_DEBUG"])}


def _nvcc() -> str:
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _stale(out: str) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "akra.h")]
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every stale variant (all translation units of all variants in parallel) and
    return the release library's path."""
    outs = [o for o in VARIANTS if force or _stale(o)]
    if not outs:
        return OUT
    nvcc = _nvcc()
    procs = []
    for out in outs:
        name, defs = VARIANTS[out]
        bdir = os.path.join(ROOT, "_build", name)
        os.makedirs(bdir, exist_ok=True)
        for tu in TUS:
            obj = os.path.join(bdir, tu + ".o")
            cmd = [nvcc, *ARCH, *FLAGS, *defs, "-c", os.path.join(CSRC, tu + ".cu"), "-o", obj]
            procs.append((out, tu, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    objs = {o: [] for o in outs}
    for out, tu, obj, pr in procs:
        res, _ = pr.communicate()
        if pr.returncode != 0:
            sys.stderr.write(res.decode(errors="replace"))
            raise RuntimeError("nvcc failed on %s (%s)" % (tu, VARIANTS[out][0]))
        if verbose:
            sys.stdout.write(res.decode(errors="replace"))
        objs[out].append(obj)
    for out in outs:
        tmp = out + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs[out]])
        os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
