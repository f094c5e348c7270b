#!/usr/bin/env python
"""Benchmark of the AKRA 3.0 hot path on GB300.

One step = one mixed-precision PCG solve (FP32 inner CG, FP64 outer refinement) of the
regularised normal equations at Nside 2048, lmax 4096 on a synthetic DES-like footprint, to
relative residual 1e-6 -- every H application inside it runs the full chain (KS,
spin-2 synthesis, ring FFT x W x FFT, exact adjoint, epilogue) in libakra.so.

Metric (as named): "H-applies/s and CG solve time at Nside=2048 (mixed vs FP64, rel.res 1e-6)";
`value` = H applications (FP32 inner + FP64 outer + the FP64 A^T of b) per second over the
timed solves, whole job (summed over ranks); ms_per_step = the CG solve time, the number to
compare (a policy that needs fewer inner iterations lowers `value` while the solve gets faster).

After the timed region the same line reports, untimed: a plain FP64 GPU CG solve of the same
system to 1e-6 (measured), the solution errors of both against a reference solved to an FP64
residual of 1e-10, the Nside 512 / lmax 1024 FP64-vs-mixed workload, the batched uneven-instance
workload (64 RHS), the differentiation workload (Nside 512), the roofline of the dominant kernel,
the CPU oracle baseline and the end-to-end solve from host buffers.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
       [--headline-only]   (skip the untimed comparison blocks)
Under torchrun each rank solves its own replica (independent noise realisation): weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H-applies/s and CG solve time at Nside=2048 (mixed vs FP64, rel.res 1e-6)"
UNIT = "H-applies/s"
NSIDE, LMAX, TOL = 2048, 4096, 1e-6
REF_TOL = 1e-10          # FP64 residual of the reference solutions the errors are taken against
FP32_LANES = 128         # FP32 FMA lanes per SM (sm_100 family)
PROFILES = os.path.join(ROOT, "profiles")


def _hbm_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


HBM_GBS = _hbm_gbs()


def _sm_max_mhz():
    """Maximum SM clock: the measured record of this machine, else GB300's 2070 MHz."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["sm_max_mhz"])
    except Exception:
        return 2070.0


def fp32_peak_tflops(sm_count, mhz):
    # SMs x 128 FP32 lanes x 2 flops (FMA) x clock
    return sm_count * FP32_LANES * 2 * mhz * 1e6 / 1e12


def kernel_source_sha():
    """Short hash of the CUDA-core Legendre kernels' device code (scalar items and the paired
    FP32 adjoint): a DRAM-traffic capture is only valid for the kernel code it was taken with.
    Comments and blank lines are left out, so that an edit of the comments keeps a capture."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in ("akra_legendre_impl.cuh", "akra_legendre_f32x2.cuh"):
        with open(os.path.join(ROOT, "paper_2606_06175_gb300", "csrc", f), encoding="utf-8") as fh:
            src = fh.read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        code = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
        h.update(code.encode("utf-8"))
    return h.hexdigest()[:12]


def captured_traffic(kernel):
    """DRAM bytes per launch of `kernel` at the bench workload from the committed ncu summary
    (profiles/legendre_traffic_des2048.md, line `bench-traffic: kernel=... source=<sha>
    dram_bytes_per_launch=<n>`).  (bytes, note); bytes is None when no capture matches the
    current kernel source."""
    path = os.path.join(PROFILES, "legendre_traffic_des2048.md")
    sha = kernel_source_sha()
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None, "no traffic capture committed"
    for ln in lines:
        if not ln.startswith("bench-traffic:"):
            continue
        kv = dict(t.split("=", 1) for t in ln.split()[1:] if "=" in t)
        if kv.get("kernel") != kernel:
            continue
        if kv.get("source") != sha:
            return None, "capture of an older kernel source (%s, now %s): recapture" % (kv.get("source"), sha)
        return float(kv["dram_bytes_per_launch"]), "profiles/legendre_traffic_des2048.md (source %s)" % sha
    return None, "no capture of %s in profiles/legendre_traffic_des2048.md" % kernel


class ClockSampler:
    """nvidia-smi samples (SM clock, throttle reasons) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def replica_noise(wl, rank):
    """Shape noise of one rank's replica: rank 0 solves the workload's own realisation, rank r > 0
    an independent one (seed 10000 + r), so replicas never repeat each other's data."""
    import synthetic as S

    if rank == 0:
        return wl["noise"]
    return S.shape_noise(wl["ninv"], np.random.default_rng(10_000 + rank))[0]


def whole_job(elapsed, applies, world, device=None):
    """Whole-job numbers of a replicated run: (slowest rank's time, H applications of all ranks).
    Collectives on the default process group (NCCL on GPUs; any backend works)."""
    if world == 1:
        return elapsed, float(applies)
    import torch
    import torch.distributed as dist

    tt = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    aa = torch.tensor([float(applies)], dtype=torch.float64, device=device)
    dist.all_reduce(aa, op=dist.ReduceOp.SUM)
    return float(tt), float(aa)


def make_inputs(rank, dev, name="des2048"):
    """A named DES-like workload (seeded), shear y = M (A x_true + n) formed with our FP64 forward
    operator (input preparation, not timed)."""
    import torch

    import synthetic as S
    from paper_2606_06175_gb300 import akra as A

    wl = S.workload(name)
    plan = A.akra_plan_create(wl["nside"], wl["lmax"])
    ninv = torch.from_numpy(wl["ninv"]).to(dev)
    A.akra_plan_set_weights(plan, ninv, 1e-3)
    x_true = torch.from_numpy(np.stack(wl["x_true"])[None]).to(dev)
    y = A.akra_apply_A(plan, A.F64, x_true)
    noise = replica_noise(wl, rank)
    y += torch.from_numpy(noise[None]).to(dev)
    y *= (ninv > 0).to(y.dtype)
    torch.cuda.synchronize()
    return plan, y, wl


def timed_solve(A, plan, prec, y, tol, maxiter=20000):
    """One blocking solve, wall-clock seconds around it (device synchronised on both sides)."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, info = A.akra_cg_solve(plan, prec, y, tol=tol, maxiter=maxiter)
    torch.cuda.synchronize()
    return x, info, time.perf_counter() - t0


def rel_err(a, b):
    import torch

    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def solve_summary(info, seconds):
    d = {"solve_s": seconds, "iters": info["iters"], "relres": info["relres"], "status": info["status"]}
    if info["outer"]:
        d.update({"outer": info["outer"], "h_applies_f64": info["h_applies_f64"]})
    return d


def fp64_vs_mixed(A, plan, y, x_mixed, mixed_s, mixed_info, f64_reference):
    """The plain FP64 GPU CG solve of the same system to TOL (measured), and the errors of both
    solutions against a reference solved to an FP64 residual of REF_TOL: a plain FP64 CG solve
    when f64_reference, else a mixed solve (its outer residual b - H x is evaluated in FP64, so
    it meets the same FP64 residual bound)."""
    A.akra_cg_solve(plan, A.F64, y, tol=1e-2, maxiter=3)          # graph capture, untimed
    x64, i64, t64 = timed_solve(A, plan, A.F64, y, TOL)
    xr, ir, tr = timed_solve(A, plan, A.F64 if f64_reference else A.MIXED, y, REF_TOL)
    # solution error <= κ x residual: the mixed solve run to 1e-8 shows what a solution error
    # below 1e-6 costs
    xm8, im8, tm8 = timed_solve(A, plan, A.MIXED, y, 1e-8)
    e_m, e_64 = rel_err(x_mixed, xr), rel_err(x64, xr)
    return {
        "fp64": solve_summary(i64, t64),
        "mixed": solve_summary(mixed_info, mixed_s),
        "mixed_speedup_vs_fp64": t64 / mixed_s,
        "reference": dict(solve_summary(ir, tr), how="%s solve to FP64 residual %g"
                          % ("plain FP64 CG" if f64_reference else "mixed (FP64 outer residual)", REF_TOL)),
        "rel_err_mixed_vs_reference": e_m,
        "rel_err_fp64_vs_reference": e_64,
        "rel_err_mixed_vs_fp64": rel_err(x_mixed, x64),
        "error_over_residual": {"mixed": e_m / max(mixed_info["relres"], 1e-300),
                                "fp64": e_64 / max(i64["relres"], 1e-300)},
        "mixed_tol_1e-8": dict(solve_summary(im8, tm8), rel_err_vs_reference=rel_err(xm8, xr)),
    }, x64, xr


def config2_block(A, dev):
    """Nside 512 / lmax 1024, DES-like footprint (seed 1002), single RHS: FP64 and mixed solves to
    1e-6, errors against a plain FP64 solve to 1e-10 (and the mixed 1e-10 solve against it)."""
    plan, y, wl = make_inputs(0, dev, "des512")
    A.akra_autotune(plan, A.MIXED, 1)
    A.akra_cg_solve(plan, A.MIXED, y, tol=TOL, maxiter=6000)       # graph capture, untimed
    xm, im, tm = timed_solve(A, plan, A.MIXED, y, TOL)
    out, x64, xr = fp64_vs_mixed(A, plan, y, xm, tm, im, f64_reference=True)
    xm10, im10, tm10 = timed_solve(A, plan, A.MIXED, y, REF_TOL)
    out["mixed_to_reference_tol"] = solve_summary(im10, tm10)
    out["rel_err_mixed_1e-10_vs_fp64_1e-10"] = rel_err(xm10, xr)
    out["workload"] = "des512: Nside 512, lmax 1024, DES-like footprint, seed 1002, tol 1e-6"
    A.akra_plan_destroy(plan)
    return out


def batch_uneven_block(A, dev):
    """BASELINE config 4: 32 RHS at Nside 1024 / lmax 2048, 16 at 512 / 1024, 16 at 256 / 512
    (DES-like footprints, per-pixel Gaussian shape-noise realisations) in one batched mixed solve
    with persistent work-queue Legendre launches; tile shape and the tensor-core synthesis group
    autotuned."""
    import torch

    import synthetic as S

    spec = [(1024, 2048, 32), (512, 1024, 16), (256, 512, 16)]
    bplans, bshears = [], []
    for k, (nb, lb, rb) in enumerate(spec):
        svb = S.survey(nb, "des", S.SEEDS["batch"] + k)
        pb = A.akra_plan_create(nb, lb)
        A.akra_plan_set_weights(pb, torch.from_numpy(svb["ninv"]).to(dev), 1e-3)
        bplans.append(pb)
        bshears.append(torch.from_numpy(S.shape_noise(svb["ninv"], svb["rng_noise"], nreal=rb)).to(dev))
    bt = A.akra_batch_create(bplans, [r for *_, r in spec])
    A.akra_batch_autotune(bt)
    A.akra_batch_cg_solve(bt, A.MIXED, bshears, tol=TOL, maxiter=3000)   # graph capture, untimed
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, binfos = A.akra_batch_cg_solve(bt, A.MIXED, bshears, tol=TOL, maxiter=3000)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    nrhs = sum(r for *_, r in spec)
    out = {"instances": [{"nside": nb, "lmax": lb, "rhs": rb} for nb, lb, rb in spec], "rhs": nrhs,
           "solve_s": t_b, "s_per_rhs": t_b / nrhs,
           "inner_iters": [i["iters"] for i in binfos], "outer": [i["outer"] for i in binfos],
           "max_relres": max(max(i["relres_rhs"]) for i in binfos),
           "status": max(i["status"] for i in binfos), "tile": A.akra_batch_describe(bt),
           "tc_synthesis_group": A.akra_batch_get_tc_synthesis(bt)}
    del bt
    for pb in bplans:
        A.akra_plan_destroy(pb)
    return out


def differentiation_block(A, dev):
    """BASELINE config 5: Nside 512 / lmax 1024 (seed 1005); the loss is the sum of the E-mode
    band powers of the reconstruction in 8 log bins over 10 < l < 1024, differentiated through
    the CG solve (implicit adjoint solve) w.r.t. the float32 shear maps and N^-1.  Forward +
    backward time per precision, and the mixed gradients' relative difference from FP64."""
    import torch

    from paper_2606_06175_gb300.autograd import akra_solve, band_power_loss

    plan, y, wl = make_inputs(0, dev, "grad512")
    L = wl["lmax"]
    y32 = y[0].float()
    ninv = torch.from_numpy(wl["ninv"]).to(dev)
    edges = np.geomspace(10, 1024, 9)
    out, grads = {}, {}
    for name, prec in (("fp64", A.F64), ("mixed", A.MIXED)):
        for rep in range(2):   # the first run captures the graphs
            yt = y32.clone().requires_grad_(True)
            nt = ninv.clone().requires_grad_(True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = band_power_loss(akra_solve(yt, nt, plan, prec, tol=TOL, maxiter=6000), L, edges)
            loss.backward()
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
        grads[name] = (yt.grad.double(), nt.grad.double())
        out[name] = {"forward_backward_s": dt, "loss": float(loss.detach())}
    out["rel_diff_mixed_vs_fp64_grad_y"] = rel_err(grads["mixed"][0], grads["fp64"][0])
    out["rel_diff_mixed_vs_fp64_grad_ninv"] = rel_err(grads["mixed"][1], grads["fp64"][1])
    out["workload"] = "grad512: Nside 512, lmax 1024, DES-like footprint, seed 1005, tol 1e-6"
    A.akra_plan_destroy(plan)
    return out


def legendre_flops(desc, R=1):
    """Work of one FP32 Legendre launch over the active ring pairs.

    Unit: one (l, m, ring pair) step.  The hot-path model counts 2 spin recurrences x 3 FMA
    plus 4 FMA of contraction per RHS: (6 + 4R) FMA = 2 (6 + 4R) flops per step.  The kernels
    execute a monic recurrence of 2 x 2 FMA and a contraction of 8 FMA per RHS for pairs that
    need both rings, 4 for pairs that need one (the one-ring contraction): (4 + 8R) or (4 + 4R)
    FMA per step; both counts are returned.  Steps counted: for each (m, pair) from where its
    harmonics first exceed 2^-40 (the plan's start table) to lmax; the full triangle (every
    l >= 2) is returned as well."""
    steps = desc["legendre_steps_f32"]
    one = desc.get("legendre_steps_f32_one_ring", 0)
    full = desc["n_active_units"] * (desc["ntri"] - 3)
    return {"steps": steps, "steps_one_ring": one, "steps_full_triangle": full,
            "model_flops": steps * (6 + 4 * R) * 2, "model_flops_full_triangle": full * (6 + 4 * R) * 2,
            "executed_flops": ((steps - one) * (4 + 8 * R) + one * (4 + 4 * R)) * 2}


def cpu_oracle_H_estimate(nside, lmax, target_s=15.0):
    """Time the FP64 CPU oracle on a bounded sample of one full H application at (nside, lmax)
    and extrapolate: Legendre synthesis on a sample of rings, the adjoint on a sample of m
    columns, numpy ring DFTs on a sample of rings."""
    from oracle import oracle as O

    O.build()
    th = O.num_threads()
    nring = 4 * nside - 1
    rng = np.random.default_rng(0)
    nt = O.ntri(lmax)
    aE = rng.normal(size=nt) + 1j * rng.normal(size=nt)
    aB = rng.normal(size=nt) + 1j * rng.normal(size=nt)
    nr = max(2 * th, 8)
    rings = np.linspace(1, nring, nr).astype(np.int32)
    t0 = time.perf_counter()
    F = O.legendre_synth(nside, lmax, aE, aB, rings)
    t_syn = time.perf_counter() - t0
    # per-ring phase sums (numpy) on a sample of ring lengths
    t0 = time.perf_counter()
    nfft = 0
    for k, r in enumerate(rings):
        ct, st, n, sg, first = O.ring_info(nside, int(r))
        f = O.ring_phase_sum(F[k], lmax, n, sg)
        O.ring_phase_adjoint(f, lmax, sg)
        nfft += 1
    t_fft = (time.perf_counter() - t0) / nfft
    # adjoint Legendre on a sample of m columns (cost ∝ lmax - m + 1)
    nm = max(th, 4)
    ms = np.linspace(0, lmax, nm).astype(np.int32)
    G = np.ascontiguousarray(np.repeat(F[:1], nring, axis=0))
    g = np.zeros(nt, np.complex128)
    h = np.zeros(nt, np.complex128)
    t0 = time.perf_counter()
    O._lib().orc_legendre_adjoint(nside, lmax, O._dptr(G.view(np.float64)), len(ms), O._iptr(ms),
                                  O._dptr(g.view(np.float64)), O._dptr(h.view(np.float64)))
    t_adj = time.perf_counter() - t0
    t_H = t_syn * nring / nr + t_adj * (lmax + 1) / nm + t_fft * nring
    sample = ("FP64 oracle on %d of %d rings (Legendre synthesis), %d of %d m-columns "
              "(adjoint), %d ring DFT pairs; extrapolated to one H application at Nside %d, "
              "lmax %d (the oracle transforms every ring)" % (nr, nring, nm, lmax + 1, nfft, nside, lmax))
    return t_H, th, sample, t_syn + t_adj + t_fft * nfft


def run_reference(args, rank, world):
    """The reference arm: the FP64 CPU oracle (there is no reference implementation of this
    method).  A full oracle H application at Nside 2048 / lmax 4096 takes minutes on the host, so
    each step times the oracle on a bounded sample of one H application and extrapolates to the
    whole H; the line says so (`extrapolated`), and ms_per_step is the wall time a step really
    took (its sample), so steps x ms_per_step is the work actually done."""
    if rank != 0:
        return
    vals, spent = [], []
    for _ in range(args.warmup):
        cpu_oracle_H_estimate(NSIDE, LMAX)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        t_H, th, sample, _ = cpu_oracle_H_estimate(NSIDE, LMAX)
        spent.append(time.perf_counter() - t0)
        vals.append(1.0 / t_H)
    v = statistics.median(vals)
    step_s = statistics.median(spent)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "des2048: Nside 2048, lmax 4096, DES-like 4123 deg2 footprint, "
                                   "one H application (the oracle is FP64 only)"},
            "extrapolated": True,
            "extrapolation": "value = 1 / (oracle time of one whole H application, extrapolated from "
                             "the sample each step times); ms_per_step = measured wall time of one "
                             "step's sample, not of a whole H",
            "h_apply_s_extrapolated": 1.0 / v, "sample_s_per_step": step_s,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample,
                             "extrapolated": True},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the untimed comparison blocks (FP64 solve and solution errors, the "
                         "Nside 512, batched and differentiation workloads)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fields", action="store_true",
                    help="also time the E-only solve and the conditional B-mode solve (App. A)")
    ap.add_argument("--flat", type=int, default=0, metavar="N",
                    help="also time the flat-sky variant on an N x N grid (mixed solve, H applies)")
    ap.add_argument("--per-l-precond", action="store_true",
                    help="also time the mixed solve with the per-l diagonal preconditioner")
    ap.add_argument("--noise-realisations", type=int, default=0, metavar="K",
                    help="also time the shuffled-noise pipeline with K realisations in one batched solve")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    from paper_2606_06175_gb300 import akra as A

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    plan, y, wl = make_inputs(rank, dev)
    A.akra_autotune(plan, A.MIXED, 1)
    desc = A.akra_plan_describe(plan)
    x = torch.empty((1, 2, plan.ntri), dtype=torch.complex128, device=dev)
    for _ in range(args.warmup):
        A.akra_cg_solve(plan, A.MIXED, y, x, tol=TOL, maxiter=2000)
    torch.cuda.synchronize()

    # ---- timed region: K mixed-precision solves, inputs resident in HBM ----
    infos = []
    barrier()
    torch.cuda.synchronize()
    launches0 = A.akra_plan_describe(plan)["kernel_launches"]
    print("timed region starts after %d libakra kernel launches" % launches0, file=sys.stderr, flush=True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record()
        for _ in range(args.steps):
            _, info = A.akra_cg_solve(plan, A.MIXED, y, x, tol=TOL, maxiter=2000)
            infos.append(info)
        ev1.record()
        torch.cuda.synchronize()
    barrier()
    launches = A.akra_plan_describe(plan)["kernel_launches"] - launches0
    elapsed = ev0.elapsed_time(ev1) / 1e3
    applies = sum(i["h_applies_f32"] + i["h_applies_f64"] for i in infos)
    t_max, applies_all = whole_job(elapsed, applies, world, dev)
    value = applies_all / t_max
    ms_per_step = 1e3 * t_max / args.steps
    last = infos[-1]

    # ---- per-stage kernel timing (CUDA events on this stream, kernels timed alone) ----
    st32 = A.akra_time_H_stages(plan, A.F32, 1, 5)
    st64 = A.akra_time_H_stages(plan, A.F64, 1, 2)

    # ---- one inner iteration inside the captured graph: a fixed-length FP32 CG, event-timed ----
    b32 = x.to(torch.complex64)
    A.akra_cg_solve_b(plan, A.F32, b32, tol=1e-30, maxiter=2)          # graph already captured
    n_it = 40
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    _, inf_it = A.akra_cg_solve_b(plan, A.F32, b32, tol=1e-30, maxiter=n_it)
    e1.record()
    torch.cuda.synchronize()
    per_iter_ms = e0.elapsed_time(e1) / inf_it["iters"]
    # the same from the solve: (solve time - its FP64 work) / inner iterations, with the FP64
    # work = (FP64 H applications - 1) whole H + one A^T (b), from the stage times
    t_at64 = st64["ring_fft"] + st64["legendre_adjoint"] + st64["epilogue"]
    f64_ms = (last["h_applies_f64"] - 1) * st64["total"] + t_at64
    per_iter_derived = (ms_per_step - f64_ms) / max(last["iters"], 1)

    # ---- roofline of the dominant kernel (FP32 Legendre) ----
    props = torch.cuda.get_device_properties(dev)
    sm_count = props.multi_processor_count
    clocks = clk.summary()
    sm_max = clocks.get("sm_max_mhz") or _sm_max_mhz()
    peak = fp32_peak_tflops(sm_count, sm_max)
    work = legendre_flops(desc)
    dom = "legendre_adjoint" if st32["legendre_adjoint"] >= st32["legendre_synth"] else "legendre_synth"
    kname = {"legendre_adjoint": "k_leg_adjoint<float>", "legendre_synth": "k_leg_synth<float>"}[dom]
    shape = A.akra_plan_get_shape(plan, A.F32, 1)
    rga = A.akra_plan_get_adjoint_shape(plan, A.F32, 1)["RGA"]
    kfull = "%s<float,%d,%d,128>" % ("k_leg_adjoint" if dom == "legendre_adjoint" else "k_leg_synth",
                                     shape["PA"] if dom == "legendre_adjoint" else shape["P"],
                                     rga if dom == "legendre_adjoint" else shape["RG"])
    achieved = work["model_flops"] / (st32[dom] * 1e-3) / 1e12
    traffic, traffic_note = captured_traffic(kfull)
    f32_meas = A.akra_fma_rate(A.F32)
    f64_meas = A.akra_fma_rate(A.F64)
    flops64 = desc["legendre_steps_f64"] * (6 + 4) * 2
    one64 = desc.get("legendre_steps_f64_one_ring", 0)
    exec64 = ((desc["legendre_steps_f64"] - one64) * (4 + 8) + one64 * (4 + 4)) * 2
    roofline = {
        "bound": "alu", "kernel": kname, "launch_shape": kfull,
        "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
        "traffic": traffic, "traffic_source": traffic_note,
        "peak_basis": "%d SMs (device) x 128 FP32 lanes x 2 flops x %.0f MHz (maximum SM clock)" % (sm_count, sm_max),
        "work_basis": "(6 + 4R) FMA = 2 (6 + 4R) flops per (l, m, ring pair) step at R = 1 (two 3-FMA spin "
                      "recurrences + 4 FMA contraction), over the steps of the plan's start table",
        "flops_per_launch": work["model_flops"], "lm_pair_steps_per_launch": work["steps"],
        "lm_pair_steps_full_triangle": work["steps_full_triangle"],
        "achieved_full_triangle": work["model_flops_full_triangle"] / (st32[dom] * 1e-3) / 1e12,
        "executed": {"flops_per_launch": work["executed_flops"],
                     "basis": "FMA per step as executed: monic recurrence 2 x 2 FMA; contraction of both "
                              "rings' E and B parts 8 FMA per RHS, 4 for pairs that need one ring (%d of %d "
                              "steps here)" % (work["steps_one_ring"], work["steps"]),
                     "achieved": work["executed_flops"] / (st32[dom] * 1e-3) / 1e12,
                     "frac": work["executed_flops"] / (st32[dom] * 1e-3) / 1e12 / peak},
        "measured_fma_tflops": {"fp32": f32_meas, "fp64": f64_meas},
        "frac_of_measured_fp32": achieved / f32_meas,
        "stage_ms_fp32": st32, "stage_ms_fp64": st64,
        "lm_pair_steps_per_launch_fp64": desc["legendre_steps_f64"],
        "fp32_legendre": {k: {"ms": st32[k], "achieved": work["model_flops"] / (st32[k] * 1e-3) / 1e12,
                              "frac": work["model_flops"] / (st32[k] * 1e-3) / 1e12 / peak}
                          for k in ("legendre_synth", "legendre_adjoint")},
        # FP64 on the same (6 + 4R) model and on the executed FMA (monic recurrence 2 x 2, 8 per
        # RHS for pairs needing both rings, 4 for one-ring pairs): the model can exceed the FP64
        # peak once the one-ring contraction executes fewer FMA than it counts
        "fp64_legendre": {k: {"ms": st64[k], "achieved": flops64 / (st64[k] * 1e-3) / 1e12,
                              "frac_of_nominal_fp64": flops64 / (st64[k] * 1e-3) / 1e12 / 1.25,
                              "executed_achieved": exec64 / (st64[k] * 1e-3) / 1e12,
                              "executed_frac_of_nominal_fp64": exec64 / (st64[k] * 1e-3) / 1e12 / 1.25}
                          for k in ("legendre_synth", "legendre_adjoint")},
        # counted steps / lane-steps the warps execute at the chosen shapes (start-point spread
        # within a warp and 64-step tile granularity)
        "lane_efficiency": {
            "legendre_synth": A.akra_legendre_lane_steps(plan, A.F32, False, shape["P"])["efficiency"],
            "legendre_adjoint": A.akra_legendre_lane_steps(plan, A.F32, True, shape["PA"])["efficiency"]},
    }

    # ---- untimed comparison blocks ----
    compare = cfg2 = batch = grad = None
    if not args.headline_only:
        xm = x.clone()
        compare, _, _ = fp64_vs_mixed(A, plan, y, xm, ms_per_step / 1e3, last, f64_reference=False)
        compare["fp64"]["h_apply_ms"] = st64["total"]
        compare["fp32_h_apply_ms"] = st32["total"]
        cfg2 = config2_block(A, dev)
        batch = batch_uneven_block(A, dev)
        grad = differentiation_block(A, dev)

    # ---- field-restricted solves (App. A), same workload and tolerance ----
    fields = None
    if args.fields:
        xf = torch.empty_like(x)
        A.akra_cg_solve_fields(plan, A.MIXED, A.SOLVE_E, y, xf, tol=TOL, maxiter=2000)   # capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ie = A.akra_cg_solve_fields(plan, A.MIXED, A.SOLVE_E, y, xf, tol=TOL, maxiter=2000)
        torch.cuda.synchronize()
        t_e = time.perf_counter() - t0
        A.akra_cg_solve_fields(plan, A.MIXED, A.SOLVE_B_GIVEN_E, y, xf.clone(), tol=TOL, maxiter=2000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ib = A.akra_cg_solve_fields(plan, A.MIXED, A.SOLVE_B_GIVEN_E, y, xf, tol=TOL, maxiter=2000)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        fields = {"e_only": solve_summary(ie, t_e), "b_given_e": solve_summary(ib, t_b)}

    # ---- the per-l diagonal preconditioner (beyond the paper's scalar Eq. 15) ----
    per_l = None
    if args.per_l_precond:
        A.akra_plan_set_preconditioner(plan, A.PRECOND_PER_L)
        A.akra_cg_solve(plan, A.MIXED, y, torch.empty_like(x), tol=TOL, maxiter=2000)   # capture
        _, ip, t_p = timed_solve(A, plan, A.MIXED, y, TOL, 2000)
        per_l = solve_summary(ip, t_p)
        A.akra_plan_set_preconditioner(plan, A.PRECOND_SCALAR)

    # ---- flat-sky variant (2D FFTs in place of the SHTs): N x N DES-like patch ----
    flat = None
    if args.flat > 0:
        import synthetic as S
        nf = args.flat
        sv = S.flat_survey(nf)
        fp = A.akra_flat_plan_create(nf)
        ninv_f = torch.from_numpy(sv["ninv"]).to(dev)
        A.akra_plan_set_weights(fp, ninv_f, 1e-3)
        xt = torch.from_numpy(sv["x_true"][None]).to(dev)
        yf = A.akra_apply_A(fp, A.F64, xt)
        yf += torch.from_numpy(sv["noise"][None]).to(dev)
        yf *= (ninv_f > 0).to(yf.dtype)
        A.akra_cg_solve(fp, A.MIXED, yf, tol=TOL, maxiter=3000)   # capture
        _, inf_f, t_f = timed_solve(A, fp, A.MIXED, yf, TOL, 3000)
        h_ms = {}
        for pr, nm in ((A.F32, "fp32"), (A.F64, "fp64")):
            xx = xt.to(torch.complex64) if pr == A.F32 else xt
            yy = A.akra_apply_H(fp, pr, xx)
            for _ in range(3):
                A.akra_apply_H(fp, pr, xx, yy)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(10):
                A.akra_apply_H(fp, pr, xx, yy)
            e1.record()
            torch.cuda.synchronize()
            h_ms[nm] = e0.elapsed_time(e1) / 10
        # HBM traffic of one H: 5 passes over the complex field (row FFT in/out, 2 transposes,
        # fused middle pass, last pass reading x for the λ_eff term) + the weights
        cb = {"fp32": 8, "fp64": 16}
        trf = {k: (11 * cb[k] + cb[k] // 2) * nf * nf for k in cb}
        hbm = {k: trf[k] / (h_ms[k] * 1e-3) / 1e9 for k in cb}
        flat = dict(solve_summary(inf_f, t_f), n=nf, pixels=nf * nf, h_apply_ms=h_ms, h_traffic_bytes=trf,
                    h_achieved_gbs=hbm, h_frac_of_hbm={k: hbm[k] / HBM_GBS for k in hbm})
        A.akra_plan_destroy(fp)

    # ---- noise-realisation pipeline (Sec. IV): K shuffled maps as the RHS of one solve ----
    noise = None
    if args.noise_realisations > 0:
        from paper_2606_06175_gb300 import spectra as SP
        K = args.noise_realisations
        perms = SP.shuffle_permutations(wl["mask"], K, seed=2024)
        A.akra_autotune(plan, A.MIXED, K)
        SP.noise_realisations(plan, A.MIXED, y[0], perms, tol=TOL, maxiter=2000)   # capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bp, _, inf = SP.noise_realisations(plan, A.MIXED, y[0], perms, tol=TOL, maxiter=2000)
        torch.cuda.synchronize()
        t_n = time.perf_counter() - t0
        noise = {"realisations": K, "total_s": t_n, "s_per_realisation": t_n / K,
                 "inner_iters": inf["iters"], "outer": inf["outer"], "relres": inf["relres"],
                 "shape_f32": A.akra_plan_get_shape(plan, A.F32, K),
                 "noise_bias_EE_band_powers": SP.noise_bias(bp)[0][0].cpu().tolist()}

    # ---- end to end through the C ABI with host buffers ----
    y_host = y.cpu().pin_memory()
    x_host = torch.empty(x.shape, dtype=x.dtype).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    y_dev = y_host.to(dev, non_blocking=True)
    _, info_e = A.akra_cg_solve(plan, A.MIXED, y_dev, x, tol=TOL, maxiter=2000)
    x_host.copy_(x, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e_applies = info_e["h_applies_f32"] + info_e["h_applies_f64"]
    e2e = {"value": e2e_applies / t_e2e, "unit": UNIT, "h2d_bytes_per_step": y_host.numel() * 8,
           "d2h_bytes_per_step": x_host.numel() * 16, "solve_s": t_e2e}

    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        t_H, th, sample, _ = cpu_oracle_H_estimate(NSIDE, LMAX)
        cpu = {"value": 1.0 / t_H, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample,
               "extrapolated": True, "h_apply_s_extrapolated": t_H}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "des2048: Nside 2048, lmax 4096, DES-like footprint %.0f deg2, "
                               "mixed FP32-inner/FP64-refinement PCG to rel.res 1e-6"
                               % (float(np.mean(wl["mask"])) * 41252.96),
                   "nside": NSIDE, "lmax": LMAX, "tol": TOL, "rhs": 1,
                   "active_rings": desc["n_active_rings"], "active_ring_pairs": desc["n_active_units"],
                   "l2": "inputs larger than L2 (FP64 shear maps 805 MB, phase array 0.5-1.1 GB per H)"},
        "note": "value counts FP32 and FP64 H applications alike; the solve time (ms_per_step) is the "
                "number to compare",
        "cg": {"solve_s": ms_per_step / 1e3, "inner_iters": last["iters"], "outer": last["outer"],
               "h_applies_f32": last["h_applies_f32"], "h_applies_f64": last["h_applies_f64"],
               "relres": last["relres"], "per_inner_iter_ms": per_iter_ms,
               "per_inner_iter_basis": "%d-iteration FP32 CG replaying the captured iteration graph, CUDA events"
                                       % inf_it["iters"],
               "per_inner_iter_ms_from_solve": per_iter_derived},
        "fp64_vs_mixed": compare,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clocks,
    }
    if cfg2 is not None:
        line["config2_des512"] = cfg2
    if batch is not None:
        line["batch_uneven"] = batch
    if grad is not None:
        line["differentiation_grad512"] = grad
    if fields is not None:
        line["fields"] = fields
    if noise is not None:
        line["noise_realisations"] = noise
    if per_l is not None:
        line["per_l_preconditioner"] = per_l
    if flat is not None:
        line["flat_sky"] = flat
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
