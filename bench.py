#!/usr/bin/env python
"""Benchmark of the AKRA 3.0 hot path on GB300.

One step = one mixed-precision PCG solve (FP32 inner CG, FP64 outer refinement) of the
regularised normal equations at Nside 2048, lmax 4096 on a synthetic DES-like footprint, to
relative residual 1e-6 -- every H application inside it runs the full chain (KS,
spin-2 synthesis, ring FFT x W x FFT, exact adjoint, epilogue) in libakra.so.

Metric (as named): "H-applies/s and CG solve time at Nside=2048 (mixed vs FP64, rel.res 1e-6)";
`value` = H applications (FP32 inner + FP64 outer + the FP64 A^T of b) per second over the
timed solves, whole job (summed over ranks); ms_per_step = the CG solve time.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def _hbm_gbs():
    """Measured copy bandwidth of the GB300s (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return 6800.0


HBM_GBS = _hbm_gbs()


def fp32_peak_tflops(mhz=SM_MAX_MHZ):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock
    return SM_COUNT * FP32_LANES * 2 * mhz * 1e6 / 1e12


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


def make_inputs(rank, dev):
    """des2048 workload (seeded), shear y = M (A x_true + n) formed with our FP64 forward operator."""
    import torch

    import synthetic as S
    from paper_2606_06175_gb300 import akra as A

    wl = S.workload("des2048")
    plan = A.akra_plan_create(NSIDE, LMAX)
    ninv = torch.from_numpy(wl["ninv"]).to(dev)
    A.akra_plan_set_weights(plan, ninv, 1e-3)
    x_true = torch.from_numpy(np.stack(wl["x_true"])[None]).to(dev)
    y = A.akra_apply_A(plan, A.F64, x_true)
    noise = replica_noise(wl, rank)
    y += torch.from_numpy(noise[None]).to(dev)
    y *= (ninv > 0).to(y.dtype)
    torch.cuda.synchronize()
    return plan, y, wl


def legendre_flops(desc, R=1):
    """FP32 work of one Legendre launch over the active ring pairs: every (l, m, pair) step
    does two monic spin recurrences (4 FMA) and 8 FMA of contraction per RHS; flops = 2 x FMA.
    The steps counted are those the method needs: for each (m, pair) from where its harmonics
    first exceed 2^-40 (the plan's start table) to lmax.  The full triangle (every l >= 2) is
    returned as well."""
    steps = desc["legendre_steps_f32"]
    full = desc["n_active_units"] * (desc["ntri"] - 3)
    return steps * (4 + 8 * R) * 2, steps, full


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
    if rank != 0:
        return
    vals = []
    t_total = 0.0
    for _ in range(args.warmup):
        cpu_oracle_H_estimate(NSIDE, LMAX)
    for _ in range(args.steps):
        t_H, th, sample, spent = cpu_oracle_H_estimate(NSIDE, LMAX)
        vals.append(1.0 / t_H)
        t_total += spent
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "des2048: Nside 2048, lmax 4096, DES-like 4123 deg2 footprint, "
                                   "one H application (the oracle is FP64 only)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-solve", action="store_true", help="also run one full FP64 CG solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fields", action="store_true",
                    help="also time the E-only solve and the conditional B-mode solve (App. A)")
    ap.add_argument("--batch-uneven", action="store_true",
                    help="also time the batched uneven-instance solve: 32 RHS at Nside 1024 / lmax 2048, "
                         "16 at 512 / 1024, 16 at 256 / 512, one batched mixed solve")
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

    # ---- per-stage kernel timing (CUDA events on this stream, kernels timed alone) ----
    st32 = A.akra_time_H_stages(plan, A.F32, 1, 5)
    st64 = A.akra_time_H_stages(plan, A.F64, 1, 2)
    flops, steps, full_steps = legendre_flops(desc)
    dom = "legendre_adjoint" if st32["legendre_adjoint"] >= st32["legendre_synth"] else "legendre_synth"
    achieved = flops / (st32[dom] * 1e-3) / 1e12
    peak = fp32_peak_tflops()
    roofline = {"bound": "alu", "kernel": "k_leg_adjoint<float>" if dom == "legendre_adjoint" else "k_leg_synth<float>",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                # DRAM bytes of one launch of the dominant kernel (k_leg_adjoint<float, 4, 1, 128>)
                # read from an ncu capture (1-pass dram__bytes metrics) at this workload
                "traffic": 574.87e6 + 786.99e6,
                "peak_basis": "152 SMs x 128 FP32 lanes x 2 flops x 2070 MHz (unit counts and maximum clock)",
                "flops_per_launch": flops, "lm_pair_steps_per_launch": steps,
                "lm_pair_steps_full_triangle": full_steps,
                "lm_pair_steps_per_launch_fp64": desc["legendre_steps_f64"],
                "stage_ms_fp32": st32, "stage_ms_fp64": st64}
    # measured FMA rates (saturating FMA-chain kernel on this GPU) beside the nominal peak
    f32_meas = A.akra_fma_rate(A.F32)
    f64_meas = A.akra_fma_rate(A.F64)
    flops64 = desc["legendre_steps_f64"] * (4 + 8) * 2
    roofline["measured_fma_tflops"] = {"fp32": f32_meas, "fp64": f64_meas}
    roofline["frac_of_measured_fp32"] = achieved / f32_meas
    roofline["fp64_legendre"] = {
        k: {"achieved": flops64 / (st64[k] * 1e-3) / 1e12,
            "frac_of_measured_fp64": flops64 / (st64[k] * 1e-3) / 1e12 / f64_meas}
        for k in ("legendre_synth", "legendre_adjoint")}
    roofline["fp32_legendre"] = {
        k: {"achieved": flops / (st32[k] * 1e-3) / 1e12,
            "frac_of_measured_fp32": flops / (st32[k] * 1e-3) / 1e12 / f32_meas}
        for k in ("legendre_synth", "legendre_adjoint")}

    # ---- FP64 comparison (the plain FP64 GPU path) ----
    t_h64 = st64["total"] * 1e-3
    inner = infos[-1]["iters"]
    fp64 = {"h_applies_per_s": 1.0 / t_h64, "h_apply_ms": st64["total"],
            "fp32_h_apply_ms": st32["total"]}
    if args.fp64_solve:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, info64 = A.akra_cg_solve(plan, A.F64, y, x, tol=TOL, maxiter=3000)
        torch.cuda.synchronize()
        fp64.update({"cg_solve_s": time.perf_counter() - t0, "cg_iters": info64["iters"],
                     "relres": info64["relres"]})
    else:
        # FP64 CG needs about as many iterations as the FP32 inner CG took to reach the same
        # residual; this is labelled as an extrapolation
        fp64["cg_solve_s_extrapolated"] = (inner + 1) * t_h64
        fp64["extrapolation"] = "FP64 H time x (mixed inner iterations + 1)"

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
        fields = {"e_only": {"solve_s": t_e, "inner_iters": ie["iters"], "outer": ie["outer"],
                             "h_applies_f64": ie["h_applies_f64"], "relres": ie["relres"]},
                  "b_given_e": {"solve_s": t_b, "inner_iters": ib["iters"], "outer": ib["outer"],
                                "h_applies_f64": ib["h_applies_f64"], "relres": ib["relres"]}}

    # ---- the per-l diagonal preconditioner (beyond the paper's scalar Eq. 15) ----
    per_l = None
    if args.per_l_precond:
        A.akra_plan_set_preconditioner(plan, A.PRECOND_PER_L)
        xp = torch.empty_like(x)
        A.akra_cg_solve(plan, A.MIXED, y, xp, tol=TOL, maxiter=2000)   # capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ip = A.akra_cg_solve(plan, A.MIXED, y, xp, tol=TOL, maxiter=2000)
        torch.cuda.synchronize()
        per_l = {"solve_s": time.perf_counter() - t0, "inner_iters": ip["iters"], "outer": ip["outer"],
                 "relres": ip["relres"]}
        A.akra_plan_set_preconditioner(plan, A.PRECOND_SCALAR)

    # ---- batched uneven instances in one persistent launch per step ----
    batch = None
    if args.batch_uneven:
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
        A.akra_batch_cg_solve(bt, A.MIXED, bshears, tol=TOL, maxiter=3000)   # capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, binfos = A.akra_batch_cg_solve(bt, A.MIXED, bshears, tol=TOL, maxiter=3000)
        torch.cuda.synchronize()
        t_b = time.perf_counter() - t0
        nrhs = sum(r for *_, r in spec)
        batch = {"instances": [{"nside": nb, "lmax": lb, "rhs": rb} for nb, lb, rb in spec], "rhs": nrhs,
                 "solve_s": t_b, "s_per_rhs": t_b / nrhs,
                 "inner_iters": [i["iters"] for i in binfos], "outer": [i["outer"] for i in binfos],
                 "max_relres": max(max(i["relres_rhs"]) for i in binfos),
                 "tile": A.akra_batch_describe(bt)}
        del bt, bplans, bshears

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
        xf = torch.empty_like(xt)
        A.akra_cg_solve(fp, A.MIXED, yf, xf, tol=TOL, maxiter=3000)   # capture
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, inf_f = A.akra_cg_solve(fp, A.MIXED, yf, xf, tol=TOL, maxiter=3000)
        torch.cuda.synchronize()
        t_f = time.perf_counter() - t0
        h_ms = {}
        for pr, nm in ((A.F32, "fp32"), (A.F64, "fp64")):
            xx = xf.to(torch.complex64) if pr == A.F32 else xf
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
        traffic = {k: (11 * cb[k] + cb[k] // 2) * nf * nf for k in cb}
        hbm = {k: traffic[k] / (h_ms[k] * 1e-3) / 1e9 for k in cb}
        flat = {"n": nf, "pixels": nf * nf, "solve_s": t_f, "inner_iters": inf_f["iters"],
                "outer": inf_f["outer"], "h_applies_f64": inf_f["h_applies_f64"], "relres": inf_f["relres"],
                "h_apply_ms": h_ms, "h_traffic_bytes": traffic, "h_achieved_gbs": hbm,
                "h_frac_of_hbm": {k: hbm[k] / HBM_GBS for k in hbm}}
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
               "h_apply_s_extrapolated": t_H}
    last = infos[-1]
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
        "cg": {"solve_s": ms_per_step / 1e3, "inner_iters": last["iters"], "outer": last["outer"],
               "h_applies_f32": last["h_applies_f32"], "h_applies_f64": last["h_applies_f64"],
               "relres": last["relres"], "per_inner_iter_ms": st32["total"]},
        "fp64": fp64,
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk.summary(),
    }
    if fields is not None:
        line["fields"] = fields
    if noise is not None:
        line["noise_realisations"] = noise
    if per_l is not None:
        line["per_l_preconditioner"] = per_l
    if flat is not None:
        line["flat_sky"] = flat
    if batch is not None:
        line["batch_uneven"] = batch
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
