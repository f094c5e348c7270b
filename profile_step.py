"""Profiling driver: build a DES-like problem at (nside, lmax) and run `reps` H applications
(or one mixed solve) -- a small, self-contained command for Nsight Compute captures.

    python profile_step.py --nside 1024 --lmax 2048 --prec f32 --reps 2

`--cufft` instead times the library's FP32 ring-FFT stage (fold, backward DFT, ×W, forward
DFT, unfold on every ring that holds a weighted pixel) next to cuFFT (through torch.fft) doing
only the two DFTs and the ×W on the same rings, grouped by ring length; a timed comparison,
cuFFT is not used by the library.
"""
import json
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import synthetic as S  # noqa: E402
from paper_2606_06175_gb300 import akra as A  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nside", type=int, default=1024)
    ap.add_argument("--lmax", type=int, default=2048)
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--solve", action="store_true", help="one mixed-precision solve instead")
    ap.add_argument("--flat", type=int, default=0, metavar="N",
                    help="H applications of the flat-sky variant on an N x N grid instead")
    ap.add_argument("--shape", type=int, nargs=3, metavar=("P", "PA", "RG"),
                    help="force the Legendre tile shape of --prec (R = 1)")
    ap.add_argument("--cufft", action="store_true",
                    help="time the FP32 ring-FFT stage against cuFFT on the same rings")
    ap.add_argument("--autotune", action="store_true", help="autotune the tile shapes of --prec first")
    ap.add_argument("--tc", type=int, default=0, metavar="G",
                    help="FP32 synthesis on the tensor core with RHS groups of G (with --rhs)")
    ap.add_argument("--rhs", type=int, default=1, help="right-hand sides of the H applications")
    ap.add_argument("--south-only", action="store_true",
                    help="drop the footprint's pixels at dec >= 0 (every active ring pair then needs its south ring alone)")
    ap.add_argument("--stages", action="store_true",
                    help="print the CUDA-event stage times of one H (akra_time_H_stages, 5 runs) as JSON")
    ap.add_argument("--batch", action="store_true",
                    help="one batched FP32 H over two instances (Nside and Nside/2, --rhs RHS each) instead")
    args = ap.parse_args()
    N, L = args.nside, args.lmax
    dev = torch.device("cuda", 0)
    if args.batch:
        plans, xs = [], []
        for k, (nb, lb) in enumerate(((N, L), (N // 2, L // 2))):
            svb = S.survey(nb, "des", S.SEEDS["batch"] + k)
            pb = A.akra_plan_create(nb, lb)
            A.akra_plan_set_weights(pb, torch.from_numpy(svb["ninv"]).to(dev), 1e-3)
            plans.append(pb)
            xs.append(torch.zeros((args.rhs, 2, pb.ntri), dtype=torch.complex64, device=dev))
        bt = A.akra_batch_create(plans, [args.rhs, args.rhs])
        if args.autotune:
            A.akra_batch_autotune(bt)
        if args.tc:
            A.akra_batch_set_tc_synthesis(bt, args.tc)
        for _ in range(args.reps):
            A.akra_batch_apply_H(bt, xs)
        torch.cuda.synchronize()
        print("ok batch", A.akra_batch_describe(bt), "tc", A.akra_batch_get_tc_synthesis(bt))
        return
    if args.flat:
        sv = S.flat_survey(args.flat)
        fp = A.akra_flat_plan_create(args.flat)
        A.akra_plan_set_weights(fp, torch.from_numpy(sv["ninv"]).to(dev), 1e-3)
        pr = A.F32 if args.prec == "f32" else A.F64
        x = torch.from_numpy(sv["x_true"][None]).to(dev, torch.complex64 if pr == A.F32 else torch.complex128)
        for _ in range(args.reps):
            A.akra_apply_H(fp, pr, x)
        torch.cuda.synchronize()
        print("ok", A.akra_plan_describe(fp)["kernel_launches"])
        return
    sv = S.survey(N, "des", S.SEEDS["des2048"])
    ninv = sv["ninv"]
    if args.south_only:
        z = S.pixel_positions(N)[0]
        ninv = np.where(z < 0, ninv, 0.0)
    plan = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(plan, torch.from_numpy(ninv).to(dev), 1e-3)
    prec = A.F32 if args.prec == "f32" else A.F64
    R = args.rhs
    if args.shape:
        A.akra_plan_set_shape(plan, prec, R, *args.shape)
    if args.autotune:
        A.akra_autotune(plan, prec, R)
    if args.tc:
        A.akra_plan_set_tc_synthesis(plan, R, args.tc)
    kE = S.grf_alm(L, S.cl_kappa(L), sv["rng_alm"])
    x64 = torch.from_numpy(np.stack([kE, np.zeros_like(kE)])[None]).to(dev)
    if args.cufft:
        print(json.dumps(cufft_comparison(plan, sv["ninv"], N, dev)))
        return
    if args.stages:
        st = A.akra_time_H_stages(plan, prec, R, 5)
        print(json.dumps({"nside": N, "lmax": L, "prec": args.prec, "rhs": R, "tc_group": args.tc,
                          "shape": A.akra_plan_get_shape(plan, prec, R), "stage_ms": st,
                          "per_rhs_ms": {k: v / R for k, v in st.items()}}))
        return
    if args.solve:
        y = A.akra_apply_A(plan, A.F64, x64)
        _, info = A.akra_cg_solve(plan, A.MIXED, y, tol=1e-6, maxiter=2000)
        print(info)
    else:
        x = x64 if prec == A.F64 else x64.to(torch.complex64)
        x = x.repeat(R, 1, 1).contiguous()
        for _ in range(args.reps):
            A.akra_apply_H(plan, prec, x)
    torch.cuda.synchronize()
    sh = A.akra_plan_get_shape(plan, prec, R)
    print("shape", sh["P"], sh["PA"], sh["RG"], "tc", A.akra_plan_get_tc_synthesis(plan, R) if prec == A.F32 else 0)
    print("ok", A.akra_plan_describe(plan)["kernel_launches"])


def ring_table(N):
    """HEALPix RING rings (i = 1 .. 4N-1): (first pixel, number of pixels)."""
    npix = 12 * N * N
    out = []
    for i in range(1, 4 * N):
        if i < N:
            out.append((2 * i * (i - 1), 4 * i))
        elif i <= 3 * N:
            out.append((2 * N * (N - 1) + 4 * N * (i - N), 4 * N))
        else:
            k = 4 * N - i
            out.append((npix - 2 * k * (k + 1), 4 * k))
    return out


def cufft_comparison(plan, ninv, N, dev, reps=5):
    ours = A.akra_time_H_stages(plan, A.F32, 1, reps)["ring_fft"]
    groups = {}
    for first, n in ring_table(N):
        if np.any(ninv[first:first + n] > 0):
            groups.setdefault(n, []).append(first)
    w = torch.from_numpy((4 * np.pi / ninv.size) * ninv).to(dev, torch.float32)
    g = torch.Generator(device="cpu").manual_seed(7)
    data = []
    for n, firsts in sorted(groups.items()):
        idx = (torch.tensor(firsts)[:, None] + torch.arange(n)[None, :]).to(dev)
        x = torch.randn(len(firsts), n, generator=g, dtype=torch.complex64).to(dev)
        data.append((n, x, w[idx]))

    def run(sel):
        for n, x, wg in sel:
            y = torch.fft.ifft(x, norm="forward") * wg   # backward DFT (no 1/n), then ×W
            torch.fft.fft(y)                            # forward DFT
    belt = [d for d in data if d[0] == 4 * N]
    out = {"nside": N, "active_rings": sum(d[1].shape[0] for d in data), "ring_lengths": len(data),
           "belt_rings": sum(d[1].shape[0] for d in belt), "ring_fft_stage_ms": ours}
    for key, sel in (("cufft_all_rings_ms", data), ("cufft_belt_rings_ms", belt)):
        for _ in range(3):
            run(sel)   # plans are created and cached here
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            run(sel)
        e1.record()
        torch.cuda.synchronize()
        out[key] = e0.elapsed_time(e1) / reps
    return out


if __name__ == "__main__":
    main()
