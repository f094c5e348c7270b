"""Profiling driver: build a DES-like problem at (nside, lmax) and run `reps` H applications
(or one mixed solve) -- a small, self-contained command for Nsight Compute captures.

    python -m paper_2606_06175_gb300.profile_step --nside 1024 --lmax 2048 --prec f32 --reps 2
"""
import argparse
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

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
    args = ap.parse_args()
    N, L = args.nside, args.lmax
    dev = torch.device("cuda", 0)
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
    plan = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(plan, torch.from_numpy(sv["ninv"]).to(dev), 1e-3)
    prec = A.F32 if args.prec == "f32" else A.F64
    if args.shape:
        A.akra_plan_set_shape(plan, prec, 1, *args.shape)
    kE = S.grf_alm(L, S.cl_kappa(L), sv["rng_alm"])
    x64 = torch.from_numpy(np.stack([kE, np.zeros_like(kE)])[None]).to(dev)
    if args.solve:
        y = A.akra_apply_A(plan, A.F64, x64)
        _, info = A.akra_cg_solve(plan, A.MIXED, y, tol=1e-6, maxiter=2000)
        print(info)
    else:
        x = x64 if prec == A.F64 else x64.to(torch.complex64)
        for _ in range(args.reps):
            A.akra_apply_H(plan, prec, x)
    torch.cuda.synchronize()
    print("ok", A.akra_plan_describe(plan)["kernel_launches"])


if __name__ == "__main__":
    main()
