"""The Nside 512 / lmax 1024 workload (DES-like footprint, seed 1002): FP64 and mixed GPU solves.

The oracle cannot run a whole CG at this size on the host, but it can evaluate its own
operator once: the GPU's FP64 solution must satisfy the ORACLE's normal equations
(||b_o - H_o x|| / ||b_o|| at the solve tolerance), with b_o and H_o the FP64 oracle's
right-hand side (Eq. 8) and operator (Eq. 14), and the GPU's full-size forward operator and
right-hand side must equal the oracle's.  The mixed solve is then checked against the FP64
GPU solve: at the same stopping residual it is as accurate as plain FP64, and run to 1e-8 its
solution is within 1e-6 of the FP64 solution at 1e-10 (solution error <= κ x residual, with a
measured ratio of ~20-60 here, so a 1e-6 solution error needs a residual below ~1e-7).
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N, L = 512, 1024


def _rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def case():
    wl = S.workload("des512")
    w = O.Weights(N, wl["ninv"], 1e-3)
    kE, kB = wl["x_true"]
    g1, g2 = O.forward_A(N, L, kE, kB)
    m = wl["mask"]
    y = np.stack([np.where(m, g1 + wl["noise"][0], 0.0), np.where(m, g2 + wl["noise"][1], 0.0)])
    bE, bB = O.rhs_b(N, L, w, y[0], y[1])
    plan = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(plan, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    yd = torch.from_numpy(y[None]).to(DEV)
    return dict(w=w, y=y, b=np.stack([bE, bB]), plan=plan, yd=yd)


def test_fp64_solve_satisfies_the_oracle_normal_equations(case):
    plan, w = case["plan"], case["w"]
    b_gpu = A.akra_apply_At(plan, A.F64, case["yd"], weighted=True)
    assert _rel(b_gpu[0].cpu().numpy(), case["b"]) < 1e-10
    x, info = A.akra_cg_solve(plan, A.F64, case["yd"], tol=1e-10, maxiter=3000)
    assert info["status"] == 0 and info["relres"] < 1e-10
    x = x[0].cpu().numpy()
    # forward operator at full size against the oracle's
    gx = A.akra_apply_A(plan, A.F64, torch.from_numpy(x[None]).to(DEV))[0].cpu().numpy()
    f1, f2 = O.forward_A(N, L, x[0], x[1])
    assert _rel(gx, np.stack([f1, f2])) < 1e-10
    # the oracle's residual of the GPU solution
    hE, hB = O.adjoint_A(N, L, w.W * f1, w.W * f2)
    hE, hB = hE + w.lam_eff * x[0], hB + w.lam_eff * x[1]
    r = case["b"] - np.stack([hE, hB])
    num = O.pair_dot(L, r, r) ** 0.5
    den = O.pair_dot(L, case["b"], case["b"]) ** 0.5
    assert num / den < 1e-9, num / den
    case["x64"] = torch.from_numpy(x[None]).to(DEV)


def test_mixed_solve_against_fp64_solve(case):
    plan, yd = case["plan"], case["yd"]
    x64 = case.get("x64")
    if x64 is None:
        x64, _ = A.akra_cg_solve(plan, A.F64, yd, tol=1e-10, maxiter=3000)
    xf6, i6 = A.akra_cg_solve(plan, A.F64, yd, tol=1e-6, maxiter=3000)
    xm6, im6 = A.akra_cg_solve(plan, A.MIXED, yd, tol=1e-6, maxiter=3000)
    xm8, im8 = A.akra_cg_solve(plan, A.MIXED, yd, tol=1e-8, maxiter=3000)
    assert i6["status"] == 0 and im6["status"] == 0 and im8["status"] == 0
    assert im6["relres"] < 1e-6 and im8["relres"] < 1e-8
    rel = lambda a: float(torch.linalg.vector_norm(a - x64) / torch.linalg.vector_norm(x64))
    e_f6, e_m6, e_m8 = rel(xf6), rel(xm6), rel(xm8)
    # same stopping residual: the mixed solution is as accurate as the plain FP64 one
    assert e_m6 <= 2 * e_f6 + 1e-7, (e_m6, e_f6)
    # run below the κ-scaled bound, the mixed solution is within 1e-6 of the FP64 one
    assert e_m8 < 1e-6, e_m8
