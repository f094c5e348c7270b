"""Field-restricted solves (App. A): the E-mode normal equations H_EE κ_E = b_E and the
conditional B-mode solve H_BB κ_B = b_B - H_BE κ̂_E (Eq. A8), through akra_cg_solve_fields,
against the oracle's E-only and conditional solves (both to 1e-12 for FP64)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def cap32():
    wl = S.workload("cap32")
    N, L = wl["nside"], wl["lmax"]
    y = np.stack(O.forward_A(N, L, *wl["x_true"])) + wl["noise"]
    y = np.where(wl["ninv"] > 0, y, 0.0)
    w = O.Weights(N, wl["ninv"], 1e-3)
    (eE, eB), _, _, _ = O.cg_solve_E(N, L, w, y[0], y[1], tol=1e-12, maxiter=3000)
    (_, cB), _, _, _ = O.cg_solve_B_given_E(N, L, w, y[0], y[1], eE, tol=1e-12, maxiter=3000)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    return p, N, L, y, eE, cB


@pytest.mark.parametrize("prec,tol,bound", [(A.F64, 1e-12, 1e-10), (A.MIXED, 1e-9, 1e-6)])
def test_e_only_and_conditional_b_match_oracle(cap32, prec, tol, bound):
    p, N, L, y, eE, cB = cap32
    yd = torch.from_numpy(y[None]).to(DEV)
    x, info = A.akra_cg_solve_fields(p, prec, A.SOLVE_E, yd, tol=tol, maxiter=3000)
    assert info["status"] == 0 and info["relres"] < tol, info
    xn = x[0].cpu().numpy()
    assert rel(xn[0], eE) < bound
    assert not np.any(xn[1])                      # κ_B held at zero
    e_in = x[0, 0].clone()
    x2, info2 = A.akra_cg_solve_fields(p, prec, A.SOLVE_B_GIVEN_E, yd, out=x, tol=tol, maxiter=3000)
    assert info2["status"] == 0 and info2["relres"] < tol, info2
    assert torch.equal(x2[0, 0], e_in)            # the E field is kept as given
    assert rel(x2[0, 1].cpu().numpy(), cB) < bound


def test_f32_e_only_close_to_oracle(cap32):
    p, N, L, y, eE, cB = cap32
    x, info = A.akra_cg_solve_fields(p, A.F32, A.SOLVE_E, torch.from_numpy(y[None]).to(DEV, torch.float32),
                                     tol=1e-5, maxiter=3000)
    assert info["status"] == 0
    assert rel(x[0, 0].to(torch.complex128).cpu().numpy(), eE) < 1e-3


def test_conditional_b_given_joint_e_equals_joint_b(cap32):
    """Eq. A7 is the lower block row of the joint system: with the joint κ̂_E the reduced
    B solve returns the joint κ̂_B (a property of the GPU path alone)."""
    p, N, L, y, eE, cB = cap32
    yd = torch.from_numpy(y[None]).to(DEV)
    xj, _ = A.akra_cg_solve(p, A.F64, yd, tol=1e-12, maxiter=3000)
    x = xj.clone()
    x[:, 1] = 0
    xb, info = A.akra_cg_solve_fields(p, A.F64, A.SOLVE_B_GIVEN_E, yd, out=x, tol=1e-12, maxiter=3000)
    assert rel(xb[0, 1].cpu().numpy(), xj[0, 1].cpu().numpy()) < 1e-9


def test_multi_rhs_fields_match_single(cap32):
    p, N, L, y, eE, cB = cap32
    rng = np.random.default_rng(5)
    y2 = np.where(y != 0, y + 0.01 * rng.normal(size=y.shape), 0.0)
    ys = torch.from_numpy(np.stack([y, y2])).to(DEV)
    x, info = A.akra_cg_solve_fields(p, A.F64, A.SOLVE_E, ys, tol=1e-12, maxiter=3000)
    x1, _ = A.akra_cg_solve_fields(p, A.F64, A.SOLVE_E, ys[1:].contiguous(), tol=1e-12, maxiter=3000)
    assert rel(x[0, 0].cpu().numpy(), eE) < 1e-10
    assert rel(x[1].cpu().numpy(), x1[0].cpu().numpy()) < 1e-10
    # the joint solver's graphs are unaffected by the field-restricted ones
    xj, _ = A.akra_cg_solve(p, A.F64, ys[:1].contiguous(), tol=1e-12, maxiter=3000)
    (jE, jB), _, _, _ = O.cg_solve(N, L, O.Weights(N, S.workload("cap32")["ninv"], 1e-3), y[0], y[1],
                                   tol=1e-12, maxiter=3000)
    assert rel(xj[0].cpu().numpy(), np.stack([jE, jB])) < 1e-10


def test_fields_errors(cap32):
    p, N, L, y, eE, cB = cap32
    yd = torch.from_numpy(y[None]).to(DEV)
    with pytest.raises(A.AkraError):
        A.akra_cg_solve_fields(p, A.F64, 3, yd, tol=1e-6)
    with pytest.raises(ValueError):
        A.akra_cg_solve_fields(p, A.F64, A.SOLVE_B_GIVEN_E, yd, tol=1e-6)
