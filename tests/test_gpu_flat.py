"""Flat-sky variant (Sec. II B: each SHT replaced by a 2D FFT): the CUDA operators and solves on
an n x n grid against the oracle's numpy-FFT forms.

Tolerances: FP64 at rel. L2 1e-10; FP32 operators at 2e-6 log2(n) (rounding of the radix-4
passes grows with their number); mixed solves at 1e-6 against the oracle solved to 1e-12."""
import math

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


def tolf(n):
    return 2e-6 * math.log2(n)


@pytest.mark.parametrize("n", [16, 64, 256, 2048])
@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_flat_operators_match_oracle(n, prec):
    rng = np.random.default_rng(n)
    p = A.akra_flat_plan_create(n)
    sv = S.flat_survey(n, seed=77 + n)
    A.akra_plan_set_weights(p, torch.from_numpy(sv["ninv"]).to(DEV), 1e-3)
    w = O.FlatWeights(sv["ninv"].reshape(n, n), 1e-3)
    R = 2
    xs = [rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)) for _ in range(R)]
    us = [rng.normal(size=(2, n * n)) for _ in range(R)]
    cdt = torch.complex128 if prec == A.F64 else torch.complex64
    rdt = torch.float64 if prec == A.F64 else torch.float32
    xd = torch.from_numpy(np.stack(xs)).to(DEV, cdt)
    ud = torch.from_numpy(np.stack(us)).to(DEV, rdt)
    tol = 1e-10 if prec == A.F64 else tolf(n)
    g = A.akra_apply_A(p, prec, xd).double().cpu().numpy()
    gw = A.akra_apply_A(p, prec, xd, weighted=True).double().cpu().numpy()
    a = A.akra_apply_At(p, prec, ud).to(torch.complex128).cpu().numpy()
    h = A.akra_apply_H(p, prec, xd).to(torch.complex128).cpu().numpy()
    for r in range(R):
        g1, g2 = O.flat_forward_A(n, xs[r])
        ref = np.stack([g1.ravel(), g2.ravel()])
        assert rel(g[r], ref) < tol, ("A", r)
        assert rel(gw[r], ref * w.W.ravel()) < tol, ("WA", r)
        refa = O.flat_adjoint_A(n, us[r][0].reshape(n, n), us[r][1].reshape(n, n))
        assert rel(a[r], refa) < tol, ("At", r)
        assert rel(h[r], O.flat_apply_H(n, w, xs[r])) < tol, ("H", r)


@pytest.fixture(scope="module")
def flat256():
    n = 256
    sv = S.flat_survey(n, seed=5)
    y = np.stack(O.flat_forward_A(n, sv["x_true"]))
    y = np.stack([y[0].ravel(), y[1].ravel()]) + sv["noise"]
    y = np.where(sv["mask"], y, 0.0)
    w = O.FlatWeights(sv["ninv"].reshape(n, n), 1e-3)
    xref, it, rr = O.flat_cg_solve(n, w, y[0].reshape(n, n), y[1].reshape(n, n), tol=1e-12, maxiter=5000)
    p = A.akra_flat_plan_create(n)
    A.akra_plan_set_weights(p, torch.from_numpy(sv["ninv"]).to(DEV), 1e-3)
    return n, p, y, xref, it


def test_flat_cg_fp64_matches_oracle(flat256):
    n, p, y, xref, it = flat256
    x, info = A.akra_cg_solve(p, A.F64, torch.from_numpy(y[None]).to(DEV), tol=1e-12, maxiter=5000)
    assert info["status"] == 0 and info["relres"] < 1e-11
    assert rel(x[0].cpu().numpy(), xref) < 1e-10
    assert abs(info["iters"] - it) <= 2


def test_flat_cg_mixed_and_fp32(flat256):
    n, p, y, xref, it = flat256
    x, info = A.akra_cg_solve(p, A.MIXED, torch.from_numpy(y[None]).to(DEV), tol=1e-9, maxiter=5000)
    assert info["status"] == 0 and info["relres"] < 1e-9 and info["outer"] >= 1
    assert rel(x[0].cpu().numpy(), xref) < 1e-6
    x32, i32 = A.akra_cg_solve(p, A.F32, torch.from_numpy(y[None]).to(DEV, torch.float32), tol=1e-5,
                               maxiter=5000)
    assert i32["status"] == 0
    assert rel(x32[0].to(torch.complex128).cpu().numpy(), xref) < 1e-3


def test_flat_multi_rhs_and_describe(flat256):
    n, p, y, xref, it = flat256
    ys = torch.from_numpy(np.stack([y, -2.0 * y])).to(DEV)
    x, info = A.akra_cg_solve(p, A.F64, ys, tol=1e-12, maxiter=5000)
    assert rel(x[0].cpu().numpy(), xref) < 1e-10 and rel(x[1].cpu().numpy(), -2.0 * xref) < 1e-10
    d = A.akra_plan_describe(p)
    assert d["npix"] == n * n and d["has_weights"] == 1 and d["nring"] == 0


def test_flat_rejects_sphere_only_calls(flat256):
    n, p, y, xref, it = flat256
    x = torch.zeros(p.alm_shape(1), dtype=torch.complex128, device=DEV)
    with pytest.raises(A.AkraError):
        A.akra_synth_spin2(p, A.F64, x)
    with pytest.raises(A.AkraError):
        A.akra_autotune(p, A.MIXED, 1)
    with pytest.raises(A.AkraError):
        A.akra_cg_solve_fields(p, A.F64, A.SOLVE_E, torch.from_numpy(y[None]).to(DEV), tol=1e-6)
    with pytest.raises(A.AkraError):
        A.akra_cg_solve_adjoint(p, A.F64, x, tol=1e-6)
    with pytest.raises(A.AkraError):
        A.akra_flat_plan_create(100)
