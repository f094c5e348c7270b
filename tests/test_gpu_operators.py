"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances: FP64 operators and FP64 solves at rel. L2 1e-10; FP32 operators at
tol32(L) = 4 ε32 L (FP32 rounding of the l-recurrence grows linearly in the number of steps);
mixed-precision solves at 1e-6 on the solved alm against the oracle solved to 1e-12.
"""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
import synthetic as S
from paper_2606_06175_gb300 import akra as A

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL64 = 1e-10


def tol32(lmax):
    # the three-term recurrence is neutrally stable on the oscillatory side, so FP32 rounding
    # grows linearly with the number of l-steps: rel. error ~ ε32 L / 2 (measured); bound 4 ε32 L
    return 4 * 2.0 ** -24 * max(lmax, 16)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def alm_dev(pairs, prec=A.F64):
    arr = np.stack([np.stack(p) for p in pairs])
    return torch.from_numpy(arr).to(DEV, torch.complex128 if prec == A.F64 else torch.complex64)


def map_dev(maps, prec=A.F64):
    arr = np.stack([np.stack(m) for m in maps])
    return torch.from_numpy(arr).to(DEV, torch.float64 if prec == A.F64 else torch.float32)


_plans = {}


def plan(N, L):
    if (N, L) not in _plans:
        _plans[(N, L)] = A.akra_plan_create(N, L)
    return _plans[(N, L)]


SIZES = [(1, 2), (2, 5), (4, 8), (8, 31), (16, 40), (32, 64), (64, 150), (256, 300)]


@pytest.mark.parametrize("N,L", SIZES)
@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_synthesis_matches_oracle(N, L, prec):
    rng = np.random.default_rng(N * 1000 + L)
    aE, aB = S.random_alm(L, rng), S.random_alm(L, rng)
    g = A.akra_synth_spin2(plan(N, L), prec, alm_dev([(aE, aB)], prec))[0].cpu().numpy()
    ref = np.stack(O.synth_spin2(N, L, aE, aB))
    err = rel(g, ref)
    assert err < (TOL64 if prec == A.F64 else tol32(L)), err


@pytest.mark.parametrize("N,L", SIZES)
@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_adjoint_matches_oracle(N, L, prec):
    rng = np.random.default_rng(N * 1000 + L + 1)
    u = rng.normal(size=(2, 12 * N * N))
    a = A.akra_adjoint_synth_spin2(plan(N, L), prec, map_dev([u], prec))[0].cpu().numpy()
    ref = np.stack(O.adjoint_synth_spin2(N, L, u[0], u[1]))
    err = rel(a, ref)
    assert err < (TOL64 if prec == A.F64 else tol32(L)), err
    ls, ms = O.lm_arrays(L)
    assert np.all(a[:, ms == 0].imag == 0)


def _mask_weights(N, seed, cap=1.0):
    rng = np.random.default_rng(seed)
    th, ph = O.pixel_angles(N)
    ninv = np.where((th > cap) & (np.sin(3 * ph) > -0.7), rng.poisson(20, 12 * N * N) / 0.26 ** 2, 0.0)
    return ninv


@pytest.mark.parametrize("N,L", [(4, 8), (8, 31), (16, 40), (32, 64), (256, 300)])
@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_H_matches_oracle(N, L, prec):
    ninv = _mask_weights(N, N + L)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    w = O.Weights(N, ninv, 1e-3)
    d = A.akra_plan_describe(p)
    assert abs(d["lambda_eff"] - w.lam_eff) <= 1e-12 * w.lam_eff
    assert abs(d["precond"] - w.precond) <= 1e-12 * w.precond
    rng = np.random.default_rng(L)
    xE, xB = S.random_alm(L, rng), S.random_alm(L, rng)
    h = A.akra_apply_H(p, prec, alm_dev([(xE, xB)], prec))[0].cpu().numpy()
    ref = np.stack(O.apply_H(N, L, w, xE, xB))
    err = rel(h, ref)
    assert err < (TOL64 if prec == A.F64 else tol32(L)), err


SHAPES = [(1, 1), (2, 1), (3, 1), (4, 1), (5, 1), (6, 1), (8, 1), (1, 2), (2, 2), (1, 4)]


@pytest.mark.parametrize("P,RG", SHAPES)
@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_every_tile_shape_matches_oracle(P, RG, prec):
    """Each compiled Legendre shape (synthesis and adjoint) on H, with R = RG + 1 RHS so that
    the last RHS group is ragged; the adjoint uses a different P where one is compiled."""
    if P in (3, 5, 6, 8) and prec == A.F64:
        pytest.skip("P = 3, 5, 6, 8 are compiled for FP32 only")
    N, L, R = 16, 40, RG + 1
    if RG == 1:
        pa = {1: 2, 2: 1, 3: 5, 4: 8 if prec == A.F32 else 1, 5: 6, 6: 3, 8: 4}[P]
    else:
        pa = 2 if (RG, P) == (2, 1) else 1 if RG == 2 else 1
    p = A.akra_plan_create(N, L)
    rng = np.random.default_rng(97 + P + 10 * RG)
    th, ph = O.pixel_angles(N)
    ninv = np.where(np.cos(th) < 0.4, 1.0 + rng.random(12 * N * N), 0.0)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    A.akra_plan_set_shape(p, prec, R, P, pa, RG)
    assert A.akra_plan_get_shape(p, prec, R) == {"P": P, "PA": pa, "RG": RG}
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    y = A.akra_apply_H(p, prec, alm_dev(pairs, prec)).to(torch.complex128).cpu().numpy()
    w = O.Weights(N, ninv, 1e-3)
    for r in range(R):
        ref = np.stack(O.apply_H(N, L, w, *pairs[r]))
        assert rel(y[r], ref) < (TOL64 if prec == A.F64 else tol32(L)), (P, RG, r)
    # the adjoint alone on every ring (unweighted) with the forced shape
    maps = [tuple(rng.normal(size=(2, 12 * N * N))) for _ in range(R)]
    a = A.akra_adjoint_synth_spin2(p, prec, map_dev(maps, prec)).to(torch.complex128).cpu().numpy()
    for r in range(R):
        ref = np.stack(O.adjoint_synth_spin2(N, L, *maps[r]))
        assert rel(a[r], ref) < (TOL64 if prec == A.F64 else tol32(L)), (P, RG, r)


def test_start_table_step_counts():
    """The per-pair start points only drop steps: FP32 (threshold 2^-40) takes no more steps
    than FP64 (2^-90), and neither more than the full triangle."""
    N, L = 64, 150
    p = A.akra_plan_create(N, L)
    d = A.akra_plan_describe(p)
    full = d["nunit"] * (d["ntri"] - 3)
    assert 0 < d["legendre_steps_f32"] <= d["legendre_steps_f64"] <= full
    th, _ = O.pixel_angles(N)
    A.akra_plan_set_weights(p, torch.from_numpy(np.where(np.cos(th) > 0.5, 1.0, 0.0)).to(DEV), 1e-3)
    d2 = A.akra_plan_describe(p)
    assert 0 < d2["legendre_steps_f32"] <= d2["legendre_steps_f64"] <= d2["n_active_units"] * (d["ntri"] - 3)
    assert d2["legendre_steps_f32"] < d["legendre_steps_f32"]


def test_shape_errors():
    p = A.akra_plan_create(8, 12)
    for bad in [(3, 3, 1), (4, 4, 2), (2, 2, 4), (8, 8, 1)]:
        with pytest.raises(A.AkraError):
            A.akra_plan_set_shape(p, A.F64, 1, *bad)
    with pytest.raises(A.AkraError):
        A.akra_plan_set_shape(p, A.MIXED, 1, 1, 1, 1)


@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_apply_A_and_At_match_oracle(prec):
    N, L = 16, 40
    ninv = _mask_weights(N, 3)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    w = O.Weights(N, ninv, 1e-3)
    rng = np.random.default_rng(11)
    xE, xB = S.random_alm(L, rng), S.random_alm(L, rng)
    tol = TOL64 if prec == A.F64 else tol32(L)
    y = A.akra_apply_A(p, prec, alm_dev([(xE, xB)], prec))[0].cpu().numpy()
    assert rel(y, np.stack(O.forward_A(N, L, xE, xB))) < tol
    yw = A.akra_apply_A(p, prec, alm_dev([(xE, xB)], prec), weighted=True)[0].cpu().numpy()
    assert rel(yw, w.W * np.stack(O.forward_A(N, L, xE, xB))) < tol
    u = rng.normal(size=(2, 12 * N * N))
    b = A.akra_apply_At(p, prec, map_dev([u], prec), weighted=True)[0].cpu().numpy()
    assert rel(b, np.stack(O.rhs_b(N, L, w, u[0], u[1]))) < tol


@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_batched_rhs_match_oracle(prec):
    """R = 3 right-hand sides in one launch (a ragged RHS group for the 2- and 4-wide tiles)."""
    N, L = 16, 40
    R = 3
    rng = np.random.default_rng(5)
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    p = plan(N, L)
    g = A.akra_synth_spin2(p, prec, alm_dev(pairs, prec)).cpu().numpy()
    tol = TOL64 if prec == A.F64 else tol32(L)
    for r in range(R):
        assert rel(g[r], np.stack(O.synth_spin2(N, L, *pairs[r]))) < tol
    us = [rng.normal(size=(2, 12 * N * N)) for _ in range(R)]
    a = A.akra_adjoint_synth_spin2(p, prec, map_dev(us, prec)).cpu().numpy()
    for r in range(R):
        assert rel(a[r], np.stack(O.adjoint_synth_spin2(N, L, us[r][0], us[r][1]))) < tol


def test_adjoint_identity_gpu_512():
    """<A x, u> = <x, A^T u> to 1e-12 on the GPU at Nside 512, lmax 1024 (FP64)."""
    N, L = 512, 1024
    p = plan(N, L)
    rng = np.random.default_rng(9)
    x = alm_dev([(S.random_alm(L, rng), S.random_alm(L, rng))])
    u = torch.randn((1, 2, 12 * N * N), dtype=torch.float64, device=DEV)
    g = A.akra_synth_spin2(p, A.F64, x)
    a = A.akra_adjoint_synth_spin2(p, A.F64, u)
    lhs = float((g * u).sum())
    ls, ms = O.lm_arrays(L)
    w = torch.from_numpy(np.where(ms == 0, 1.0, 2.0)).to(DEV)
    xr, ar = x[0].real, a[0].real
    xi = torch.where(torch.from_numpy(ms == 0).to(DEV), 0.0, x[0].imag)
    rhs = float((w * (xr * ar + xi * a[0].imag)).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# ---------------------------------------------------------------------------
# CG
# ---------------------------------------------------------------------------
def _cap32():
    wl = S.workload("cap32")
    N, L = wl["nside"], wl["lmax"]
    y = np.stack(O.forward_A(N, L, *wl["x_true"])) + wl["noise"]
    y = np.where(wl["ninv"] > 0, y, 0.0)
    return wl, N, L, y


@pytest.fixture(scope="module")
def cap32_ref():
    wl, N, L, y = _cap32()
    w = O.Weights(N, wl["ninv"], 1e-3)
    (xE, xB), it, rr, hist = O.cg_solve(N, L, w, y[0], y[1], tol=1e-12, maxiter=3000)
    return wl, N, L, y, np.stack([xE, xB]), it, hist


def test_cg_fp64_cap32_matches_oracle(cap32_ref):
    wl, N, L, y, xref, it_ref, _ = cap32_ref
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    x, info = A.akra_cg_solve(p, A.F64, torch.from_numpy(y[None]).to(DEV), tol=1e-12, maxiter=3000)
    assert info["status"] == 0 and info["relres"] < 1e-11
    assert rel(x[0].cpu().numpy(), xref) < TOL64
    # iteration count at the same tolerance equals the oracle's up to rounding
    assert abs(info["iters"] - it_ref) <= 2
    # the workload's own tolerance (1e-8): recursive and true FP64 residuals below it
    x8, info8 = A.akra_cg_solve(p, A.F64, torch.from_numpy(y[None]).to(DEV), tol=1e-8, maxiter=3000)
    assert info8["status"] == 0 and info8["relres"] < 1e-8


def test_cg_mixed_cap32_matches_oracle(cap32_ref):
    wl, N, L, y, xref, _, _ = cap32_ref
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    x, info = A.akra_cg_solve(p, A.MIXED, torch.from_numpy(y[None]).to(DEV), tol=1e-9, maxiter=3000)
    assert info["status"] == 0 and info["relres"] < 1e-9
    assert info["outer"] >= 1 and info["h_applies_f32"] > 0
    assert rel(x[0].cpu().numpy(), xref) < 1e-6


def test_cg_fp32_cap32_close_to_oracle(cap32_ref):
    wl, N, L, y, xref, _, _ = cap32_ref
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    x, info = A.akra_cg_solve(p, A.F32, torch.from_numpy(y[None]).to(DEV, torch.float32), tol=1e-5,
                              maxiter=3000)
    assert info["status"] == 0
    assert rel(x[0].cpu().numpy(), xref) < 1e-3


def test_cg_multi_rhs_matches_single(cap32_ref):
    wl, N, L, y, xref, _, _ = cap32_ref
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    ys = np.stack([y, 0.5 * y, -y])
    x, info = A.akra_cg_solve(p, A.F64, torch.from_numpy(ys).to(DEV), tol=1e-12, maxiter=3000)
    assert info["status"] == 0
    xs = x.cpu().numpy()
    assert rel(xs[0], xref) < TOL64
    assert rel(xs[1], 0.5 * xref) < TOL64
    assert rel(xs[2], -xref) < TOL64


def test_cg_solve_b_equals_cg_solve(cap32_ref):
    wl, N, L, y, xref, _, _ = cap32_ref
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    b = A.akra_apply_At(p, A.F64, torch.from_numpy(y[None]).to(DEV), weighted=True)
    x, info = A.akra_cg_solve_b(p, A.F64, b, tol=1e-12, maxiter=3000)
    assert rel(x[0].cpu().numpy(), xref) < TOL64


@pytest.mark.parametrize("prec,tol,bound", [(A.F64, 1e-12, TOL64), (A.MIXED, 1e-9, 1e-6)])
def test_per_l_preconditioner_matches_oracle(cap32_ref, prec, tol, bound):
    """The per-l diagonal preconditioner: same solution as the oracle's PCG with the same
    weights, FP64 iteration count equal up to rounding; switching back restores Eq. 15."""
    wl, N, L, y, xref, it_ref, _ = cap32_ref
    w = O.Weights(N, wl["ninv"], 1e-3)
    Pl = O.per_l_preconditioner(L, w)
    b = O.rhs_b(N, L, w, y[0], y[1])
    (oE, oB), it_o, _, _ = O.pcg(lambda e, bb: O.apply_H(N, L, w, e, bb), b, Pl, L, 1e-12, 3000)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    yd = torch.from_numpy(y[None]).to(DEV)
    A.akra_cg_solve(p, prec, yd, tol=tol, maxiter=3000)          # scalar form captured first
    A.akra_plan_set_preconditioner(p, A.PRECOND_PER_L)
    x, info = A.akra_cg_solve(p, prec, yd, tol=tol, maxiter=3000)
    assert info["status"] == 0 and info["relres"] < tol
    assert rel(x[0].cpu().numpy(), np.stack([oE, oB])) < bound
    if prec == A.F64:
        assert abs(info["iters"] - it_o) <= 2
    A.akra_plan_set_preconditioner(p, A.PRECOND_SCALAR)
    x2, info2 = A.akra_cg_solve(p, prec, yd, tol=tol, maxiter=3000)
    assert rel(x2[0].cpu().numpy(), xref) < bound
    if prec == A.F64:
        assert abs(info2["iters"] - it_ref) <= 2
    with pytest.raises(A.AkraError):
        A.akra_plan_set_preconditioner(p, 7)


def test_reweighting_after_a_solve(cap32_ref):
    """New weights (another footprint, so other active rings and λ_eff) after solves whose
    CG iterations were captured: the next solves use the new operator."""
    wl, N, L, y, xref, _, _ = cap32_ref
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(wl["ninv"]).to(DEV), 1e-3)
    yd = torch.from_numpy(y[None]).to(DEV)
    A.akra_cg_solve(p, A.F64, yd, tol=1e-12, maxiter=3000)
    A.akra_cg_solve(p, A.MIXED, yd, tol=1e-9, maxiter=3000)
    th, _ = O.pixel_angles(N)
    ninv2 = np.where(th > 2.38, 3.0 * wl["ninv"], 0.0)   # the southern half of the cap
    y2 = np.where(ninv2 > 0, y, 0.0)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv2).to(DEV), 1e-3)
    w2 = O.Weights(N, ninv2, 1e-3)
    x2ref = np.stack(O.cg_solve(N, L, w2, y2[0], y2[1], tol=1e-12, maxiter=3000)[0])
    y2d = torch.from_numpy(y2[None]).to(DEV)
    x, info = A.akra_cg_solve(p, A.F64, y2d, tol=1e-12, maxiter=3000)
    assert info["status"] == 0 and rel(x[0].cpu().numpy(), x2ref) < TOL64
    x, info = A.akra_cg_solve(p, A.MIXED, y2d, tol=1e-9, maxiter=3000)
    assert info["status"] == 0 and rel(x[0].cpu().numpy(), x2ref) < 1e-6


# ---------------------------------------------------------------------------
# error statuses (faults injected on the host; nothing faults the GPU)
# ---------------------------------------------------------------------------
def test_error_statuses():
    N, L = 8, 12
    p = A.akra_plan_create(N, L)
    x = torch.zeros((1, 2, p.ntri), dtype=torch.complex128, device=DEV)
    with pytest.raises(A.AkraError) as ei:
        A.akra_apply_H(p, A.F64, x)
    assert ei.value.status == 7   # ENOWEIGHTS
    bad = torch.full((p.npix,), -1.0, dtype=torch.float64, device=DEV)
    with pytest.raises(A.AkraError) as ei:
        A.akra_plan_set_weights(p, bad, 1e-3)
    assert ei.value.status == 1
    nan = torch.full((p.npix,), float("nan"), dtype=torch.float64, device=DEV)
    with pytest.raises(A.AkraError):
        A.akra_plan_set_weights(p, nan, 1e-3)
    A.akra_plan_set_weights(p, torch.full((p.npix,), 100.0, dtype=torch.float64, device=DEV), 1e-3)
    y = torch.randn((1, 2, p.npix), dtype=torch.float64, device=DEV)
    _, info = A.akra_cg_solve(p, A.F64, y, tol=1e-14, maxiter=1)
    assert info["status"] == 4 and info["iters"] == 1          # ENOCONV after maxiter
    A.akra_set_timeout(1e-9)
    try:
        with pytest.raises(A.AkraError) as ei:
            A.akra_cg_solve(p, A.F64, y, tol=1e-14, maxiter=100000)
        assert ei.value.status == 6                               # ETIMEOUT
    finally:
        A.akra_set_timeout(3600.0)
        torch.cuda.synchronize()
    # the plan and context are still usable after the timeout
    _, info = A.akra_cg_solve(p, A.F64, y, tol=1e-8, maxiter=500)
    assert info["status"] == 0
    yn = y.clone()
    yn[0, 0, 0] = float("nan")
    _, info = A.akra_cg_solve(p, A.F64, yn, tol=1e-8, maxiter=50)
    assert info["status"] == 5                                    # ENUMERIC


def test_timeout_leaves_the_callers_stream_ordered_after_queued_work():
    """After ETIMEOUT the solve's already launched iterations may still run; the caller's stream
    must wait for them, so buffers can be freed and reused in stream order with no device-wide
    synchronize.  Checked on a problem whose iterations take milliseconds: right after the
    ETIMEOUT return the caller's stream is still busy, and a fresh solve on reused memory
    gives the same solution as before."""
    N, L = 512, 1024
    p = A.akra_plan_create(N, L)
    sv = S.survey(N, "des", 1002)
    A.akra_plan_set_weights(p, torch.from_numpy(sv["ninv"]).to(DEV), 1e-3)
    g = torch.Generator(device=DEV).manual_seed(5)
    y = torch.randn((1, 2, p.npix), dtype=torch.float64, device=DEV, generator=g)
    y *= torch.from_numpy(sv["mask"]).to(DEV)
    xref, info = A.akra_cg_solve(p, A.F64, y, tol=1e-4, maxiter=500)   # also captures the graph
    assert info["status"] == 0
    torch.cuda.synchronize()
    x = torch.zeros_like(xref)
    A.akra_set_timeout(0.05)
    try:
        with pytest.raises(A.AkraError) as ei:
            A.akra_cg_solve(p, A.F64, y, x, tol=1e-14, maxiter=100000)
        assert ei.value.status == 6
        busy = not torch.cuda.current_stream().query()
    finally:
        A.akra_set_timeout(3600.0)
    assert busy, "the caller's stream is not ordered after the abandoned iterations"
    # free the solve's buffers and reuse the memory in stream order, without synchronising
    yc = y.clone()
    del x, y
    y2 = torch.empty_like(yc)
    y2.copy_(yc)
    x2 = torch.full_like(xref, float("nan"))
    x2, info = A.akra_cg_solve(p, A.F64, y2, x2, tol=1e-4, maxiter=500)
    torch.cuda.synchronize()
    assert info["status"] == 0
    assert float(torch.linalg.vector_norm(x2 - xref) / torch.linalg.vector_norm(xref)) < 1e-12


# ---------------------------------------------------------------------------
# degenerate input: an empty footprint (every N^-1 zero)
# ---------------------------------------------------------------------------
def test_empty_footprint_gives_zero_operator_and_zero_solution():
    N, L = 8, 12
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.zeros((p.npix,), dtype=torch.float64, device=DEV), 1e-3)
    d = A.akra_plan_describe(p)
    assert d["n_active_rings"] == 0 and d["n_active_units"] == 0 and d["lambda_eff"] == 0.0
    x = torch.randn((1, 2, p.ntri), dtype=torch.complex128, device=DEV)
    assert torch.count_nonzero(A.akra_apply_H(p, A.F64, x)) == 0
    shear = torch.randn((1, 2, p.npix), dtype=torch.float64, device=DEV)
    for prec in (A.F64, A.MIXED):
        xs, info = A.akra_cg_solve(p, prec, shear, tol=1e-6, maxiter=50)
        assert info["status"] == 0 and torch.count_nonzero(xs) == 0


def test_lane_steps_count_the_plans_steps():
    """The work accounting of a Legendre launch: its counted steps are the plan's start-table
    steps for every layout, and no layout executes fewer lane-steps than it counts."""
    N, L = 64, 128
    p = A.akra_plan_create(N, L)
    th, _ = O.pixel_angles(N)
    ninv = np.where(np.cos(th) < -0.2, 1.0, 0.0)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    d = A.akra_plan_describe(p)
    # a southern footprint: every active pair needs its south ring only
    assert d["legendre_steps_f32_one_ring"] == d["legendre_steps_f32"] > 0
    assert d["legendre_steps_f64_one_ring"] == d["legendre_steps_f64"] > 0
    for prec, key in ((A.F32, "legendre_steps_f32"), (A.F64, "legendre_steps_f64")):
        for adj in (False, True):
            for P in (1, 3, 4, 8):
                w = A.akra_legendre_lane_steps(p, prec, adj, P)
                assert w["steps"] == d[key], (prec, adj, P, w, d[key])
                assert w["lane_steps"] >= w["steps"]
                # a warp executes at most 32 P lanes over the whole triangle's l-range per m
                nw = -(-d["n_active_units"] // (128 * P)) * 4
                assert w["lane_steps"] <= nw * 32 * P * sum(L - max(m, 2) + 1 for m in range(L + 1))


@pytest.mark.parametrize("prec,RG,RGA", [(A.F32, 4, 1), (A.F32, 2, 1), (A.F64, 4, 2), (A.F64, 1, 2)])
def test_adjoint_rhs_group_differs_from_synthesis(prec, RG, RGA):
    """H with the synthesis taking RG right-hand sides per block and the adjoint RGA (R = 5: both
    groups partly filled), against the oracle; then the default shape and the autotuned one."""
    N, L, R = 16, 40, 5
    p = A.akra_plan_create(N, L)
    rng = np.random.default_rng(300 + RG * 10 + RGA)
    th, ph = O.pixel_angles(N)
    ninv = np.where(np.cos(th) < 0.4, 1.0 + rng.random(12 * N * N), 0.0)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    pa = 5 if prec == A.F32 and RGA == 1 else (2 if RGA == 2 else 1)
    A.akra_plan_set_shape(p, prec, R, 1, 1, RG)
    A.akra_plan_set_adjoint_shape(p, prec, R, pa, RGA)
    assert A.akra_plan_get_adjoint_shape(p, prec, R) == {"PA": pa, "RGA": RGA}
    assert A.akra_plan_get_shape(p, prec, R) == {"P": 1, "PA": pa, "RG": RG}
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    w = O.Weights(N, ninv, 1e-3)
    refs = [np.stack(O.apply_H(N, L, w, *q)) for q in pairs]
    tol = TOL64 if prec == A.F64 else tol32(L)
    y = A.akra_apply_H(p, prec, alm_dev(pairs, prec)).to(torch.complex128).cpu().numpy()
    for r in range(R):
        assert rel(y[r], refs[r]) < tol, (prec, RG, RGA, r)
    with pytest.raises(A.AkraError):
        A.akra_plan_set_adjoint_shape(p, prec, R, pa, 3)
    # a fresh plan's default shape and the autotuner's pick give the same operator
    q = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(q, torch.from_numpy(ninv).to(DEV), 1e-3)
    for tune in (False, True):
        if tune:
            A.akra_autotune(q, prec, R)
        y = A.akra_apply_H(q, prec, alm_dev(pairs, prec)).to(torch.complex128).cpu().numpy()
        for r in range(R):
            assert rel(y[r], refs[r]) < tol, (prec, tune, r)


@pytest.mark.parametrize("hemi", ["north", "south", "north_with_equator"])
@pytest.mark.parametrize("prec", [A.F64, A.F32])
def test_one_hemisphere_footprint_matches_oracle(hemi, prec):
    """Footprints in one hemisphere: every active ring pair needs one ring only, and the Legendre
    kernels take the one-ring contraction (the equator ring, alone in its pair, counts as north).
    H and the weighted adjoint against the oracle for several tile shapes, 2 RHS."""
    N, L, R = 16, 40, 2
    rng = np.random.default_rng({"north": 7, "south": 8, "north_with_equator": 9}[hemi])
    th, ph = O.pixel_angles(N)
    z = np.cos(th)
    sel = {"north": z > 0.05, "south": z < -0.05, "north_with_equator": z > -1e-12}[hemi]
    ninv = np.where(sel, 1.0 + rng.random(12 * N * N), 0.0)
    w = O.Weights(N, ninv, 1e-3)
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    refs = [np.stack(O.apply_H(N, L, w, *q)) for q in pairs]
    tol = TOL64 if prec == A.F64 else tol32(L)
    shapes = [(1, 1, 1), (2, 4, 1), (1, 2, 2)] if prec == A.F64 else [(1, 5, 1), (2, 3, 1), (1, 1, 2)]
    for P, PA, RG in shapes:
        p = A.akra_plan_create(N, L)
        A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
        A.akra_plan_set_shape(p, prec, R, P, PA if RG == 1 else 1, RG)
        y = A.akra_apply_H(p, prec, alm_dev(pairs, prec)).to(torch.complex128).cpu().numpy()
        for r in range(R):
            assert rel(y[r], refs[r]) < tol, (hemi, prec, P, PA, RG, r, rel(y[r], refs[r]))


@pytest.mark.parametrize("prec", [A.F32, A.F64])
def test_mostly_one_ring_footprint_matches_oracle(prec):
    """A southern footprint with a thin band just north of the equator: nearly every active ring
    pair needs its south ring only and one needs both, so one warp of the Legendre kernels takes
    the two-ring contraction and the rest the one-ring one. H against the oracle for every
    adjoint width."""
    N, L, R = 16, 40, 2
    rng = np.random.default_rng(41)
    th, ph = O.pixel_angles(N)
    z = np.cos(th)
    ninv = np.where(z < 0.08, 1.0 + rng.random(12 * N * N), 0.0)
    # the unit mix the test relies on: at least 90 % of the active pairs need one ring, not all
    act = [bool(np.any(ninv[first:first + n] > 0)) for _, _, n, _, first in O.rings(N)]
    nr = len(act)
    units = [(act[u], act[nr - 1 - u] if nr - 1 - u != u else False) for u in range((nr + 1) // 2)]
    both = sum(1 for a, b in units if a and b)
    active = sum(1 for a, b in units if a or b)
    assert 0 < both and (active - both) * 10 >= active * 9, (both, active)
    w = O.Weights(N, ninv, 1e-3)
    pairs = [(S.random_alm(L, rng), S.random_alm(L, rng)) for _ in range(R)]
    refs = [np.stack(O.apply_H(N, L, w, *q)) for q in pairs]
    tol = TOL64 if prec == A.F64 else tol32(L)
    p = A.akra_plan_create(N, L)
    A.akra_plan_set_weights(p, torch.from_numpy(ninv).to(DEV), 1e-3)
    d = A.akra_plan_describe(p)
    assert 0 < d["legendre_steps_f32_one_ring"] < d["legendre_steps_f32"]
    widths = (3, 4, 5, 6, 8) if prec == A.F32 else (1, 2, 4)
    for PA in widths:
        A.akra_plan_set_shape(p, prec, R, 1, PA, 1)
        A.akra_plan_set_adjoint_shape(p, prec, R, PA, 1)
        y = A.akra_apply_H(p, prec, alm_dev(pairs, prec)).to(torch.complex128).cpu().numpy()
        for r in range(R):
            assert rel(y[r], refs[r]) < tol, (prec, PA, r, rel(y[r], refs[r]))
