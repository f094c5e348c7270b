"""Differentiation through the CG solve (the autograd form).

CPU: the oracle's analytic gradient (implicit adjoint CG) is pinned by central finite
differences of the oracle's own forward solve, and the band-power loss gradient by finite
differences of the loss.  GPU: torch.autograd through libakra.so against the oracle's
gradient, against central finite differences (FP64 solves at tol 1e-12, step 1e-4 relative)
on 20 pixels, and mixed precision against FP64.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
import synthetic as S


def _problem(N=4, L=6, seed=0):
    rng = np.random.default_rng(seed)
    th, ph = O.pixel_angles(N)
    npix = 12 * N * N
    ninv = np.where(th > 0.9, rng.uniform(100, 400, npix), 0.0)
    kE = S.random_alm(L, rng, lmin=2) * 0.1
    y = np.stack(O.forward_A(N, L, kE, np.zeros_like(kE))) + 0.02 * rng.normal(size=(2, npix))
    y = np.where(ninv > 0, y, 0.0)
    return N, L, ninv, y, rng


def _edges(L):
    return np.geomspace(1.5, L, 5)


def test_band_power_gradient_finite_differences():
    L = 9
    rng = np.random.default_rng(3)
    kE = S.random_alm(L, rng)
    ed = _edges(L)
    g = O.band_power_grad(L, kE, ed)
    _, ms = O.lm_arrays(L)
    h = 1e-6
    for ix in rng.choice(len(kE), 12, replace=False):
        for part in (1.0, 1j):
            if part == 1j and ms[ix] == 0:
                continue
            kp = kE.copy()
            kp[ix] += h * part
            km = kE.copy()
            km[ix] -= h * part
            fd = (O.band_power_loss(L, kp, ed) - O.band_power_loss(L, km, ed)) / (2 * h)
            an = g[ix].real if part == 1.0 else g[ix].imag
            assert abs(fd - an) < 1e-7 * max(1.0, abs(an))


def test_oracle_solve_gradient_matches_finite_differences():
    N, L, ninv, y, rng = _problem()
    ed = _edges(L)
    lam = 1e-3
    gfun = lambda x: (O.band_power_grad(L, x[0], ed), np.zeros_like(x[1]))
    (xE, xB), dy, dn = O.solve_grad(N, L, ninv, y, lam, gfun)
    w0 = O.Weights(N, ninv, lam)

    def loss(yv, nv):
        # λ_eff held fixed at its value for the unperturbed N^-1
        w = O.Weights(N, nv, lam)
        w.lam_eff = w0.lam_eff
        (e, b), _, _, _ = O.pcg(lambda a, c: O.apply_H(N, L, w, a, c), O.rhs_b(N, L, w, yv[0], yv[1]),
                                w.precond, L, 1e-13, 5000)
        return O.band_power_loss(L, e, ed)

    mask = np.flatnonzero(ninv > 0)
    for p in rng.choice(mask, 4, replace=False):
        for c in (0, 1):
            h = 1e-4 * max(abs(y[c, p]), 1e-3)
            yp, ym = y.copy(), y.copy()
            yp[c, p] += h
            ym[c, p] -= h
            fd = (loss(yp, ninv) - loss(ym, ninv)) / (2 * h)
            assert abs(fd - dy[c, p]) < 1e-6 * max(abs(fd), 1e-12) + 1e-14, (p, c, fd, dy[c, p])
        h = 1e-4 * ninv[p]
        np_, nm = ninv.copy(), ninv.copy()
        np_[p] += h
        nm[p] -= h
        fd = (loss(y, np_) - loss(y, nm)) / (2 * h)
        assert abs(fd - dn[p]) < 1e-6 * max(abs(fd), 1e-14) + 1e-16, (p, fd, dn[p])


def test_torch_complex_gradient_convention():
    torch = pytest.importorskip("torch")
    z = torch.tensor([1.0 + 2.0j], dtype=torch.complex128, requires_grad=True)
    (z.real ** 2 + 3 * z.imag ** 2).sum().backward()
    assert torch.allclose(z.grad, torch.tensor([2.0 + 12.0j], dtype=torch.complex128))


# ---------------------------------------------------------------------------
# GPU
# ---------------------------------------------------------------------------
def _gpu_case(N, L, seed, prec_name="F64"):
    torch = pytest.importorskip("torch")
    from paper_2606_06175_gb300 import akra as A
    from paper_2606_06175_gb300.autograd import akra_solve, band_power_loss

    rng = np.random.default_rng(seed)
    sv = S.survey(N, "des" if N >= 64 else "full", 1005)
    ninv = sv["ninv"]
    if N < 64:
        th, _ = O.pixel_angles(N)
        ninv = np.where(th > 0.9, ninv, 0.0)
    kE = S.grf_alm(L, S.cl_kappa(L), rng)
    y = np.stack(O.forward_A(N, L, kE, np.zeros_like(kE))) if N <= 32 else None
    return torch, A, akra_solve, band_power_loss, ninv, kE, y, rng


@pytest.mark.gpu
def test_autograd_fp64_matches_oracle_gradient():
    N, L = 16, 24
    torch, A, akra_solve, bpl, ninv, kE, y, rng = _gpu_case(N, L, 1)
    y = y + 0.01 * rng.normal(size=y.shape)
    y = np.where(ninv > 0, y, 0.0)
    ed = np.geomspace(2, L, 9)
    plan = A.akra_plan_create(N, L)
    yt = torch.tensor(y, dtype=torch.float64, device="cuda", requires_grad=True)
    nt = torch.tensor(ninv, dtype=torch.float64, device="cuda", requires_grad=True)
    x = akra_solve(yt, nt, plan, A.F64, tol=1e-12, maxiter=4000)
    loss = bpl(x, L, ed)
    loss.backward()
    gfun = lambda xx: (O.band_power_grad(L, xx[0], ed), np.zeros_like(xx[1]))
    (xE, xB), dy, dn = O.solve_grad(N, L, ninv, y, 1e-3, gfun, tol=1e-13)
    assert abs(float(loss.detach()) - O.band_power_loss(L, xE, ed)) < 1e-10 * abs(float(loss.detach()))
    gy = yt.grad.cpu().numpy()
    gn = nt.grad.cpu().numpy()
    assert np.linalg.norm(gy - dy) < 1e-8 * np.linalg.norm(dy)
    assert np.linalg.norm(gn - dn) < 1e-8 * np.linalg.norm(dn)


@pytest.mark.gpu
def test_autograd_fp64_finite_differences_20_pixels():
    """Central differences (step 1e-4 relative, FP64 solves at tol 1e-12) on 20 mask pixels."""
    N, L = 64, 128
    torch, A, akra_solve, bpl, ninv, kE, _, rng = _gpu_case(N, L, 2)
    plan = A.akra_plan_create(N, L)
    x_true = torch.tensor(np.stack([kE, np.zeros_like(kE)])[None], device="cuda")
    A.akra_plan_set_weights(plan, torch.tensor(ninv, device="cuda"), 1e-3)
    y = A.akra_apply_A(plan, A.F64, x_true)[0].cpu().numpy() + \
        S.shape_noise(ninv, np.random.default_rng(5))[0]
    y = np.where(ninv > 0, y, 0.0).astype(np.float32)
    ed = np.geomspace(10, L, 9)
    yt = torch.tensor(y, device="cuda", requires_grad=True)
    nt = torch.tensor(ninv, device="cuda", requires_grad=True)
    loss = bpl(akra_solve(yt, nt, plan, A.F64, tol=1e-12, maxiter=6000), L, ed)
    loss.backward()
    gy, gn = yt.grad.cpu().numpy(), nt.grad.cpu().numpy()
    lam_eff = A.akra_plan_describe(plan)["lambda_eff"]

    def L_of(yv, nv):
        # λ_eff held fixed: rescale λ so that λ <N^-1>_M stays at the unperturbed value
        lam = lam_eff / nv[nv > 0].mean()
        with torch.no_grad():
            xx = akra_solve(torch.tensor(yv, device="cuda"), torch.tensor(nv, device="cuda"), plan,
                            A.F64, tol=1e-12, maxiter=6000, lam=lam)
            return float(bpl(xx, L, ed))

    # the loss is quadratic in y, so central differences are exact up to the solver's own
    # error; the step is 1e-4 of the map scale and the check has a floor at 1e-6 max|g|
    pix = rng.choice(np.flatnonzero(ninv > 0), 20, replace=False)
    ymax = float(np.abs(y).max())
    for k, p in enumerate(pix):
        c = k % 2
        h = 1e-4 * ymax
        yp, ym = y.astype(np.float64), y.astype(np.float64)
        yp = yp.copy(); ym = ym.copy()
        yp[c, p] += h
        ym[c, p] -= h
        fd = (L_of(yp, ninv) - L_of(ym, ninv)) / (2 * h)
        assert abs(fd - gy[c, p]) < 1e-5 * abs(fd) + 1e-6 * np.abs(gy).max(), (p, fd, gy[c, p])
    for p in pix[:6]:
        h = 1e-4 * ninv[p]
        np_, nm = ninv.copy(), ninv.copy()
        np_[p] += h
        nm[p] -= h
        fd = (L_of(y.astype(np.float64), np_) - L_of(y.astype(np.float64), nm)) / (2 * h)
        assert abs(fd - gn[p]) < 1e-5 * abs(fd) + 1e-6 * np.abs(gn).max(), (p, fd, gn[p])


@pytest.mark.gpu
def test_autograd_mixed_close_to_fp64_at_nside512():
    """The differentiation workload's size (Nside 512, lmax 1024): mixed-precision gradients
    within 1e-3 of the FP64 ones; FP64 directional derivative against central differences."""
    N, L = 512, 1024
    torch, A, akra_solve, bpl, ninv, kE, _, rng = _gpu_case(N, L, 3)
    plan = A.akra_plan_create(N, L)
    x_true = torch.tensor(np.stack([kE, np.zeros_like(kE)])[None], device="cuda")
    A.akra_plan_set_weights(plan, torch.tensor(ninv, device="cuda"), 1e-3)
    y = A.akra_apply_A(plan, A.F64, x_true)[0] + torch.tensor(
        S.shape_noise(ninv, np.random.default_rng(6))[0], device="cuda")
    y = torch.where(torch.tensor(ninv > 0, device="cuda"), y, 0.0).float()
    ed = np.geomspace(10, 1024, 9)
    grads = {}
    for name, prec, tol in (("f64", A.F64, 1e-10), ("mixed", A.MIXED, 1e-8)):
        yt = y.clone().requires_grad_(True)
        nt = torch.tensor(ninv, device="cuda", requires_grad=True)
        bpl(akra_solve(yt, nt, plan, prec, tol=tol, maxiter=6000), L, ed).backward()
        grads[name] = (yt.grad.double(), nt.grad.double())
    for a, b in zip(grads["mixed"], grads["f64"]):
        assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b)) < 1e-3
    # directional derivative of the FP64 loss along a random masked direction of y
    v = torch.randn_like(y, dtype=torch.float64) * torch.tensor(ninv > 0, device="cuda")
    h = 1e-4 * float(y.abs().max())
    with torch.no_grad():
        lp = float(bpl(akra_solve(y.double() + h * v, torch.tensor(ninv, device="cuda"), plan, A.F64,
                                  tol=1e-10, maxiter=6000), L, ed))
        lm = float(bpl(akra_solve(y.double() - h * v, torch.tensor(ninv, device="cuda"), plan, A.F64,
                                  tol=1e-10, maxiter=6000), L, ed))
    fd = (lp - lm) / (2 * h)
    an = float((grads["f64"][0] * v).sum())
    assert abs(fd - an) < 1e-5 * abs(an), (fd, an)
