"""Plain FP64 CPU oracle for the AKRA 3.0 hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s cpu_baseline /
reference leg import this module.  It shares no code with the CUDA library
(``paper_2606_06175_gb300``) and never imports it.

Two tiers:

* O1 -- direct sums over pixels of the Goldberg et al. (1967) spin-weighted
  harmonics evaluated in arbitrary precision (mpmath); tiny sizes only.
* O2 -- the same operators with the harmonics separated as
  ``sY_lm(θ,φ) = sλ_lm(θ) e^{imφ}``: Legendre sums in plain C
  (``akra_oracle.c``), per-ring phase sums here with numpy's FFT as a library
  step.

Operator chain (Sec. II B, "The storage problem"):
``x = (κ_E, κ_B)  --KS, Eq. 3-->  (a_E, a_B)  --SHT^-1, Eqs. 1-2-->  γ on pixels
--×W-->  --exact transpose-->  (Hx) + λ_eff x`` (Eq. 14), solved by PCG
(Sec. II B, "The inversion problem"; preconditioner Eq. 15).

Readings where the paper is silent or inconsistent:
  * KS sign: Eq. 3, γ_{±2,lm} = D_l κ_lm, i.e. a_E = -D_l κ_E and likewise for B.
  * W_p = ω M_p N^{-1}_p with ω = 4π/N_pix; λ_eff = λ · mean of N^{-1} over the
    unmasked pixels; preconditioner P = 1/(mean over all pixels of M N^{-1} + λ_eff).
  * the harmonic vector is real (κ_{l,-m} = (-1)^m conj κ_lm) and its inner
    product counts every real degree of freedom:
    <x,y> = Σ_l [x_l0 y_l0 + 2 Re Σ_{m>0} x_lm conj(y_lm)].
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from functools import lru_cache

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "akra_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the C half of the oracle (plain gcc, FP64, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


@lru_cache(maxsize=1)
def _lib():
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.orc_ring_info.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, llp, ip, llp]
    lib.orc_ring_info.restype = ctypes.c_int
    lib.orc_spin_lambda.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_double, dp]
    lib.orc_spin_lambda.restype = None
    lib.orc_legendre_synth.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int, ip, dp]
    lib.orc_legendre_synth.restype = None
    lib.orc_legendre_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, dp, dp]
    lib.orc_legendre_adjoint.restype = None
    lib.orc_num_threads.argtypes = []
    lib.orc_num_threads.restype = ctypes.c_int
    return lib


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    return int(_lib().orc_num_threads())


# ----------------------------------------------------------------------------
# index helpers (packed m-major triangle)
# ----------------------------------------------------------------------------
def ntri(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def tri_index(lmax: int, l: int, m: int) -> int:
    return m * (2 * lmax + 1 - m) // 2 + l


@lru_cache(maxsize=16)
def lm_arrays(lmax: int):
    """(l, m) of every packed index."""
    ls = np.empty(ntri(lmax), np.int64)
    ms = np.empty(ntri(lmax), np.int64)
    for m in range(lmax + 1):
        i0 = tri_index(lmax, m, m)
        ls[i0:i0 + lmax + 1 - m] = np.arange(m, lmax + 1)
        ms[i0:i0 + lmax + 1 - m] = m
    return ls, ms


# ----------------------------------------------------------------------------
# geometry
# ----------------------------------------------------------------------------
def ring_info(nside: int, ring: int):
    """(cosθ, sinθ, nφ, σ, first pixel) of ring 1..4N-1 (HEALPix RING)."""
    ct, st = ctypes.c_double(), ctypes.c_double()
    n, first = ctypes.c_longlong(), ctypes.c_longlong()
    sg = ctypes.c_int()
    rc = _lib().orc_ring_info(nside, ring, ctypes.byref(ct), ctypes.byref(st), ctypes.byref(n),
                              ctypes.byref(sg), ctypes.byref(first))
    if rc != 0:
        raise ValueError("ring out of range")
    return ct.value, st.value, n.value, sg.value, first.value


@lru_cache(maxsize=8)
def rings(nside: int):
    return [ring_info(nside, r) for r in range(1, 4 * nside)]


def pixel_angles(nside: int):
    """(θ, φ) of every pixel, RING order; φ_j = π(2j+σ)/nφ."""
    npix = 12 * nside * nside
    theta = np.empty(npix)
    phi = np.empty(npix)
    for ct, st, n, sg, first in rings(nside):
        theta[first:first + n] = math.atan2(st, ct)
        phi[first:first + n] = np.pi * (2 * np.arange(n) + sg) / n
    return theta, phi


# ----------------------------------------------------------------------------
# spin-weighted harmonics
# ----------------------------------------------------------------------------
def spin_lambda(s: int, lmax: int, m: int, theta: float) -> np.ndarray:
    """sλ_lm(θ), l = 0..lmax (O2 recurrence, C)."""
    out = np.zeros(lmax + 1)
    _lib().orc_spin_lambda(int(s), int(lmax), int(m), math.cos(theta), math.sin(theta), _dptr(out))
    return out


def goldberg_sYlm(s: int, l: int, m: int, theta: float, phi: float, dps: int = 40) -> complex:
    """O1: Goldberg et al. (1967) closed form of sY_lm, evaluated with mpmath.

    sY_lm = (-1)^m sqrt((l+m)!(l-m)!(2l+1) / (4π (l+s)!(l-s)!)) sin^{2l}(θ/2)
            Σ_r C(l-s, r) C(l+s, r+s-m) (-1)^{l-r-s} e^{imφ} cot^{2r+s-m}(θ/2)
    """
    import mpmath as mp

    if l < abs(s) or l < abs(m):
        return 0j
    with mp.workdps(dps):
        th = mp.mpf(theta)
        pref = (-1) ** m * mp.sqrt(mp.factorial(l + m) * mp.factorial(l - m) * (2 * l + 1)
                                   / (4 * mp.pi * mp.factorial(l + s) * mp.factorial(l - s)))
        sh, ch = mp.sin(th / 2), mp.cos(th / 2)
        tot = mp.mpf(0)
        for r in range(0, l - s + 1):
            k = r + s - m
            if k < 0 or k > l + s:
                continue
            p = 2 * r + s - m
            # sin^{2l} cot^p = sin^{2l-p} cos^p (exponents are >= 0 here)
            tot += mp.binomial(l - s, r) * mp.binomial(l + s, k) * (-1) ** (l - r - s) \
                * sh ** (2 * l - p) * ch ** p
        val = pref * tot * mp.expj(m * mp.mpf(phi))
        return complex(val)


# ----------------------------------------------------------------------------
# spin-2 synthesis and its exact adjoint (Eqs. 1-2)
# ----------------------------------------------------------------------------
def _as_packed(a, lmax) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    assert a.shape == (ntri(lmax),)
    return a


def legendre_synth(nside: int, lmax: int, aE, aB, ring_list=None) -> np.ndarray:
    """F(ring, m) = Σ_l γ_{2,lm} 2λ_lm(θ_ring), m = -L..L (rows follow ring_list)."""
    aE = _as_packed(aE, lmax).view(np.float64)
    aB = _as_packed(aB, lmax).view(np.float64)
    if ring_list is None:
        ring_list = np.arange(1, 4 * nside, dtype=np.int32)
    ring_list = np.ascontiguousarray(ring_list, dtype=np.int32)
    F = np.zeros((len(ring_list), 2 * lmax + 1), np.complex128)
    _lib().orc_legendre_synth(nside, lmax, _dptr(aE), _dptr(aB), len(ring_list), _iptr(ring_list),
                              _dptr(F.view(np.float64)))
    return F


def ring_phase_sum(F_row: np.ndarray, lmax: int, n: int, sigma: int) -> np.ndarray:
    """f_j = Σ_{m=-L}^{L} F(m) e^{imφ_j},  φ_j = π(2j+σ)/n.

    Since e^{imφ_j} = e^{iπmσ/n} e^{2πijm/n} and the second factor depends on m
    only through m mod n, the sum regroups exactly as
    f_j = Σ_k e^{2πijk/n} Σ_{m≡k (mod n)} F(m) e^{iπmσ/n},
    and the k-sum is numpy's inverse FFT (a library step).
    """
    m = np.arange(-lmax, lmax + 1)
    t = np.mod(m * sigma, 2 * n)  # exact integer reduction of the phase
    ph = np.exp(1j * np.pi * t / n)
    bins = np.zeros(n, np.complex128)
    np.add.at(bins, np.mod(m, n), F_row * ph)
    return np.fft.ifft(bins) * n


def ring_phase_adjoint(w: np.ndarray, lmax: int, sigma: int) -> np.ndarray:
    """G(m) = Σ_j w_j e^{-imφ_j}, m = -L..L (exact transpose of ring_phase_sum).

    G(m) = e^{-iπmσ/n} Σ_j w_j e^{-2πi j m/n} = e^{-iπmσ/n} fft(w)[m mod n].
    """
    n = len(w)
    m = np.arange(-lmax, lmax + 1)
    t = np.mod(m * sigma, 2 * n)
    W = np.fft.fft(w)
    return np.exp(-1j * np.pi * t / n) * W[np.mod(m, n)]


def synth_spin2(nside: int, lmax: int, aE, aB):
    """γ = Σ_lm γ_{2,lm} 2Y_lm with γ_{2,lm} = -(a_E + i a_B) (Eqs. 1-2).

    Returns (γ1, γ2) = (Re γ, Im γ) on all pixels in RING order.
    """
    F = legendre_synth(nside, lmax, aE, aB)
    npix = 12 * nside * nside
    g = np.zeros(npix, np.complex128)
    for k, (ct, st, n, sg, first) in enumerate(rings(nside)):
        g[first:first + n] = ring_phase_sum(F[k], lmax, n, sg)
    return g.real.copy(), g.imag.copy()


def adjoint_synth_spin2(nside: int, lmax: int, u1, u2, m_list=None):
    """Exact transpose of synth_spin2 in the real-dof inner product.

    With w = u1 + i u2, g_lm = Σ_p w_p 2Y*_lm and h_lm = Σ_p conj(w_p) (-2)Y*_lm,
    the transpose is (a_E, a_B) = (-(g+h)/2, (i/2)(g-h)), i.e. Eq. 2 applied to
    (g, h).  The m = 0 entries are real.
    """
    w = np.asarray(u1, np.float64) + 1j * np.asarray(u2, np.float64)
    G = np.zeros((4 * nside - 1, 2 * lmax + 1), np.complex128)
    for k, (ct, st, n, sg, first) in enumerate(rings(nside)):
        G[k] = ring_phase_adjoint(w[first:first + n], lmax, sg)
    if m_list is None:
        m_list = np.arange(lmax + 1, dtype=np.int32)
    m_list = np.ascontiguousarray(m_list, dtype=np.int32)
    g = np.zeros(ntri(lmax), np.complex128)
    h = np.zeros(ntri(lmax), np.complex128)
    _lib().orc_legendre_adjoint(nside, lmax, _dptr(G.view(np.float64)), len(m_list), _iptr(m_list),
                                _dptr(g.view(np.float64)), _dptr(h.view(np.float64)))
    aE = -(g + h) / 2
    aB = 0.5j * (g - h)
    ls, ms = lm_arrays(lmax)
    aE[ms == 0] = aE[ms == 0].real
    aB[ms == 0] = aB[ms == 0].real
    return aE, aB


# ----------------------------------------------------------------------------
# O1: direct sums over pixels (tiny sizes)
# ----------------------------------------------------------------------------
def direct_synth_spin2(nside: int, lmax: int, aE, aB):
    """γ(p) = Σ_{l>=2} Σ_{m=-l}^{l} -(a_E,lm + i a_B,lm) 2Y_lm(p), Goldberg 2Y, real fields."""
    theta, phi = pixel_angles(nside)
    g = np.zeros(len(theta), np.complex128)
    for l in range(2, lmax + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            ix = tri_index(lmax, l, am)
            e, b = complex(aE[ix]), complex(aB[ix])
            if am == 0:
                e, b = complex(e.real), complex(b.real)
            if m < 0:
                sgn = (-1) ** am
                e, b = sgn * e.conjugate(), sgn * b.conjugate()
            c2 = -(e + 1j * b)
            Y = np.array([goldberg_sYlm(2, l, m, t, p, dps=30) for t, p in zip(theta, phi)])
            g += c2 * Y
    return g.real.copy(), g.imag.copy()


# ----------------------------------------------------------------------------
# KS kernel, weights, H (Eqs. 3, 7-9, 14-15)
# ----------------------------------------------------------------------------
def ks_kernel(lmax: int) -> np.ndarray:
    """D_l = -sqrt((l-1)(l+2)/(l(l+1))) (Eq. 3); D_0 := 0 (0/0), D_1 = 0."""
    D = np.zeros(lmax + 1)
    l = np.arange(2, lmax + 1, dtype=np.float64)
    D[2:] = -np.sqrt((l - 1) * (l + 2) / (l * (l + 1)))
    return D


def forward_A(nside: int, lmax: int, kE, kB):
    """A x: a_E = -D_l κ_E, a_B = -D_l κ_B (Eq. 3 with Eq. 2), then SHT^-1 (Eq. 1)."""
    ls, _ = lm_arrays(lmax)
    D = ks_kernel(lmax)[ls]
    return synth_spin2(nside, lmax, -D * np.asarray(kE), -D * np.asarray(kB))


def adjoint_A(nside: int, lmax: int, u1, u2):
    """A^T u = diag(-D_l) (SHT^-1)^T u."""
    ls, _ = lm_arrays(lmax)
    D = ks_kernel(lmax)[ls]
    aE, aB = adjoint_synth_spin2(nside, lmax, u1, u2)
    return -D * aE, -D * aB


class Weights:
    """W_p = ω M_p N^{-1}_p, λ_eff = λ <N^{-1}>_M, P = (<M N^{-1}> + λ_eff)^{-1} (Eqs. 14-15)."""

    def __init__(self, nside: int, ninv, lam: float = 1e-3):
        ninv = np.asarray(ninv, np.float64)
        npix = 12 * nside * nside
        assert ninv.shape == (npix,)
        mask = ninv > 0
        self.nside = nside
        self.omega = 4 * np.pi / npix
        self.W = self.omega * np.where(mask, ninv, 0.0)
        self.lam = lam
        self.lam_eff = lam * (ninv[mask].mean() if mask.any() else 0.0)
        self.mean_mninv = np.where(mask, ninv, 0.0).mean()
        self.precond = 1.0 / (self.mean_mninv + self.lam_eff)


def apply_H(nside: int, lmax: int, wts: Weights, kE, kB):
    """H_λ x = A^T W A x + λ_eff x (Eq. 14 operator)."""
    g1, g2 = forward_A(nside, lmax, kE, kB)
    hE, hB = adjoint_A(nside, lmax, wts.W * g1, wts.W * g2)
    return hE + wts.lam_eff * np.asarray(kE), hB + wts.lam_eff * np.asarray(kB)


def rhs_b(nside: int, lmax: int, wts: Weights, y1, y2):
    """b = A^T N^{-1} y (Eq. 8; the misprint in Sec. II B's CG display is read as Eq. 8)."""
    return adjoint_A(nside, lmax, wts.W * np.asarray(y1), wts.W * np.asarray(y2))


def realdof_dot(lmax: int, x, y) -> float:
    """<x,y> over the real degrees of freedom: Σ_l [x_l0 y_l0 + 2 Re Σ_{m>0} x conj(y)]."""
    _, ms = lm_arrays(lmax)
    x = np.asarray(x)
    y = np.asarray(y)
    w = np.where(ms == 0, 1.0, 2.0)
    xr, yr = x.real, y.real
    xi = np.where(ms == 0, 0.0, x.imag)
    yi = np.where(ms == 0, 0.0, y.imag)
    return float(np.sum(w * (xr * yr + xi * yi)))


def pair_dot(lmax, x, y) -> float:
    return realdof_dot(lmax, x[0], y[0]) + realdof_dot(lmax, x[1], y[1])


def pcg(apply, b, precond, lmax: int, tol: float, maxiter: int, x0=None):
    """Preconditioned CG (Saad 2003, as cited in Sec. II B) on pairs (κ_E, κ_B).

    `precond` is the scalar P of Eq. 15 or an array of per-packed-index weights (a diagonal
    preconditioner applied to both fields).

    x_0 = 0, r_0 = b, z = P r, p = z; each step q = H p, α = <r,z>/<p,q>,
    x += α p, r -= α q, stop when ||r||/||b|| < tol, β = <r',z'>/<r,z>, p = z' + β p.
    Returns (x, iterations, recursive relative residual, history of (α, β)).
    """
    bE, bB = (np.asarray(v, np.complex128) for v in b)
    if x0 is None:
        xE, xB = np.zeros_like(bE), np.zeros_like(bB)
        rE, rB = bE.copy(), bB.copy()
    else:
        xE, xB = (np.asarray(v, np.complex128).copy() for v in x0)
        hE, hB = apply(xE, xB)
        rE, rB = bE - hE, bB - hB
    bnorm = math.sqrt(pair_dot(lmax, (bE, bB), (bE, bB)))
    if bnorm == 0:
        return (xE, xB), 0, 0.0, []
    zE, zB = precond * rE, precond * rB
    pE, pB = zE.copy(), zB.copy()
    rz = pair_dot(lmax, (rE, rB), (zE, zB))
    hist = []
    it = 0
    relres = math.sqrt(pair_dot(lmax, (rE, rB), (rE, rB))) / bnorm
    while relres >= tol and it < maxiter:
        qE, qB = apply(pE, pB)
        alpha = rz / pair_dot(lmax, (pE, pB), (qE, qB))
        xE, xB = xE + alpha * pE, xB + alpha * pB
        rE, rB = rE - alpha * qE, rB - alpha * qB
        it += 1
        relres = math.sqrt(pair_dot(lmax, (rE, rB), (rE, rB))) / bnorm
        zE, zB = precond * rE, precond * rB
        rz_new = pair_dot(lmax, (rE, rB), (zE, zB))
        beta = rz_new / rz
        rz = rz_new
        hist.append((alpha, beta))
        if relres < tol:
            break
        pE, pB = zE + beta * pE, zB + beta * pB
    return (xE, xB), it, relres, hist


def per_l_preconditioner(lmax: int, wts: Weights):
    """Per-l diagonal preconditioner (mean_all(M N^-1) D_l^2 + λ_eff)^-1 per packed index: the
    uniform-sky diagonal of H with the Eq. 3 kernel (beyond the paper's scalar Eq. 15)."""
    ls, _ = lm_arrays(lmax)
    D = ks_kernel(lmax)
    d = wts.mean_mninv * D[ls] ** 2 + wts.lam_eff
    return np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)


def cg_solve(nside: int, lmax: int, wts: Weights, y1, y2, tol: float = 1e-8, maxiter: int = 1000):
    """x̂ = (A^T N^{-1} A + λ_eff I)^{-1} A^T N^{-1} y (Eq. 14) by PCG."""
    b = rhs_b(nside, lmax, wts, y1, y2)
    return pcg(lambda e, bb: apply_H(nside, lmax, wts, e, bb), b, wts.precond, lmax, tol, maxiter)


def cg_solve_E(nside: int, lmax: int, wts: Weights, y1, y2, tol: float = 1e-8, maxiter: int = 1000):
    """E-mode normal equations H_EE κ_E = b_E (App. A: the E block row and column of Eq. A3,
    κ_B held at zero) by PCG on the E field; returns ((κ̂_E, 0), iterations, relres, history)."""
    bE, _ = rhs_b(nside, lmax, wts, y1, y2)
    zero = np.zeros_like(bE)

    def apply_EE(e, _b):
        hE, _ = apply_H(nside, lmax, wts, e, zero)
        return hE, zero

    return pcg(apply_EE, (bE, zero), wts.precond, lmax, tol, maxiter)


def cg_solve_B_given_E(nside: int, lmax: int, wts: Weights, y1, y2, kE, tol: float = 1e-8,
                       maxiter: int = 1000):
    """Conditional B-mode solve (App. A, Eq. A8): H_BB κ_B = b_B - H_BE κ̂_E, where H_BE κ̂_E is
    the B part of H applied to (κ̂_E, 0).  Returns ((0, κ̂_B), iterations, relres, history)."""
    _, bB = rhs_b(nside, lmax, wts, y1, y2)
    zero = np.zeros_like(bB)
    _, hBE = apply_H(nside, lmax, wts, np.asarray(kE, np.complex128), zero)
    rhs = bB - hBE

    def apply_BB(_e, b):
        _, hB = apply_H(nside, lmax, wts, zero, b)
        return zero, hB

    return pcg(apply_BB, (zero, rhs), wts.precond, lmax, tol, maxiter)


def lanczos_condition(hist) -> float:
    """κ of the (preconditioned) operator from CG's α, β (the CG-Lanczos tridiagonal)."""
    k = len(hist)
    if k == 0:
        return 1.0
    T = np.zeros((k, k))
    for j, (a, _) in enumerate(hist):
        T[j, j] = 1.0 / a + (hist[j - 1][1] / hist[j - 1][0] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(hist[j][1]) / a
    ev = np.linalg.eigvalsh(T)
    return float(ev.max() / ev.min())


# ----------------------------------------------------------------------------
# dense H (the AKRA 2.0 object, Sec. II B "Calculation problem") at tiny lmax
# ----------------------------------------------------------------------------
def realdof_basis(lmax: int):
    """Orthonormal basis of one real field in the real-dof inner product.

    m = 0: unit real part;  m > 0: real or imaginary part 1/sqrt(2).
    Returns a list of (packed index, complex value) for l = 0..lmax.
    """
    out = []
    s = 1.0 / math.sqrt(2.0)
    for m in range(lmax + 1):
        for l in range(m, lmax + 1):
            ix = tri_index(lmax, l, m)
            if m == 0:
                out.append((ix, 1.0 + 0j))
            else:
                out.append((ix, s + 0j))
                out.append((ix, 1j * s))
    return out


def dense_H(nside: int, lmax: int, wts: Weights):
    """Dense H_λ in an orthonormal real-dof basis of (κ_E, κ_B), column by column."""
    basis = realdof_basis(lmax)
    nt = ntri(lmax)
    cols = []
    vecs = []
    for field in (0, 1):
        for ix, v in basis:
            e = np.zeros(nt, np.complex128)
            b = np.zeros(nt, np.complex128)
            (e if field == 0 else b)[ix] = v
            vecs.append((e, b))
    for e, b in vecs:
        cols.append(apply_H(nside, lmax, wts, e, b))
    n = len(vecs)
    H = np.zeros((n, n))
    for j in range(n):
        for i in range(n):
            H[i, j] = pair_dot(lmax, vecs[i], cols[j])
    return H, vecs


def cholesky_solve(nside: int, lmax: int, wts: Weights, b):
    """x̂ = H_λ^{-1} b with dense H_λ and LAPACK Cholesky (the direct AKRA 2.0 route)."""
    H, vecs = dense_H(nside, lmax, wts)
    rhs = np.array([pair_dot(lmax, v, b) for v in vecs])
    Lc = np.linalg.cholesky(H)
    c = np.linalg.solve(Lc.T, np.linalg.solve(Lc, rhs))
    xE = sum(ci * v[0] for ci, v in zip(c, vecs))
    xB = sum(ci * v[1] for ci, v in zip(c, vecs))
    return (xE, xB), H


# ----------------------------------------------------------------------------
# band-power loss and its gradient (the differentiation workload)
# ----------------------------------------------------------------------------
def band_power_loss(lmax: int, kE, edges) -> float:
    """Σ_b mean_{l in (e_b, e_{b+1}]} C_l^E,  C_l^E = [|κ_l0|^2 + 2 Σ_{m>0}|κ_lm|^2]/(2l+1)."""
    ls, ms = lm_arrays(lmax)
    kE = np.asarray(kE)
    p = np.where(ms == 0, kE.real ** 2, 2 * np.abs(kE) ** 2)
    cl = np.bincount(ls, weights=p, minlength=lmax + 1) / (2 * np.arange(lmax + 1) + 1)
    tot = 0.0
    for b in range(len(edges) - 1):
        sel = (np.arange(lmax + 1) > edges[b]) & (np.arange(lmax + 1) <= edges[b + 1])
        if sel.any():
            tot += cl[sel].mean()
    return float(tot)


def band_power_grad(lmax: int, kE, edges):
    """Gradient of band_power_loss w.r.t. the stored components of κ_E, packed as
    dL/dRe + i dL/dIm (m = 0 imaginary parts do not enter the loss)."""
    ls, ms = lm_arrays(lmax)
    kE = np.asarray(kE)
    ell = np.arange(lmax + 1)
    coef = np.zeros(lmax + 1)
    for b in range(len(edges) - 1):
        sel = (ell > edges[b]) & (ell <= edges[b + 1])
        if sel.any():
            coef[sel] += 1.0 / sel.sum()
    c = coef[ls] / (2 * ls + 1)
    w = np.where(ms == 0, 2.0, 4.0)        # d(x^2)/dx = 2x, doubled for m > 0
    g = c * w * kE.real + 1j * np.where(ms == 0, 0.0, c * 4.0 * kE.imag)
    return g


def shuffle_shear(y, perm):
    """Pixel shuffling of the observed shear (Sec. IV, "Power spectrum results"): output pixel
    p takes the (γ1, γ2) of pixel perm[p]."""
    y = np.asarray(y)
    return np.stack([y[0][perm], y[1][perm]])


def cl_spectra(lmax: int, a, b):
    """C_l^{XY} = [Re a_X,l0 Re b_Y,l0 + 2 Re Σ_{m>0} a_X,lm conj(b_Y,lm)]/(2l+1) for
    (X, Y) = EE, EB, BE, BB (the real-dof inner product of item 3 restricted to one l)."""
    ls, ms = lm_arrays(lmax)
    out = np.zeros((4, lmax + 1))
    for k, (x, y) in enumerate([(a[0], b[0]), (a[0], b[1]), (a[1], b[0]), (a[1], b[1])]):
        x = np.asarray(x)
        y = np.asarray(y)
        prod = np.where(ms == 0, x.real * y.real, 2.0 * (x * np.conj(y)).real)
        out[k] = np.bincount(ls, weights=prod, minlength=lmax + 1) / (2 * np.arange(lmax + 1) + 1)
    return out


def band_powers(cl, edges):
    """Mean of C_l over l in (e_b, e_{b+1}] per bin (0 for an empty bin); cl [..., lmax+1]."""
    cl = np.asarray(cl)
    ell = np.arange(cl.shape[-1])
    out = np.zeros(cl.shape[:-1] + (len(edges) - 1,))
    for b in range(len(edges) - 1):
        sel = (ell > edges[b]) & (ell <= edges[b + 1])
        if sel.any():
            out[..., b] = cl[..., sel].mean(axis=-1)
    return out


def solve_grad(nside: int, lmax: int, ninv, y, lam: float, gfun, tol: float = 1e-13,
               maxiter: int = 5000):
    """x̂ = H^{-1} A^T W y and the gradient of L(x̂) w.r.t. y and N^-1 (λ_eff held fixed).

    gfun(x̂) returns dL/dx̂ on the stored components (dL/dRe + i dL/dIm, for (κ_E, κ_B)).
    With G the real-dof metric (H is self-adjoint in it): u = H^{-1} G^{-1} g,
    dL/dy = W A u, dL/dN^-1_p = ω M_p <(A u)_p, y_p - (A x̂)_p>.
    """
    wts = Weights(nside, ninv, lam)
    y = np.asarray(y, np.float64)
    (xE, xB), _, _, _ = cg_solve(nside, lmax, wts, y[0], y[1], tol=tol, maxiter=maxiter)
    gE, gB = gfun((xE, xB))
    _, ms = lm_arrays(lmax)

    def ginv(v):
        v = np.asarray(v, np.complex128)
        return np.where(ms == 0, v.real + 0j, 0.5 * v)

    (uE, uB), _, _, _ = pcg(lambda e, b: apply_H(nside, lmax, wts, e, b), (ginv(gE), ginv(gB)),
                            wts.precond, lmax, tol, maxiter)
    Au = np.stack(forward_A(nside, lmax, uE, uB))
    Ax = np.stack(forward_A(nside, lmax, xE, xB))
    dy = wts.W * Au
    mask = np.asarray(ninv) > 0
    dninv = np.where(mask, wts.omega * np.sum(Au * (y - Ax), axis=0), 0.0)
    return (xE, xB), dy, dninv


# ----------------------------------------------------------------------------
# flat-sky variant (Sec. II B: each SHT replaced by a 2D FFT; the four steps of the operator
# and the CG solver unchanged).  Unknown x = F(κ_E + i κ_B) on an n x n periodic grid, F the
# unitary 2D DFT (numpy's, norm="ortho", as a library step), rows k2 / y, columns k1 / x.
# ----------------------------------------------------------------------------
def flat_ks_kernel(n: int) -> np.ndarray:
    """D(k) = (k1² - k2² + 2i k1 k2)/|k|², D(0) = 0, at integer FFT frequencies [k2, k1]."""
    k = np.fft.fftfreq(n, d=1.0 / n)
    k1, k2 = k[None, :], k[:, None]
    q = k1 ** 2 + k2 ** 2
    return np.where(q > 0, (k1 ** 2 - k2 ** 2 + 2j * k1 * k2) / np.where(q > 0, q, 1.0), 0.0)


def flat_forward_A(n: int, x):
    """(γ1, γ2) = Re / Im of F^-1 (D x)."""
    z = np.fft.ifft2(flat_ks_kernel(n) * np.asarray(x), norm="ortho")
    return z.real.copy(), z.imag.copy()


def flat_adjoint_A(n: int, u1, u2):
    """conj(D) F (u1 + i u2), the transpose of flat_forward_A in the real inner products."""
    return np.conj(flat_ks_kernel(n)) * np.fft.fft2(np.asarray(u1) + 1j * np.asarray(u2), norm="ortho")


class FlatWeights:
    """W = M N^-1 on the grid (mask M = [N^-1 > 0]), λ_eff (Eq. 14) and the scalar P (Eq. 15)."""

    def __init__(self, ninv, lam: float = 1e-3):
        ninv = np.asarray(ninv, np.float64)
        mask = ninv > 0
        self.W = np.where(mask, ninv, 0.0)
        self.lam_eff = lam * (ninv[mask].mean() if mask.any() else 0.0)
        self.mean_mninv = self.W.mean()
        self.precond = 1.0 / (self.mean_mninv + self.lam_eff)


def flat_apply_H(n: int, wts: FlatWeights, x):
    g1, g2 = flat_forward_A(n, x)
    return flat_adjoint_A(n, wts.W * g1, wts.W * g2) + wts.lam_eff * np.asarray(x)


def flat_rhs_b(n: int, wts: FlatWeights, y1, y2):
    return flat_adjoint_A(n, wts.W * np.asarray(y1), wts.W * np.asarray(y2))


def flat_dot(a, b) -> float:
    """Real inner product of complex arrays: Re Σ conj(a) b."""
    return float(np.real(np.vdot(np.asarray(a), np.asarray(b))))


def flat_cg_solve(n: int, wts: FlatWeights, y1, y2, tol: float = 1e-8, maxiter: int = 1000):
    """PCG (scalar P) on H x = b, b = A^T W y; returns (x, iterations, recursive relres)."""
    b = flat_rhs_b(n, wts, y1, y2)
    x = np.zeros_like(b)
    r = b.copy()
    bn = math.sqrt(flat_dot(b, b))
    if bn == 0:
        return x, 0, 0.0
    z = wts.precond * r
    p = z.copy()
    rz = flat_dot(r, z)
    it, relres = 0, 1.0
    while relres >= tol and it < maxiter:
        q = flat_apply_H(n, wts, p)
        alpha = rz / flat_dot(p, q)
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        relres = math.sqrt(flat_dot(r, r)) / bn
        if relres < tol:
            break
        z = wts.precond * r
        rz_new = flat_dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, it, relres
