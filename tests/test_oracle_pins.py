"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
an independent HEALPix pixel-index routine, library special functions, exact
quadrature identities, brute-force sums, a dense direct solve, and exact
recovery of noise-free data.  The last group plants plausible mistakes in copies
of oracle functions (on the CPU) and checks that a pin catches each of them.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
import synthetic as S


# ---------------------------------------------------------------------------
# HEALPix geometry: an independent ang2pix (Gorski et al. 2005) inverts the
# oracle's ring table pixel by pixel.
# ---------------------------------------------------------------------------
def ang2pix_ring(nside, z, phi):
    N = nside
    za = abs(z)
    tt = (phi / (0.5 * math.pi)) % 4.0
    if za <= 2.0 / 3.0:
        t1 = N * (0.5 + tt)
        t2 = N * z * 0.75
        jp = int(t1 - t2)
        jm = int(t1 + t2)
        ir = N + 1 + jp - jm
        kshift = 1 - (ir & 1)
        ip = (jp + jm - N + kshift + 1) // 2
        ip %= 4 * N
        return 2 * N * (N - 1) + (ir - 1) * 4 * N + ip
    tp = tt - int(tt)
    tmp = N * math.sqrt(3.0 * (1.0 - za))
    jp = int(tp * tmp)
    jm = int((1.0 - tp) * tmp)
    ir = jp + jm + 1
    ip = int(tt * ir) % (4 * ir)
    if z > 0:
        return 2 * ir * (ir - 1) + ip
    return 12 * N * N - 2 * ir * (ir + 1) + ip


@pytest.mark.parametrize("nside", [1, 2, 4, 8, 16])
def test_geometry_roundtrip_against_independent_ang2pix(nside):
    total = 0
    for r in range(1, 4 * nside):
        ct, st, n, sg, first = O.ring_info(nside, r)
        assert abs(ct * ct + st * st - 1) < 1e-14
        assert first == total
        total += n
        for j in range(n):
            phi = math.pi * (2 * j + sg) / n
            assert ang2pix_ring(nside, ct, phi) == first + j
    assert total == 12 * nside * nside


def test_geometry_matches_generator_positions():
    z, phi = S.pixel_positions(8)
    th, ph = O.pixel_angles(8)
    assert np.allclose(np.cos(th), z, atol=1e-15, rtol=0)
    assert np.allclose(ph, phi, atol=1e-14, rtol=0)


# ---------------------------------------------------------------------------
# spin-weighted harmonics
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("s", [2, -2, 0])
def test_lambda_matches_goldberg_formula(s):
    for l in range(0, 8):
        for m in range(-l, l + 1):
            for th in (0.05, 0.7, 1.9, 3.0):
                lam = O.spin_lambda(s, 9, m, th)[l]
                ref = O.goldberg_sYlm(s, l, m, th, 0.0)
                assert abs(ref.imag) < 1e-15
                assert abs(lam - ref.real) < 1e-13, (s, l, m, th, lam, ref)


def test_spin0_matches_scipy_sph_harm():
    sp = pytest.importorskip("scipy.special")
    for th in (0.01, 0.9, 2.2):
        for m in range(0, 25, 3):
            lam = O.spin_lambda(0, 40, m, th)
            for l in range(m, 41):
                ref = sp.sph_harm_y(l, m, th, 0.0)
                assert abs(lam[l] - ref.real) < 1e-12 * max(1.0, abs(ref))


# Goldberg et al. (1967) closed forms of 2Y_lm for l = 2, 3 (e^{imφ} removed), t = θ/2
CLOSED = {
    (2, 2): lambda th, t: 0.5 * math.sqrt(5 / math.pi) * math.sin(t) ** 4,
    (2, 1): lambda th, t: -math.sqrt(5 / math.pi) * math.sin(t) ** 3 * math.cos(t),
    (2, 0): lambda th, t: math.sqrt(30 / math.pi) / 8 * math.sin(th) ** 2,
    (2, -1): lambda th, t: -math.sqrt(5 / math.pi) * math.sin(t) * math.cos(t) ** 3,
    (2, -2): lambda th, t: 0.5 * math.sqrt(5 / math.pi) * math.cos(t) ** 4,
    (3, 3): lambda th, t: -0.5 * math.sqrt(42 / math.pi) * math.sin(t) ** 5 * math.cos(t),
    (3, 2): lambda th, t: 0.5 * math.sqrt(7 / math.pi) * (3 * math.cos(th) + 2) * math.sin(t) ** 4,
    (3, 0): lambda th, t: math.sqrt(210 / math.pi) / 8 * math.cos(th) * math.sin(th) ** 2,
    (3, -3): lambda th, t: 0.5 * math.sqrt(42 / math.pi) * math.sin(t) * math.cos(t) ** 5,
}


def test_spin2_closed_forms_l2_l3():
    for (l, m), f in CLOSED.items():
        for th in (0.2, 1.0, 1.6, 2.7):
            assert abs(O.spin_lambda(2, 4, m, th)[l] - f(th, th / 2)) < 1e-14


def test_parity_relation():
    """sλ_lm(π-θ) = (-1)^{l+m} (-s)λ_lm(θ)."""
    L = 60
    for m in (0, 1, 2, 7, 33):
        for th in (0.3, 1.2):
            a = O.spin_lambda(2, L, m, math.pi - th)
            b = O.spin_lambda(-2, L, m, th)
            sg = np.array([(-1) ** (l + m) for l in range(L + 1)])
            assert np.max(np.abs(a - sg * b)) < 1e-12


@pytest.mark.parametrize("s", [2, -2, 0])
def test_addition_theorem_sum_over_m(s):
    """Spin-weighted addition theorem at coincident points: Σ_{m=-l..l} |sY_lm(θ)|² = (2l+1)/4π
    for l >= |s| and every θ, which fixes the normalisation of all m at once, at any latitude
    (including rings next to a pole)."""
    L = 1000
    ref = (2 * np.arange(L + 1) + 1) / (4 * math.pi)
    for th in (0.004, 0.4, 1.3, math.pi / 2, 2.9):
        acc = np.zeros(L + 1)
        for m in range(-L, L + 1):
            acc += O.spin_lambda(s, L, m, th) ** 2
        l0 = abs(s)
        assert np.max(np.abs(acc[l0:] - ref[l0:]) / ref[l0:]) < 1e-10, (s, th)
        assert np.all(acc[:l0] == 0)


@pytest.mark.parametrize("s", [2, -2])
def test_orthonormality_at_high_l(s):
    """∫ sλ_lm sλ_l'm 2π d(cosθ) = δ_ll' (exact with Gauss-Legendre: the product is a
    polynomial in cosθ of degree l + l'), up to l = 1500, including the rescaled
    recurrence through deep underflow at large m."""
    L = 1500
    x, wq = np.polynomial.legendre.leggauss(L + 8)
    th = np.arccos(x)
    for m in (0, 1, 2, 3, 400, 1100, 1490):
        lam = np.array([O.spin_lambda(s, L, m, t) for t in th])  # [node, l]
        G = 2 * np.pi * (lam * wq[:, None]).T @ lam
        l0 = max(m, 2)
        G = G[l0:, l0:]
        # Gauss-Legendre nodes and weights at n ~ 1500 are themselves good to ~1e-11
        assert np.max(np.abs(G - np.eye(len(G)))) < 1e-10, m


# ---------------------------------------------------------------------------
# KS kernel (Eq. 3)
# ---------------------------------------------------------------------------
def test_ks_kernel_values():
    D = O.ks_kernel(5)
    assert D[0] == 0 and D[1] == 0
    assert abs(D[2] + math.sqrt(2 / 3)) < 1e-15
    assert abs(D[3] + math.sqrt(5 / 6)) < 1e-15
    assert abs(D[4] + math.sqrt(3 * 6 / 20)) < 1e-15


# ---------------------------------------------------------------------------
# synthesis and adjoint
# ---------------------------------------------------------------------------
def _rand_pair(lmax, rng):
    return S.random_alm(lmax, rng), S.random_alm(lmax, rng)


def test_ring_phase_sum_brute_force():
    rng = np.random.default_rng(5)
    L = 13
    for n, sg in ((4, 1), (12, 1), (16, 0), (16, 1), (40, 1)):
        F = rng.normal(size=2 * L + 1) + 1j * rng.normal(size=2 * L + 1)
        f = O.ring_phase_sum(F, L, n, sg)
        m = np.arange(-L, L + 1)
        for j in range(n):
            phij = np.pi * (2 * j + sg) / n
            assert abs(f[j] - np.sum(F * np.exp(1j * m * phij))) < 1e-12
        w = rng.normal(size=n) + 1j * rng.normal(size=n)
        G = O.ring_phase_adjoint(w, L, sg)
        phis = np.pi * (2 * np.arange(n) + sg) / n
        for k, mm in enumerate(m):
            assert abs(G[k] - np.sum(w * np.exp(-1j * mm * phis))) < 1e-12


@pytest.mark.parametrize("nside,lmax", [(2, 5), (4, 8)])
def test_ring_synthesis_equals_direct_goldberg_sum(nside, lmax):
    rng = np.random.default_rng(nside)
    aE, aB = _rand_pair(lmax, rng)
    g1, g2 = O.synth_spin2(nside, lmax, aE, aB)
    d1, d2 = O.direct_synth_spin2(nside, lmax, aE, aB)
    assert np.max(np.abs(g1 - d1)) + np.max(np.abs(g2 - d2)) < 1e-12


def test_eb_convention_single_modes():
    """Eq. 2: a pure a_E mode gives γ_{2} = -a_E, so γ = -a_E 2Y_lm (+ its m<0 mirror)."""
    N, L = 4, 3
    nt = O.ntri(L)
    th, ph = O.pixel_angles(N)
    aE = np.zeros(nt, complex)
    aB = np.zeros(nt, complex)
    aE[O.tri_index(L, 2, 0)] = 1.0
    g1, g2 = O.synth_spin2(N, L, aE, aB)
    Y = np.array([O.goldberg_sYlm(2, 2, 0, t, p) for t, p in zip(th, ph)])
    assert np.max(np.abs((g1 + 1j * g2) - (-Y))) < 1e-13
    aE[:] = 0
    aB[O.tri_index(L, 3, 0)] = 1.0
    g1, g2 = O.synth_spin2(N, L, aE, aB)
    Y = np.array([O.goldberg_sYlm(2, 3, 0, t, p) for t, p in zip(th, ph)])
    assert np.max(np.abs((g1 + 1j * g2) - (-1j * Y))) < 1e-13


def _single_mode_error(forward, N=4, L=4):
    """Largest deviation of forward(κ) from the Eq. 3 / Eq. 2 shear of single κ modes.

    Eq. 3 gives γ_{±2,lm} = D_l κ_lm with κ = κ_E + i κ_B, and the real field has
    κ_{l,-m} = (-1)^m conj(κ_lm), so a single stored mode c at (l, m > 0) must give
    γ1 + iγ2 = D_l f [c 2Y_lm + (-1)^m conj(c) 2Y_{l,-m}] with f = 1 for E and f = i for B
    (at m = 0 only the first term, c real).  2Y from the Goldberg formula (mpmath)."""
    nt = O.ntri(L)
    th, ph = O.pixel_angles(N)
    D = O.ks_kernel(L)
    worst = 0.0
    for l, m in ((2, 0), (2, 1), (3, 2), (4, 3), (4, 4)):
        Yp = np.array([O.goldberg_sYlm(2, l, m, t, p) for t, p in zip(th, ph)])
        Ym = np.array([O.goldberg_sYlm(2, l, -m, t, p) for t, p in zip(th, ph)])
        c = 0.7 - 0.3j if m > 0 else 0.7 + 0j
        for field, f in ((0, 1.0), (1, 1j)):
            kE = np.zeros(nt, complex)
            kB = np.zeros(nt, complex)
            (kE if field == 0 else kB)[O.tri_index(L, l, m)] = c
            g1, g2 = forward(N, L, kE, kB)
            expect = D[l] * f * (c * Yp + ((-1) ** m * np.conj(c) * Ym if m > 0 else 0))
            worst = max(worst, float(np.max(np.abs(g1 + 1j * g2 - expect))))
    return worst


def test_forward_A_single_modes_follow_eq3_sign():
    """Pins the KS sign of forward_A (and so adjoint_A, its transpose): single κ_E and κ_B
    modes produce D_l κ_lm 2Y_lm + mirror, not its negative (the Eq. 3 reading)."""
    assert _single_mode_error(O.forward_A) < 1e-13


def test_planted_forward_A_sign_flip_is_caught_by_single_modes():
    flipped = lambda N, L, kE, kB: tuple(-g for g in O.forward_A(N, L, kE, kB))
    assert _single_mode_error(flipped) > 0.1


def _uniform_sky_precond_error(precond_fn, N=16, L=16):
    """max |P_i diag(H_λ)_i - 1| over the real-dof basis on a uniform full sky (M ≡ 1, N^-1 =
    100, λ = 1e-3).  There H_λ is diagonal up to HEALPix quadrature error (App. A), with
    <N^-1> D_l^2 + λ_eff on the l >= 2 modes and exactly λ_eff on l < 2, which A does not see;
    the per-l preconditioner is defined as the inverse of that diagonal."""
    w = O.Weights(N, np.full(12 * N * N, 100.0), lam=1e-3)
    H, vecs = O.dense_H(N, L, w)
    P = precond_fn(L, w)
    idx = np.array([(e if e.any() else b).nonzero()[0][0] for e, b in vecs])
    return float(np.max(np.abs(P[idx] * np.diag(H) - 1.0)))


def test_per_l_preconditioner_inverts_the_uniform_sky_diagonal_of_dense_H():
    assert _uniform_sky_precond_error(O.per_l_preconditioner) < 1e-2


def test_planted_per_l_preconditioner_with_abs_D_is_caught():
    def bad(L, w):
        ls, _ = O.lm_arrays(L)
        d = w.mean_mninv * np.abs(O.ks_kernel(L))[ls] + w.lam_eff
        return 1.0 / d

    assert _uniform_sky_precond_error(bad) > 0.1


@pytest.mark.parametrize("nside,lmax", [(8, 20), (16, 40), (8, 31)])
def test_adjoint_identity(nside, lmax):
    rng = np.random.default_rng(lmax)
    aE, aB = _rand_pair(lmax, rng)
    u1 = rng.normal(size=12 * nside ** 2)
    u2 = rng.normal(size=12 * nside ** 2)
    g1, g2 = O.synth_spin2(nside, lmax, aE, aB)
    bE, bB = O.adjoint_synth_spin2(nside, lmax, u1, u2)
    lhs = g1 @ u1 + g2 @ u2
    rhs = O.realdof_dot(lmax, aE, bE) + O.realdof_dot(lmax, aB, bB)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    # adjoint outputs at m = 0 are real and below l = 2 vanish
    ls, ms = O.lm_arrays(lmax)
    assert np.all(bE[ms == 0].imag == 0) and np.all(bB[ms == 0].imag == 0)
    assert np.all(bE[ls < 2] == 0) and np.all(bB[ls < 2] == 0)


# ---------------------------------------------------------------------------
# H, CG, dense solve
# ---------------------------------------------------------------------------
def _small_problem(nside=8, lmax=10, seed=3, lam=1e-3, cap=0.6):
    rng = np.random.default_rng(seed)
    th, _ = O.pixel_angles(nside)
    npix = 12 * nside ** 2
    mask = th > cap
    ninv = np.where(mask, rng.poisson(20, npix) / 0.26 ** 2, 0.0)
    return O.Weights(nside, ninv, lam), rng


def test_H_symmetric_positive():
    w, rng = _small_problem()
    H, _ = O.dense_H(8, 10, w)
    assert np.max(np.abs(H - H.T)) < 1e-13 * np.max(np.abs(H))
    ev = np.linalg.eigvalsh(H)
    assert ev.min() > 0.999 * w.lam_eff  # H = A^T W A + λ_eff I >= λ_eff


def test_cg_equals_dense_cholesky():
    N, L = 8, 10
    w, rng = _small_problem(N, L)
    xE = S.random_alm(L, rng, lmin=2)
    xB = S.random_alm(L, rng, lmin=2)
    y1, y2 = O.forward_A(N, L, xE, xB)
    y1 = y1 + 0.01 * rng.normal(size=y1.shape)
    y2 = y2 + 0.01 * rng.normal(size=y2.shape)
    b = O.rhs_b(N, L, w, y1, y2)
    (cE, cB), _ = O.cholesky_solve(N, L, w, b)
    (gE, gB), it, rr, _ = O.pcg(lambda e, bb: O.apply_H(N, L, w, e, bb), b, w.precond, L, 1e-13, 500)
    scale = max(np.abs(cE).max(), np.abs(cB).max())
    assert np.max(np.abs(gE - cE)) < 1e-10 * scale
    assert np.max(np.abs(gB - cB)) < 1e-10 * scale


def test_per_l_preconditioned_cg_equals_dense_cholesky():
    """A diagonal preconditioner changes the iterates, not the solution: PCG with the per-l
    weights (mean_all(M N^-1) D_l^2 + λ_eff)^-1 reaches the dense Cholesky solution."""
    N, L = 8, 10
    w, rng = _small_problem(N, L)
    y1, y2 = O.forward_A(N, L, S.random_alm(L, rng, lmin=2), S.random_alm(L, rng, lmin=2))
    y1 = y1 + 0.01 * rng.normal(size=y1.shape)
    b = O.rhs_b(N, L, w, y1, y2)
    (cE, cB), _ = O.cholesky_solve(N, L, w, b)
    P = O.per_l_preconditioner(L, w)
    ls, _ = O.lm_arrays(L)
    assert np.allclose(P[ls < 2], 1.0 / w.lam_eff)
    assert np.allclose(P[ls == 2], 1.0 / (w.mean_mninv * 2.0 / 3.0 + w.lam_eff))
    (gE, gB), it, rr, _ = O.pcg(lambda e, bb: O.apply_H(N, L, w, e, bb), b, P, L, 1e-13, 500)
    scale = max(np.abs(cE).max(), np.abs(cB).max())
    assert np.max(np.abs(gE - cE)) < 1e-10 * scale and np.max(np.abs(gB - cB)) < 1e-10 * scale


def test_noise_free_pure_E_recovers_input_and_zero_B():
    """y = A x_true with κ_B = 0, λ = 0 and a full-rank footprint: x̂ = x_true, κ̂_B = 0."""
    N, L = 16, 12
    w, rng = _small_problem(N, L, lam=0.0, cap=0.3)
    xE = S.random_alm(L, rng, lmin=2)
    xB = np.zeros_like(xE)
    y1, y2 = O.forward_A(N, L, xE, xB)
    (gE, gB), it, rr, _ = O.cg_solve(N, L, w, y1, y2, tol=1e-13, maxiter=2000)
    assert np.max(np.abs(gE - xE)) < 1e-10 * np.abs(xE).max()
    assert np.max(np.abs(gB)) < 1e-10 * np.abs(xE).max()


def test_e_only_solve_equals_dense_EE_block():
    """App. A: the E-mode solve is the E block of the dense normal matrix, solved directly."""
    N, L = 8, 10
    w, rng = _small_problem(N, L)
    y1, y2 = O.forward_A(N, L, S.random_alm(L, rng, lmin=2), S.random_alm(L, rng, lmin=2))
    y1 = y1 + 0.01 * rng.normal(size=y1.shape)
    b = O.rhs_b(N, L, w, y1, y2)
    H, vecs = O.dense_H(N, L, w)
    n = H.shape[0] // 2                       # basis: the E field first, then B
    rhs = np.array([O.pair_dot(L, v, (b[0], np.zeros_like(b[0]))) for v in vecs[:n]])
    c = np.linalg.solve(np.linalg.cholesky(H[:n, :n]).T,
                        np.linalg.solve(np.linalg.cholesky(H[:n, :n]), rhs))
    xE = sum(ci * v[0] for ci, v in zip(c, vecs[:n]))
    (gE, gB), it, rr, _ = O.cg_solve_E(N, L, w, y1, y2, tol=1e-13, maxiter=500)
    assert np.max(np.abs(gE - xE)) < 1e-10 * np.abs(xE).max()
    assert not np.any(gB)
    # and it differs from the joint solve's E part (the mask couples E and B)
    (jE, _), _, _, _ = O.cg_solve(N, L, w, y1, y2, tol=1e-13, maxiter=500)
    assert np.max(np.abs(gE - jE)) > 1e-6 * np.abs(jE).max()


def test_conditional_B_given_joint_E_reproduces_joint_B():
    """Eq. A7 is the lower block row of the joint system, so with κ̂_E of the joint solve the
    reduced B equation (Eq. A8) returns the joint κ̂_B."""
    N, L = 8, 12
    w, rng = _small_problem(N, L)
    y1, y2 = O.forward_A(N, L, S.random_alm(L, rng, lmin=2), S.random_alm(L, rng, lmin=2))
    y1 = y1 + 0.01 * rng.normal(size=y1.shape)
    y2 = y2 + 0.01 * rng.normal(size=y2.shape)
    (jE, jB), _, _, _ = O.cg_solve(N, L, w, y1, y2, tol=1e-13, maxiter=1000)
    (zE, cB), it, rr, _ = O.cg_solve_B_given_E(N, L, w, y1, y2, jE, tol=1e-13, maxiter=1000)
    assert not np.any(zE)
    assert np.max(np.abs(cB - jB)) < 1e-9 * np.abs(jB).max()


def test_e_only_then_conditional_B_on_noise_free_pure_E():
    """y = A (x_E, 0), λ = 0, full-rank footprint: the E solve returns x_E and the conditional
    B solve returns zero B (the E-to-B leakage term cancels b_B exactly)."""
    N, L = 16, 12
    w, rng = _small_problem(N, L, lam=0.0, cap=0.3)
    xE = S.random_alm(L, rng, lmin=2)
    y1, y2 = O.forward_A(N, L, xE, np.zeros_like(xE))
    (gE, _), _, _, _ = O.cg_solve_E(N, L, w, y1, y2, tol=1e-13, maxiter=2000)
    assert np.max(np.abs(gE - xE)) < 1e-10 * np.abs(xE).max()
    _, bB = O.rhs_b(N, L, w, y1, y2)
    assert np.abs(bB).max() > 1e-3 * np.abs(O.rhs_b(N, L, w, y1, y2)[0]).max()   # b_B is not 0
    (_, gB), _, rr, _ = O.cg_solve_B_given_E(N, L, w, y1, y2, gE, tol=1e-13, maxiter=2000)
    assert np.max(np.abs(gB)) < 1e-9 * np.abs(xE).max()


def test_cl_spectra_parseval_single_mode_and_symmetry():
    """Σ_l (2l+1) C_l^EE = <a_E, a_E> (real-dof metric); a single (l, m>0) mode gives
    C_l = 2|c|^2/(2l+1); C^EB(a, b) = C^BE(b, a); the binned EE auto spectrum equals the
    band-power loss of the differentiation workload."""
    L = 40
    rng = np.random.default_rng(4)
    a = (S.random_alm(L, rng), S.random_alm(L, rng))
    b = (S.random_alm(L, rng), S.random_alm(L, rng))
    cl = O.cl_spectra(L, a, a)
    ell = np.arange(L + 1)
    assert abs(np.sum((2 * ell + 1) * cl[0]) - O.realdof_dot(L, a[0], a[0])) < 1e-10 * np.sum((2 * ell + 1) * cl[0])
    one = np.zeros(O.ntri(L), np.complex128)
    one[O.tri_index(L, 5, 3)] = 0.3 - 0.4j
    c1 = O.cl_spectra(L, (one, one * 0), (one, one * 0))
    assert abs(c1[0, 5] - 2 * 0.25 / 11) < 1e-15 and np.count_nonzero(c1) == 1
    ab, ba = O.cl_spectra(L, a, b), O.cl_spectra(L, b, a)
    assert np.allclose(ab[1], ba[2], rtol=0, atol=1e-14) and np.allclose(ab[0], ba[0], rtol=0, atol=1e-14)
    edges = np.geomspace(3, 40, 5)
    assert abs(O.band_powers(cl[0], edges).sum() - O.band_power_loss(L, a[0], edges)) < 1e-12


def test_cl_of_gaussian_field_matches_its_power_spectrum():
    """A Gaussian realisation's C_l averaged over 100 < l <= 300 matches the input C_l within
    a few times the cosmic-variance error sqrt(2/Σ(2l+1)) (about 0.4 %)."""
    L = 300
    rng = np.random.default_rng(11)
    cl_in = S.cl_kappa(L)
    aE = S.grf_alm(L, cl_in, rng)
    cl = O.cl_spectra(L, (aE, 0 * aE), (aE, 0 * aE))[0]
    sel = np.arange(101, L + 1)
    ratio = np.sum((2 * sel + 1) * cl[sel]) / np.sum((2 * sel + 1) * cl_in[sel])
    assert abs(ratio - 1) < 4 * np.sqrt(2.0 / np.sum(2 * sel + 1))


def test_shuffle_permutes_only_unmasked_values():
    from paper_2606_06175_gb300 import spectra as SP
    N = 8
    rng = np.random.default_rng(2)
    mask = rng.random(12 * N * N) < 0.4
    y = np.where(mask, rng.normal(size=(2, 12 * N * N)), 0.0)
    perms = SP.shuffle_permutations(mask, 3, seed=9)
    for r in range(3):
        z = O.shuffle_shear(y, perms[r])
        assert not np.any(z[:, ~mask])
        assert np.array_equal(np.sort(z[0][mask]), np.sort(y[0][mask]))
        assert np.array_equal(perms[r][~mask], np.nonzero(~mask)[0])
        # both components move together (a galaxy's shear stays a pair)
        assert np.array_equal(z[1], y[1][perms[r]])
    assert not np.array_equal(perms[0], perms[1])


def test_flat_single_mode_closed_form_and_adjoint_identity():
    """Flat sky: one Fourier mode (k1, k2) gives γ1 + iγ2 = D(k) e^{2πi(k1 x + k2 y)/n}/n at
    every pixel, D = e^{2iφ_k}; <A x, u> = <x, A^T u> to 1e-12."""
    n = 16
    for k1, k2 in [(3, 0), (2, 5), (n - 4, 7), (n // 2, 1)]:
        x = np.zeros((n, n), np.complex128)
        x[k2, k1] = 0.7 - 0.2j
        g1, g2 = O.flat_forward_A(n, x)
        f1 = k1 if k1 < n // 2 else k1 - n
        f2 = k2 if k2 < n // 2 else k2 - n
        D = (f1 * f1 - f2 * f2 + 2j * f1 * f2) / (f1 * f1 + f2 * f2)
        assert abs(abs(D) - 1) < 1e-15
        yy, xx = np.mgrid[0:n, 0:n]
        ref = (0.7 - 0.2j) * D * np.exp(2j * np.pi * (k1 * xx + k2 * yy) / n) / n
        assert np.max(np.abs(g1 + 1j * g2 - ref)) < 1e-14
    rng = np.random.default_rng(1)
    x = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    u1, u2 = rng.normal(size=(n, n)), rng.normal(size=(n, n))
    g1, g2 = O.flat_forward_A(n, x)
    lhs = np.sum(g1 * u1 + g2 * u2)
    rhs = O.flat_dot(x, O.flat_adjoint_A(n, u1, u2))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_flat_uniform_weights_H_is_diagonal_and_pure_E_recovered():
    """Uniform full coverage: H x = w |D|² x + λ_eff x (= (w + λ_eff) x off k = 0).  Random
    positive weights, λ = 0, noise-free y = A x_true with no k = 0 part: CG returns x_true."""
    n = 16
    rng = np.random.default_rng(2)
    x = rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n))
    w = O.FlatWeights(np.full((n, n), 3.0), lam=1e-3)
    hx = O.flat_apply_H(n, w, x)
    expect = (3.0 + w.lam_eff) * x
    expect[0, 0] = w.lam_eff * x[0, 0]
    assert np.max(np.abs(hx - expect)) < 1e-12 * np.abs(x).max()
    kE = rng.normal(size=(n, n))
    xt = np.fft.fft2(kE, norm="ortho")
    xt[0, 0] = 0
    w2 = O.FlatWeights(1.0 + rng.random((n, n)), lam=0.0)
    y1, y2 = O.flat_forward_A(n, xt)
    xs, it, rr = O.flat_cg_solve(n, w2, y1, y2, tol=1e-13, maxiter=500)
    assert np.max(np.abs(xs - xt)) < 1e-10 * np.abs(xt).max()
    # the recovered field is pure E: κ_B = Im F^-1 x = 0
    assert np.max(np.abs(np.fft.ifft2(xs, norm="ortho").imag)) < 1e-10 * np.abs(kE).max()


def test_flat_cg_equals_dense_solve():
    """n = 8 with a mask: CG equals the dense H solved directly (H built column by column on
    the real and imaginary unit vectors)."""
    n = 8
    rng = np.random.default_rng(3)
    ninv = np.where(rng.random((n, n)) < 0.6, 1.0 + rng.random((n, n)), 0.0)
    w = O.FlatWeights(ninv, lam=1e-2)
    y1 = np.where(ninv > 0, rng.normal(size=(n, n)), 0.0)
    y2 = np.where(ninv > 0, rng.normal(size=(n, n)), 0.0)
    basis = []
    for k in range(n * n):
        for v in (1.0, 1j):
            e = np.zeros(n * n, np.complex128)
            e[k] = v
            basis.append(e.reshape(n, n))
    H = np.array([[O.flat_dot(bi, O.flat_apply_H(n, w, bj)) for bj in basis] for bi in basis])
    assert np.max(np.abs(H - H.T)) < 1e-12 * np.abs(H).max()
    b = O.flat_rhs_b(n, w, y1, y2)
    c = np.linalg.solve(H, np.array([O.flat_dot(bi, b) for bi in basis]))
    xd = sum(ci * bi for ci, bi in zip(c, basis))
    xs, it, rr = O.flat_cg_solve(n, w, y1, y2, tol=1e-13, maxiter=500)
    assert np.max(np.abs(xs - xd)) < 1e-10 * np.abs(xd).max()


def test_full_sky_uniform_weight_is_nearly_diagonal():
    """M ≡ 1, uniform N^-1: H_EB ≈ 0 and H ≈ <N^-1> D_l^2 (App. A), within HEALPix quadrature."""
    N, L = 16, 16
    w = O.Weights(N, np.full(12 * N * N, 100.0), lam=0.0)
    H, vecs = O.dense_H(N, L, w)
    n = H.shape[0] // 2
    assert np.abs(H[:n, n:]).max() < 1e-2 * np.abs(H[:n, :n]).max()
    D = O.ks_kernel(L)
    ls, _ = O.lm_arrays(L)
    expect = np.array([100.0 * D[ls[ix]] ** 2 for ix, _ in O.realdof_basis(L)])
    assert np.max(np.abs(np.diag(H)[:n] - expect)) < 2e-2 * 100.0


def test_cg_iterations_within_eq13_bound():
    N, L = 8, 12
    w, rng = _small_problem(N, L)
    xE = S.random_alm(L, rng, lmin=2)
    y1, y2 = O.forward_A(N, L, xE, np.zeros_like(xE))
    eps = 1e-8
    _, it, rr, hist = O.cg_solve(N, L, w, y1, y2, tol=eps, maxiter=2000)
    kappa = O.lanczos_condition(hist)
    bound = 0.5 * math.sqrt(kappa) * math.log(2 / eps)
    assert rr < eps
    assert it <= math.ceil(bound) + 1, (it, bound, kappa)


def test_preconditioner_is_scalar_so_iterates_match_plain_cg():
    """Eq. 15's P is a multiple of I, which leaves the CG iterates unchanged."""
    N, L = 8, 10
    w, rng = _small_problem(N, L)
    xE = S.random_alm(L, rng, lmin=2)
    y1, y2 = O.forward_A(N, L, xE, np.zeros_like(xE))
    b = O.rhs_b(N, L, w, y1, y2)
    ap = lambda e, bb: O.apply_H(N, L, w, e, bb)
    x1, it1, _, _ = O.pcg(ap, b, w.precond, L, 1e-9, 300)
    x2, it2, _, _ = O.pcg(ap, b, 1.0, L, 1e-9, 300)
    assert it1 == it2
    assert np.max(np.abs(x1[0] - x2[0])) < 1e-9 * np.abs(x1[0]).max()


# ---------------------------------------------------------------------------
# inputs
# ---------------------------------------------------------------------------
def test_synthetic_footprints():
    sv = S.survey(64, "cap", 1001)
    z, phi = S.pixel_positions(64)
    fp = S.cap_footprint(z, phi)
    assert abs(fp.mean() - (1 - math.cos(math.radians(30))) / 2) < 3e-3
    sv = S.survey(128, "des", 1002)
    area = sv["mask"].mean() * 4 * math.pi * (180 / math.pi) ** 2
    assert abs(area - 4143) < 100
    assert np.all(sv["ninv"][~sv["mask"]] == 0)


# ---------------------------------------------------------------------------
# planted mistakes: each must be caught by one of the pins above
# ---------------------------------------------------------------------------
def test_planted_dropped_half_in_adjoint_is_caught():
    N, L = 4, 8
    rng = np.random.default_rng(0)
    aE, aB = _rand_pair(L, rng)
    u1, u2 = rng.normal(size=12 * N * N), rng.normal(size=12 * N * N)
    g1, g2 = O.synth_spin2(N, L, aE, aB)
    bE, bB = O.adjoint_synth_spin2(N, L, u1, u2)
    lhs = g1 @ u1 + g2 @ u2
    bad = O.realdof_dot(L, aE, 2 * bE) + O.realdof_dot(L, aB, 2 * bB)  # forgot the 1/2
    assert abs(lhs - bad) > 1e-3 * abs(lhs)


def test_planted_wrong_B_sign_is_caught_by_direct_sum():
    N, L = 2, 4
    rng = np.random.default_rng(1)
    aE, aB = _rand_pair(L, rng)
    g1, g2 = O.synth_spin2(N, L, aE, -aB)  # a_B with the wrong sign
    d1, d2 = O.direct_synth_spin2(N, L, aE, aB)
    assert np.max(np.abs(g1 - d1)) + np.max(np.abs(g2 - d2)) > 1e-3


def test_planted_transposed_index_is_caught():
    L = 6
    rng = np.random.default_rng(2)
    aE, aB = _rand_pair(L, rng)
    perm = np.array([O.tri_index(L, l, m) for m in range(L + 1) for l in range(m, L + 1)])
    # an l-major packing instead of m-major
    bad_idx = []
    for m in range(L + 1):
        for l in range(m, L + 1):
            bad_idx.append(l * (l + 1) // 2 + m)
    bad = np.empty_like(aE)
    bad[perm] = aE[np.array(bad_idx)]
    g1, g2 = O.synth_spin2(2, L, bad, aB)
    d1, d2 = O.direct_synth_spin2(2, L, aE, aB)
    assert np.max(np.abs(g1 - d1)) > 1e-3


def test_planted_ks_sign_flip_is_caught():
    D = -O.ks_kernel(3)
    assert abs(D[2] + math.sqrt(2 / 3)) > 1
