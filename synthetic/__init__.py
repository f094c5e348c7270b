"""Seeded synthetic inputs standing in for the DES Y3 catalogue (not in this repository).

This module draws random numbers and places footprints on the HEALPix grid; it
holds none of the operator arithmetic (no harmonic transforms, no KS kernel, no
solver), so both the CPU oracle and the CUDA path take their inputs from it.

Recipe (the catalogue itself is replaced; its summary properties are kept):
  * κ_E alm: Gaussian random field with C_l = A (l+10)^-2, A = 1e-4, C_0 = C_1 = 0;
    κ_l0 ~ sqrt(C_l) N(0,1), κ_lm ~ sqrt(C_l/2)(N + iN) for m > 0; κ_B = 0.
  * cap footprint: spherical cap of radius 30 deg centred at (dec -50, RA 30),
    counts ~ Poisson(20) per pixel.
  * DES-like footprint (4143 deg^2, Sec. III A): band dec in [-60, -40] deg with
    RA in [0, 295.1) deg plus a strip RA in [0, 10], dec in [-40, 0]; every edge
    is displaced by 1 deg x s(u), s a seeded sum of 8 random-phase sinusoids
    normalised to |s| <= 1.  Mean counts 5.6 arcmin^-2 x pixel area x (1 + 0.3 t),
    t a seeded smooth pattern (random cubic in the unit vector) scaled to
    max |t| = 1 on the footprint.
  * inverse noise N^-1_p = n_p / σ_e^2 (Eqs. 17-18 with unit weights), σ_e = 0.26;
    the mask is n_p >= 1 inside the footprint (Eq. 19 with N_th = 1); shape noise
    n_p ~ N(0, σ_e^2 / n_p) per shear component.
Seeds: one numpy SeedSequence per workload, spawned into independent streams
for alm / footprint / depth / counts / noise.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA_E = 0.26
ARCMIN2_PER_SR = (180.0 * 60.0 / math.pi) ** 2

# workload seeds: cap (Nside 32), DES-like 512, DES-like 2048, batched, differentiation
SEEDS = {"cap32": 1001, "des512": 1002, "des2048": 1003, "batch": 1004, "grad512": 1005, "flat": 1006}


def ntri(lmax: int) -> int:
    return (lmax + 1) * (lmax + 2) // 2


def streams(seed: int, n: int = 5):
    """Independent generators: alm, footprint, depth, counts, noise."""
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


def pixel_positions(nside: int):
    """(z = cos θ, φ) of the HEALPix RING pixel centres.

    Polar rings i < N: z = 1 - i^2/(3N^2), 4i pixels at φ = π(j + 1/2)/(2i);
    equatorial rings N <= i <= 2N: z = 4/3 - 2i/(3N), 4N pixels at
    φ = π(j + s/2)/(2N), s = (i - N + 1) mod 2; the south half mirrors the north.
    """
    N = nside
    npix = 12 * N * N
    z = np.empty(npix)
    phi = np.empty(npix)
    pos = 0
    for ring in range(1, 4 * N):
        i = ring if ring <= 2 * N else 4 * N - ring
        if i < N:
            zz = 1.0 - i * i / (3.0 * N * N)
            n = 4 * i
            ph = math.pi * (np.arange(n) + 0.5) / (2 * i)
        else:
            zz = 4.0 / 3.0 - 2.0 * i / (3.0 * N)
            n = 4 * N
            s = (i - N + 1) % 2
            ph = math.pi * (np.arange(n) + 0.5 * s) / (2 * N)
        z[pos:pos + n] = zz if ring <= 2 * N else -zz
        phi[pos:pos + n] = ph
        pos += n
    assert pos == npix
    return z, phi


def cl_kappa(lmax: int, amp: float = 1e-4) -> np.ndarray:
    l = np.arange(lmax + 1, dtype=np.float64)
    cl = amp * (l + 10.0) ** -2
    cl[:2] = 0.0
    return cl


def grf_alm(lmax: int, cl: np.ndarray, rng) -> np.ndarray:
    """Packed (m-major) complex alm of a real Gaussian field with spectrum cl."""
    out = np.empty(ntri(lmax), np.complex128)
    pos = 0
    for m in range(lmax + 1):
        n = lmax + 1 - m
        c = cl[m:]
        if m == 0:
            out[pos:pos + n] = np.sqrt(c) * rng.standard_normal(n)
        else:
            out[pos:pos + n] = np.sqrt(c / 2) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        pos += n
    return out


def random_alm(lmax: int, rng, lmin: int = 0) -> np.ndarray:
    """Unit-variance random packed alm (real field: m = 0 imaginary parts zero)."""
    out = np.empty(ntri(lmax), np.complex128)
    pos = 0
    for m in range(lmax + 1):
        n = lmax + 1 - m
        l = np.arange(m, lmax + 1)
        v = rng.standard_normal(n) + (0 if m == 0 else 1j * rng.standard_normal(n))
        out[pos:pos + n] = np.where(l >= lmin, v, 0)
        pos += n
    return out


def _edge_wiggle(rng, n_terms: int = 8):
    amp = rng.uniform(0.5, 1.0, n_terms)
    freq = rng.integers(1, 12, n_terms)
    phase = rng.uniform(0, 2 * np.pi, n_terms)
    norm = amp.sum()

    def s(u_deg):
        u = np.radians(np.atleast_1d(np.asarray(u_deg, np.float64)))
        return (amp[:, None] * np.sin(freq[:, None] * u[None, :] + phase[:, None])).sum(0) / norm

    return s


def cap_footprint(z, phi, radius_deg=30.0, dec0_deg=-50.0, ra0_deg=30.0):
    dec0, ra0 = math.radians(dec0_deg), math.radians(ra0_deg)
    c0 = np.array([math.cos(dec0) * math.cos(ra0), math.cos(dec0) * math.sin(ra0), math.sin(dec0)])
    st = np.sqrt(np.clip(1 - z * z, 0, None))
    dot = st * np.cos(phi) * c0[0] + st * np.sin(phi) * c0[1] + z * c0[2]
    return dot >= math.cos(math.radians(radius_deg))


def des_like_footprint(z, phi, rng, band_ra_width=295.1):
    """DES-like footprint membership by pixel centre (ring by ring: dec is constant on a
    ring and rings of equal length and offset share their RA grid)."""
    w = [_edge_wiggle(rng) for _ in range(6)]
    out = np.zeros(len(z), bool)
    zlo, zhi = math.sin(math.radians(-61.01)), math.sin(math.radians(1.01))
    # ring boundaries: z is constant along a ring and changes between rings
    starts = np.flatnonzero(np.r_[True, z[1:] != z[:-1]])
    ends = np.r_[starts[1:], len(z)]
    cache = {}
    for a, b in zip(starts, ends):
        zz = z[a]
        if zz < zlo or zz > zhi:
            continue
        dec = math.degrees(math.asin(zz))
        key = (b - a, phi[a])
        if key not in cache:
            ra = np.degrees(phi[a:b]) % 360.0
            cache[key] = (ra, w[0](ra), w[1](ra), w[4](ra))
        ra, w0, w1, w4 = cache[key]
        w2, w3, w5 = w[2](dec)[0], w[3](dec)[0], w[5](dec)[0]
        band = (dec >= -60 + w0) & (dec <= -40 + w1) & (ra >= w2) & (ra < band_ra_width + w3)
        strip = (dec > -40 + w1) & (dec <= w4) & (ra >= w2) & (ra <= 10 + w5)
        out[a:b] = band | strip
    return out


def depth_pattern(z, phi, footprint, rng):
    """Smooth depth modulation t (zero off the footprint), max |t| = 1 on it."""
    idx = np.nonzero(footprint)[0]
    zz = z[idx]
    st = np.sqrt(np.clip(1 - zz * zz, 0, None))
    x, y = st * np.cos(phi[idx]), st * np.sin(phi[idx])
    t = np.zeros_like(zz)
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                t += rng.standard_normal() * x ** a * y ** b * zz ** c
    out = np.zeros_like(z)
    if len(idx):
        t -= t.mean()
        out[idx] = t / np.abs(t).max()
    return out


def pixel_area_arcmin2(nside: int) -> float:
    return 4 * math.pi / (12 * nside * nside) * ARCMIN2_PER_SR


def survey(nside: int, kind: str, seed: int):
    """Counts, mask and N^-1 for a footprint kind ('cap' or 'des')."""
    r_alm, r_fp, r_depth, r_cnt, r_noise = streams(seed)
    z, phi = pixel_positions(nside)
    if kind == "cap":
        fp = cap_footprint(z, phi)
        nbar = np.where(fp, 20.0, 0.0)
    elif kind == "des":
        fp = des_like_footprint(z, phi, r_fp)
        t = depth_pattern(z, phi, fp, r_depth)
        nbar = np.where(fp, 5.6 * pixel_area_arcmin2(nside) * (1 + 0.3 * t), 0.0)
    elif kind == "full":
        fp = np.ones_like(z, bool)
        nbar = np.full_like(z, 20.0)
    else:
        raise ValueError(kind)
    counts = r_cnt.poisson(nbar).astype(np.float64)
    mask = fp & (counts >= 1)
    ninv = np.where(mask, counts / SIGMA_E ** 2, 0.0)
    return dict(counts=counts, mask=mask, ninv=ninv, rng_alm=r_alm, rng_noise=r_noise)


def shape_noise(ninv: np.ndarray, rng, nreal: int = 1):
    """n ~ N(0, 1/N^-1) per component on the mask, 0 elsewhere; shape (nreal, 2, npix)."""
    sd = np.where(ninv > 0, 1.0 / np.sqrt(np.where(ninv > 0, ninv, 1.0)), 0.0)
    return rng.standard_normal((nreal, 2, len(ninv))) * sd


def workload(name: str, nside: int = None, lmax: int = None):
    """Inputs of a named workload: dict(nside, lmax, x_true (κ_E, κ_B), ninv, noise, tol).

    The shear itself, y = M (A x_true + n), needs the forward operator, so the
    caller forms it with whichever implementation it is testing or timing.
    """
    table = {
        "cap32": (32, 64, "cap", 1e-8),
        "des512": (512, 1024, "des", 1e-6),
        "des2048": (2048, 4096, "des", 1e-6),
        "grad512": (512, 1024, "des", 1e-6),
    }
    n0, l0, kind, tol = table[name]
    nside = nside or n0
    lmax = lmax or l0
    sv = survey(nside, kind, SEEDS[name])
    kE = grf_alm(lmax, cl_kappa(lmax), sv["rng_alm"])
    kB = np.zeros_like(kE)
    noise = shape_noise(sv["ninv"], sv["rng_noise"])[0]
    return dict(nside=nside, lmax=lmax, x_true=(kE, kB), ninv=sv["ninv"], mask=sv["mask"],
                noise=noise, tol=tol)


def flat_survey(n: int, seed: int = SEEDS["flat"], pix_arcmin: float = 0.86):
    """Flat-sky workload on an n x n periodic grid of pix_arcmin pixels: a DES-like patch (a
    rectangle over 70 % x 50 % of the grid, each edge displaced by up to 2 % of the side by a
    sum of random-phase sinusoids), counts Poisson(5.6 arcmin^-2 x pixel area x (1 + 0.3 t)),
    t a smooth random cubic in the pixel position with max |t| = 1 on the patch.  Returns
    dict(ninv [n*n], mask, x_true [n, n] complex, noise [2, n*n]), x_true the unitary 2D
    Fourier transform of a real Gaussian field with power ∝ (|k| + 10)^-2 (κ_B = 0)."""
    r_alm, r_fp, r_depth, r_cnt, r_noise = streams(seed)
    yy, xx = np.mgrid[0:n, 0:n] / float(n)
    s_edges = [_edge_wiggle(r_fp) for _ in range(4)]
    d = 0.02
    c = np.arange(n) / float(n) * 360.0            # edges vary along the other coordinate
    x0 = (0.15 + d * s_edges[0](c))[:, None]
    x1 = (0.85 + d * s_edges[1](c))[:, None]
    y0 = (0.25 + d * s_edges[2](c))[None, :]
    y1 = (0.75 + d * s_edges[3](c))[None, :]
    fp = (xx > x0) & (xx < x1) & (yy > y0) & (yy < y1)
    t = np.zeros((n, n))
    u, v = xx - 0.5, yy - 0.5
    for a in range(4):
        for b in range(4 - a):
            t += r_depth.standard_normal() * u ** a * v ** b
    t = np.where(fp, t - t[fp].mean(), 0.0)
    t /= np.abs(t).max()
    nbar = np.where(fp, 5.6 * pix_arcmin ** 2 * (1 + 0.3 * t), 0.0)
    counts = r_cnt.poisson(nbar).astype(np.float64)
    mask = fp & (counts >= 1)
    ninv = np.where(mask, counts / SIGMA_E ** 2, 0.0).ravel()
    k = np.fft.fftfreq(n, d=1.0 / n)
    kk = np.sqrt(k[None, :] ** 2 + k[:, None] ** 2)
    amp = np.sqrt(1e-4 * (kk + 10.0) ** -2.0)
    x_true = amp * np.fft.fft2(r_alm.standard_normal((n, n)), norm="ortho")
    x_true[0, 0] = 0.0
    noise = shape_noise(ninv, r_noise)[0]
    return dict(n=n, ninv=ninv, mask=mask.ravel(), x_true=x_true, noise=noise)
