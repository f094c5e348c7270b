/*
 * akra_oracle.c -- plain, slow FP64 CPU oracle for the AKRA 3.0 operator chain.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path links, loads or calls
 * this file; only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg do.  It shares no code with the CUDA library.
 *
 * What is here (everything else -- ring DFTs, E/B recombination, the KS kernel,
 * CG -- is plain numpy in oracle/oracle.py):
 *   - HEALPix RING geometry (the pixelisation of Sec. III B; the grid itself is
 *     the standard one of Gorski et al. 2005).
 *   - spin-weighted associated Legendre functions  sλ_lm(θ), defined by
 *     sY_lm(θ,φ) = sλ_lm(θ) e^{imφ}  (Eq. 1 uses s = ±2).
 *   - the Legendre halves of the spin-2 synthesis (Eq. 1) and of its exact
 *     transpose (the adjoint A^T of Sec. II B), as direct sums.
 *
 * Conventions
 *   - sY_lm is the Goldberg et al. (1967) function; s = 0 is the Condon-Shortley
 *     Y_lm.  Seeds below are the single-term case of the Goldberg sum; the
 *     l-recurrence is the three-term Wigner-d recurrence written for the
 *     normalised sλ_lm.
 *   - packed alm index  idx(l,m) = m(2L+1-m)/2 + l,  0 <= m <= l <= L;
 *     complex values are interleaved (re, im) doubles.
 *   - ring r = 1 .. 4N-1 from the north pole; pixel phases φ_j = π(2j+σ)/nφ.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC akra_oracle.c -o liboracle.so -lm
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static long long tri_index(int lmax, int l, int m)
{
    return (long long)m * (2LL * lmax + 1 - m) / 2 + l;
}

/* ---------------------------------------------------------------------------
 * HEALPix RING geometry.
 *   north polar cap, ring i < N :  z = 1 - i^2/(3N^2), nφ = 4i, σ = 1,
 *                                  first pixel 2i(i-1)
 *   equatorial belt, N <= i <= 2N: z = 4/3 - 2i/(3N), nφ = 4N,
 *                                  σ = (i - N + 1) mod 2,
 *                                  first pixel 2N(N-1) + 4N(i-N)
 *   south half: ring 4N-i mirrors ring i (z -> -z, same nφ and σ), and the
 *   pixels of rings 4N-i .. 4N-1 are the last first(i)+nφ(i) pixels.
 * Returns 0 on success, -1 for an out-of-range ring.
 * ------------------------------------------------------------------------- */
int orc_ring_info(int nside, int ring, double *cos_theta, double *sin_theta,
                  long long *nphi, int *sigma, long long *first_pixel)
{
    long long N = nside;
    if (nside < 1 || ring < 1 || ring > 4 * nside - 1)
        return -1;
    long long npix = 12 * N * N;
    long long i = ring;
    int north = 1;
    if (i > 2 * N) {
        i = 4 * N - i;
        north = 0;
    }
    double z, st;
    long long n, first;
    int sg;
    if (i < N) {
        double one_minus_z = (double)(i * i) / (3.0 * (double)(N * N));
        z = 1.0 - one_minus_z;
        st = sqrt(one_minus_z * (2.0 - one_minus_z));
        n = 4 * i;
        sg = 1;
        first = 2 * i * (i - 1);
    } else {
        z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * (double)N);
        st = sqrt((1.0 - z) * (1.0 + z));
        n = 4 * N;
        sg = (int)((i - N + 1) % 2);
        first = 2 * N * (N - 1) + 4 * N * (i - N);
    }
    if (!north) {
        z = -z;
        first = npix - first - n;
    }
    *cos_theta = z;
    *sin_theta = st;
    *nphi = n;
    *sigma = sg;
    *first_pixel = first;
    return 0;
}

/* ---------------------------------------------------------------------------
 * Spin-weighted associated Legendre function sλ_lm(θ), l = 0..lmax, any m.
 *
 * Negative m uses the conjugation relation of spin-weighted harmonics,
 *   sY*_lm = (-1)^{s+m} (-s)Y_{l,-m}   =>   sλ_{l,-m} = (-1)^{s+m} (-s)λ_{l,m}.
 *
 * For m >= 0 the first non-zero degree is l0 = max(m,|s|).  There the Goldberg
 * sum has a single term, which gives
 *   |sλ_{l0,m}| = sqrt((2 l0 + 1)/(4π) (2 l0)!/(a! b!)) sin^a(θ/2) cos^b(θ/2),
 *     (a,b) = (m+s, m-s)      sign (-1)^m      if m >= |s|,
 *     (a,b) = (s+m, s-m)      sign (-1)^m      if s > m,
 *     (a,b) = (|s|-m, |s|+m)  sign (-1)^{|s|}  if -s > m.
 * Upward in l (three-term Wigner-d recurrence, normalised):
 *   sλ_{l+1} = A_l [ (cosθ + m s/(l(l+1))) sλ_l - B_l sλ_{l-1} ],
 *   A_l = sqrt((2l+3)/(2l+1)) (l+1)(2l+1) / sqrt(((l+1)^2-m^2)((l+1)^2-s^2)),
 *   B_l = sqrt((l^2-m^2)(l^2-s^2)) / (l(2l+1)) * sqrt((2l+1)/(2l-1)),
 * with sλ_{l0-1} = 0.  The values are carried as mantissa * 2^e so that seeds
 * far below the double range (polar rings, large m) are not lost; the output
 * is ldexp(mantissa, e), which is exactly zero where the function is below the
 * double range.
 * ------------------------------------------------------------------------- */
void orc_spin_lambda(int s, int lmax, int m, double cos_theta, double sin_theta,
                     double *out)
{
    for (int l = 0; l <= lmax; l++)
        out[l] = 0.0;
    if (m < 0) {
        orc_spin_lambda(-s, lmax, -m, cos_theta, sin_theta, out);
        if (((s + m) % 2 + 2) % 2 == 1)
            for (int l = 0; l <= lmax; l++)
                out[l] = -out[l];
        return;
    }
    int as = s < 0 ? -s : s;
    int l0 = m > as ? m : as;
    if (l0 > lmax)
        return;
    int a, b;
    double sign;
    if (m >= as) {
        a = m + s;
        b = m - s;
        sign = (m % 2) ? -1.0 : 1.0;
    } else if (s > 0) {
        a = s + m;
        b = s - m;
        sign = (m % 2) ? -1.0 : 1.0;
    } else {
        a = as - m;
        b = as + m;
        sign = (as % 2) ? -1.0 : 1.0;
    }
    /* half-angle functions, each from the numerically stable side */
    double sh, ch;
    if (cos_theta >= 0.0) {
        ch = sqrt(0.5 * (1.0 + cos_theta));
        sh = sin_theta / (2.0 * ch);
    } else {
        sh = sqrt(0.5 * (1.0 - cos_theta));
        ch = sin_theta / (2.0 * sh);
    }
    double log2_seed =
        0.5 * (log2(2.0 * l0 + 1.0) - log2(4.0 * M_PI) +
               (lgamma(2.0 * l0 + 1.0) - lgamma(a + 1.0) - lgamma(b + 1.0)) / log(2.0));
    if (a > 0)
        log2_seed += a * log2(sh);
    if (b > 0)
        log2_seed += b * log2(ch);
    int e = (int)floor(log2_seed);
    double v_prev = 0.0;
    double v_cur = sign * exp2(log2_seed - e);
    out[l0] = ldexp(v_cur, e);
    double mm = (double)m * m, ss = (double)s * s;
    for (int l = l0; l < lmax; l++) {
        double lp1 = l + 1.0;
        double A = sqrt((2.0 * l + 3.0) / (2.0 * l + 1.0)) * lp1 * (2.0 * l + 1.0) /
                   sqrt((lp1 * lp1 - mm) * (lp1 * lp1 - ss));
        double B = (l == l0) ? 0.0
                             : sqrt(((double)l * l - mm) * ((double)l * l - ss)) /
                                   ((double)l * (2.0 * l + 1.0)) *
                                   sqrt((2.0 * l + 1.0) / (2.0 * l - 1.0));
        double c = (l == 0) ? 0.0 : (double)m * s / ((double)l * lp1);
        double v_next = A * ((cos_theta + c) * v_cur - B * v_prev);
        v_prev = v_cur;
        v_cur = v_next;
        if (fabs(v_cur) > 0x1p200) {
            v_cur = ldexp(v_cur, -400);
            v_prev = ldexp(v_prev, -400);
            e += 400;
        }
        out[l + 1] = ldexp(v_cur, e);
    }
}

/* ---------------------------------------------------------------------------
 * Legendre half of the spin-2 synthesis (Eqs. 1-2).
 *   γ(θ,φ) = Σ_{l,m} γ_{2,lm} 2Y_lm(θ,φ),   γ_{2,lm} = -(a_E,lm + i a_B,lm),
 * with the negative-m coefficients of the real E and B fields given by
 *   a_{X,l,-m} = (-1)^m conj(a_{X,lm}).
 * For each selected ring this returns
 *   F(ring, m) = Σ_l γ_{2,lm} 2λ_lm(θ_ring),   m = -L..L,
 * stored as F[k][L+m] (complex interleaved).  The φ-sum is done by the caller.
 * Im(a_{X,l0}) is ignored (real fields).
 * ------------------------------------------------------------------------- */
void orc_legendre_synth(int nside, int lmax, const double *aE, const double *aB,
                        int nsel, const int *rings, double *F)
{
    int L = lmax;
    long long width = 2LL * L + 1;
#pragma omp parallel
    {
        double *lam_pos = (double *)malloc(sizeof(double) * (L + 1));
        double *lam_neg = (double *)malloc(sizeof(double) * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < nsel; k++) {
            double ct, st;
            long long nphi, first;
            int sg;
            orc_ring_info(nside, rings[k], &ct, &st, &nphi, &sg, &first);
            double *Fk = F + 2 * width * k;
            for (long long j = 0; j < 2 * width; j++)
                Fk[j] = 0.0;
            for (int m = 0; m <= L; m++) {
                orc_spin_lambda(2, L, m, ct, st, lam_pos);
                double pr = 0.0, pi = 0.0;
                for (int l = m; l <= L; l++) {
                    long long ix = tri_index(L, l, m);
                    double er = aE[2 * ix], ei = (m == 0) ? 0.0 : aE[2 * ix + 1];
                    double br = aB[2 * ix], bi = (m == 0) ? 0.0 : aB[2 * ix + 1];
                    /* γ_{2,lm} = -(a_E + i a_B) */
                    double gr = -(er - bi), gi = -(ei + br);
                    pr += gr * lam_pos[l];
                    pi += gi * lam_pos[l];
                }
                Fk[2 * (L + m)] = pr;
                Fk[2 * (L + m) + 1] = pi;
                if (m == 0)
                    continue;
                orc_spin_lambda(2, L, -m, ct, st, lam_neg);
                double sgn = (m % 2) ? -1.0 : 1.0;
                double nr = 0.0, ni = 0.0;
                for (int l = m; l <= L; l++) {
                    long long ix = tri_index(L, l, m);
                    /* a_{X,l,-m} = (-1)^m conj(a_{X,lm}) */
                    double er = sgn * aE[2 * ix], ei = -sgn * aE[2 * ix + 1];
                    double br = sgn * aB[2 * ix], bi = -sgn * aB[2 * ix + 1];
                    double gr = -(er - bi), gi = -(ei + br);
                    nr += gr * lam_neg[l];
                    ni += gi * lam_neg[l];
                }
                Fk[2 * (L - m)] = nr;
                Fk[2 * (L - m) + 1] = ni;
            }
        }
        free(lam_pos);
        free(lam_neg);
    }
}

/* ---------------------------------------------------------------------------
 * Legendre half of the exact adjoint (transpose) of the spin-2 synthesis.
 * With w_p = u1_p + i u2_p and  G(ring, m) = Σ_{j in ring} w_j e^{-i m φ_j}
 * (computed by the caller, stored G[ring-1][L+m]):
 *   g_lm = Σ_p w_p 2Y*_lm(p)           = Σ_rings 2λ_lm(θ) G(m),
 *   h_lm = Σ_p conj(w_p) (-2)Y*_lm(p)  = Σ_rings (-2)λ_lm(θ) conj(G(-m)),
 * for 0 <= m <= l <= L (packed, complex interleaved).  The caller forms
 * a_E = -(g+h)/2, a_B = (i/2)(g-h) (Eq. 2 applied to g, h).
 * Only the m listed in ms[] are computed; the other entries are left as is.
 * ------------------------------------------------------------------------- */
void orc_legendre_adjoint(int nside, int lmax, const double *G, int nm,
                          const int *ms, double *g_out, double *h_out)
{
    int L = lmax;
    int nring = 4 * nside - 1;
    long long width = 2LL * L + 1;
#pragma omp parallel
    {
        double *lam_p = (double *)malloc(sizeof(double) * (L + 1));
        double *lam_m = (double *)malloc(sizeof(double) * (L + 1));
#pragma omp for schedule(dynamic, 1)
        for (int km = 0; km < nm; km++) {
            int m = ms[km];
            for (int l = m; l <= L; l++) {
                long long ix = tri_index(L, l, m);
                g_out[2 * ix] = g_out[2 * ix + 1] = 0.0;
                h_out[2 * ix] = h_out[2 * ix + 1] = 0.0;
            }
            for (int r = 1; r <= nring; r++) {
                double ct, st;
                long long nphi, first;
                int sg;
                orc_ring_info(nside, r, &ct, &st, &nphi, &sg, &first);
                const double *Gr = G + 2 * width * (r - 1);
                double gpr = Gr[2 * (L + m)], gpi = Gr[2 * (L + m) + 1];
                /* conj(G(-m)) */
                double qr = Gr[2 * (L - m)], qi = -Gr[2 * (L - m) + 1];
                orc_spin_lambda(2, L, m, ct, st, lam_p);
                orc_spin_lambda(-2, L, m, ct, st, lam_m);
                for (int l = m; l <= L; l++) {
                    long long ix = tri_index(L, l, m);
                    g_out[2 * ix] += lam_p[l] * gpr;
                    g_out[2 * ix + 1] += lam_p[l] * gpi;
                    h_out[2 * ix] += lam_m[l] * qr;
                    h_out[2 * ix + 1] += lam_m[l] * qi;
                }
            }
        }
        free(lam_p);
        free(lam_m);
    }
}

/* number of OpenMP threads the oracle runs with (reported as cpu_baseline cores) */
int orc_num_threads(void)
{
    int n = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
#endif
    return n;
}
