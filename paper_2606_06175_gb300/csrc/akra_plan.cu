// akra_plan.cu -- plan creation (HEALPix ring geometry, recurrence coefficients, ring
// twiddles), pixel weights, operator composition and the C entry points for the
// transforms and H.  The CG entry points live in akra_cg.cu.
#include <complex>
#include <cstdarg>
#include <cstring>
#include <algorithm>
#include <mutex>

#include <type_traits>

#include "akra_internal.cuh"

namespace akra {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

// ---------------------------------------------------------------------------
// K1: HEALPix RING geometry (Gorski et al. 2005; the pixelisation of Sec. III B)
//   ring i (1..4N-1), i' = min(i, 4N-i):
//     polar  i' < N : 1 - z = i'^2/(3N^2), n = 4i', σ = 1, first = 2i'(i'-1)
//     belt  i' >= N : 1 - z = (2i'-N)/(3N), n = 4N, σ = (i'-N+1) mod 2,
//                     first = 2N(N-1) + 4N(i'-N)
//   south rings mirror: z -> -z, first = npix - first(i') - n.
//   unit u (0..2N-1): north ring u+1 and its mirror 4N-u-1 (none for the equator u = 2N-1)
// ---------------------------------------------------------------------------
__global__ void k_geometry(int N, RingInfo *rings, UnitInfo *units)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const long long NN = N;
    const long long npix = 12 * NN * NN;
    auto ring_of = [&](int ring, RingInfo &ri, double &omz) {
        const bool north = ring <= 2 * N;
        const long long i = north ? ring : 4 * NN - ring;
        long long first;
        if (i < N) {
            omz = (double)(i * i) / (3.0 * (double)(NN * NN));
            ri.nphi = (int)(4 * i);
            ri.sigma = 1;
            ri.ilen = (int)i;
            first = 2 * i * (i - 1);
        } else {
            omz = (double)(2 * i - NN) / (3.0 * (double)NN);
            ri.nphi = (int)(4 * NN);
            ri.sigma = (int)((i - NN + 1) & 1);
            ri.ilen = N;
            first = 2 * NN * (NN - 1) + 4 * NN * (i - NN);
        }
        ri.z = north ? 1.0 - omz : omz - 1.0;
        ri.st = sqrt(omz * (2.0 - omz));
        ri.first = north ? first : npix - first - ri.nphi;
        ri.tw_off = 4LL * ri.ilen * (ri.ilen - 1);
        ri.pad = 0;
    };
    if (t < 4 * N - 1) {
        RingInfo ri;
        double omz;
        ring_of(t + 1, ri, omz);
        rings[t] = ri;
    }
    if (t < 2 * N) {
        RingInfo ri;
        double omz;   // 1 - cos θ of the north ring, exact from the ring formulas
        ring_of(t + 1, ri, omz);
        UnitInfo u;
        u.x = ri.z;
        u.ls = 0.5 * log2(0.5 * omz);          // sin^2(θ/2) = (1 - z)/2
        u.lc = 0.5 * log2(0.5 * (2.0 - omz));  // cos^2(θ/2) = (1 + z)/2
        u.ring_n = t;
        u.ring_s = (t + 1 < 2 * N) ? (4 * N - (t + 1)) - 1 : -1;
        units[t] = u;
    }
}

// Recurrence coefficients per (l, m), s = ±2 (Wigner-d, normalised):
//   sλ_{l+1} = (A_l x + s A_l m/(l(l+1))) sλ_l - A_l B_l sλ_{l-1}
//   A_l = sqrt((2l+3)/(2l+1)) (l+1)(2l+1) / sqrt(((l+1)^2-m^2)((l+1)^2-4))
//   B_l = sqrt((l^2-m^2)(l^2-4))/(l(2l+1)) sqrt((2l+1)/(2l-1))   (0 at l = l0)
// stored in monic form: with sλ_l = σ_l μ_l, σ_{l0} = 1, σ_{l0+1} = κ, σ_{l+1} = A_l B_l σ_{l-1},
//   μ_{l+1} = (A'_l x ± c'_l) μ_l - μ_{l-1},  A'_l = A_l σ_l/σ_{l+1},  c'_l = A_l (2m/(l(l+1))) σ_l/σ_{l+1}.
// σ_{l+1} = A_l B_l σ_{l-1} fixes each parity chain up to its start value; κ (the odd chain's)
// is chosen so that σ_lmax = σ_{lmax-1}, which makes the scale smooth in l (A'_l -> 2 as l grows
// instead of alternating between two values).  Near the poles (x -> 1) the step of a smooth
// monic recurrence, μ_{l+1} - μ_l, is then small, which the difference form of the FP32 kernels
// relies on.  Entry {A', c', σ_l, A' - 2} (A' - 2 formed in FP64).  One thread per m.
__global__ void k_coef(int L, double4_32a *c64, float4 *c32)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > L) return;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const int l0 = m > 2 ? m : 2;
    for (int l = m; l < l0 && l <= L; l++) {
        c64[mbase + l] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
        c32[mbase + l] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const double mm = (double)m * m;
    auto AB = [&](int l, double &A, double &B) {
        const double dl = l, lp1 = l + 1.0;
        A = sqrt((2 * dl + 3) / (2 * dl + 1)) * lp1 * (2 * dl + 1) / sqrt((lp1 * lp1 - mm) * (lp1 * lp1 - 4.0));
        B = (l == l0) ? 0.0
                      : sqrt((dl * dl - mm) * (dl * dl - 4.0)) / (dl * (2 * dl + 1)) * sqrt((2 * dl + 1) / (2 * dl - 1));
    };
    // pass 1: both chains with unit start values, to σ_lmax and σ_{lmax-1}
    double kappa = 1.0;
    if (L > l0) {
        double sig_prev = 1.0, sig = 1.0;   // σ_{l-1}, σ_l
        for (int l = l0; l < L; l++) {
            double A, B;
            AB(l, A, B);
            const double sig_next = (l == l0) ? 1.0 : A * B * sig_prev;
            sig_prev = sig;
            sig = sig_next;
        }
        // now sig = σ_L, sig_prev = σ_{L-1}; the chain of l0 + 1 is the one scaled by κ
        kappa = ((L - l0) & 1) ? sig_prev / sig : sig / sig_prev;
    }
    double sig_prev = 1.0, sig = 1.0;
    for (int l = l0; l <= L; l++) {
        double A, B;
        AB(l, A, B);
        const double sig_next = (l == l0) ? kappa : A * B * sig_prev;
        const double r = sig / sig_next;
        const double a = A * r, c = A * 2.0 * m / ((double)l * (l + 1.0)) * r;
        c64[mbase + l] = make_double4_32a(a, c, sig, 0.0);
        c32[mbase + l] = make_float4((float)a, (float)c, (float)sig, (float)(a - 2.0));
        sig_prev = sig;
        sig = sig_next;
    }
}

// log2 of the seed prefactor sqrt((2 l0 + 1)/(4π) (2 l0)!/(a! b!)), a = m+2, b = |m-2|,
// l0 = max(m, 2) (single-term Goldberg sum at l = l0); also D_l of Eq. 3.
__global__ void k_seed(int L, double *seedC, double *D64, float *D32)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m > L) return;
    const int l0 = m > 2 ? m : 2, a = m + 2, b = m >= 2 ? m - 2 : 2 - m;
    seedC[m] = 0.5 * (log2(2.0 * l0 + 1.0) - log2(4.0 * 3.14159265358979323846) +
                      (lgamma(2.0 * l0 + 1.0) - lgamma(a + 1.0) - lgamma(b + 1.0)) /
                          0.69314718055994530942);
    const double l = m;
    const double D = m >= 2 ? -sqrt((l - 1) * (l + 2) / (l * (l + 1))) : 0.0;
    D64[m] = D;
    D32[m] = (float)D;
}

// Seeds of the two spin recurrences at l0 = max(m, 2) for every (m, ring pair), in FP64:
//   log2|2λ| = C_m + a log2 sin(θ/2) + b log2 cos(θ/2), (a, b) = (m+2, |m-2|), sign (-1)^m,
//   log2|(-2)λ| with (a, b) swapped, sign (-1)^m for m >= 2 and +1 below,
// scaled by 2^(-Q e) with one exponent index e <= 0 per pair (Q = 64 for the FP32 table,
// 600 for FP64) so that the larger one lies in [2^(-Q/2), 2^(Q/2)).
__device__ void seed_values(int m, double Cm, double ls, double lc, int Q, double &vp, double &vm,
                            int &e)
{
    const int a = m + 2, b = m >= 2 ? m - 2 : 2 - m;
    const double Lp = Cm + a * ls + b * lc;
    const double Lm = Cm + b * ls + a * lc;
    const double sp = (m & 1) ? -1.0 : 1.0;
    const double sm = (m >= 2) ? sp : 1.0;
    int ee = (int)floor((fmax(Lp, Lm) + 0.5 * Q) / Q);
    if (ee > 0) ee = 0;
    vp = sp * exp2(Lp - (double)Q * ee);
    vm = sm * exp2(Lm - (double)Q * ee);
    e = ee;
}

// Start states of the recurrences for every (m, ring pair).  The FP64 monic recurrence runs
// from the seed at l0 (exponent index with Q = 600) until the larger of |2λ_l|, |(-2)λ_l|
// first exceeds 2^-90 (FP64 kernels) and 2^-40 (FP32 kernels); below that the pair's
// contributions are negligible at the precision's rounding level.  Each precision's start is
// the last grid point g = l0 + 64 j at or before that l, with the state (μ_g, μ_{g-1}) of both
// spins re-scaled to the precision's exponent index (Q = 64 for FP32).  Pairs that stay below
// the threshold up to lmax get g = kNeverLive.  Also accumulates per pair the steps
// Σ_m (lmax + 1 - g) that the kernels take.
__global__ void k_start_states(int L, int nunit, const double *seedC, const UnitInfo *units,
                               const double4_32a *coef, float4 *s32, double4_32a *s64,
                               int2 *g32, int2 *g64, unsigned long long *steps, float2 *d32)
{
    const int m = blockIdx.y;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= nunit) return;
    const UnitInfo ui = units[u];
    const int l0 = m > 2 ? m : 2;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const size_t o = (size_t)m * nunit + u;
    const double x = ui.x;
    double vp, vm, vpo = 0, vmo = 0;
    int e;
    seed_values(m, seedC[m], ui.ls, ui.lc, Scale<double>::Q, vp, vm, e);
    double gp = vp, gm = vm, gpo = 0, gmo = 0;
    int ge = e, gl = l0;
    bool have64 = false;
    const double thr64 = 0x1p-90, thr32 = 0x1p-40;
    int l = l0;
    for (; l <= L; l++) {
        if (((l - l0) & (kStartGrid - 1)) == 0) {
            gp = vp;
            gm = vm;
            gpo = vpo;
            gmo = vmo;
            ge = e;
            gl = l;
        }
        const double4_32a c = coef[mbase + l];
        // |λ| = σ |μ| 2^(600 e); below 2^-300 while e < 0
        const double mag = e == 0 ? fmax(fabs(vp), fabs(vm)) * c.z : 0.0;
        if (!have64 && mag > thr64) {
            s64[o] = make_double4_32a(gp, gm, gpo, gmo);
            g64[o] = make_int2(gl, ge);
            atomicAdd(&steps[nunit + u], (unsigned long long)(L + 1 - gl));
            have64 = true;
        }
        if (mag > thr32) {
            // FP32 exponent index: the largest of the four values in [2^-32, 2^32)
            const double mx = fmax(fmax(fabs(gp), fabs(gm)), fmax(fabs(gpo), fabs(gmo)));
            int e32 = (int)floor((log2(mx) + (double)Scale<double>::Q * ge + 32.0) / 64.0);
            if (e32 > 0) e32 = 0;
            const int sh = Scale<double>::Q * ge - Scale<float>::Q * e32;
            s32[o] = make_float4((float)ldexp(gp, sh), (float)ldexp(gm, sh), (float)ldexp(gpo, sh),
                                 (float)ldexp(gmo, sh));
            // the difference form starts from (μ_g, μ_g - μ_{g-1}), the difference taken in FP64
            d32[o] = make_float2((float)ldexp(gp - gpo, sh), (float)ldexp(gm - gmo, sh));
            g32[o] = make_int2(gl, e32);
            atomicAdd(&steps[u], (unsigned long long)(L + 1 - gl));
            break;
        }
        const double np = fma(fma(c.x, x, c.y), vp, -vpo);
        const double nm = fma(fma(c.x, x, -c.y), vm, -vmo);
        vpo = vp;
        vmo = vm;
        vp = np;
        vm = nm;
        if (e < 0 && (fabs(vp) > Scale<double>::hi() || fabs(vm) > Scale<double>::hi())) {
            vp *= Scale<double>::inv();
            vm *= Scale<double>::inv();
            vpo *= Scale<double>::inv();
            vmo *= Scale<double>::inv();
            e++;
        }
    }
    if (l > L) {
        s32[o] = make_float4(0.f, 0.f, 0.f, 0.f);
        d32[o] = make_float2(0.f, 0.f);
        g32[o] = make_int2(kNeverLive, 0);
        if (!have64) {
            s64[o] = make_double4_32a(0.0, 0.0, 0.0, 0.0);
            g64[o] = make_int2(kNeverLive, 0);
        }
    }
}

// e^{iπ t/n} for every ring length n = 4i (i = 1..N), t in [0, 2n), at offset 4i(i-1)
__global__ void k_twiddles(int N, double2 *tw64, float2 *tw32)
{
    const int i = blockIdx.y + 1;
    const int n = 4 * i;
    const long long off = 4LL * i * (i - 1);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 2 * n; t += gridDim.x * blockDim.x) {
        double s, c;
        sincospi((double)t / (double)n, &s, &c);
        tw64[off + t] = make_double2(c, s);
        tw32[off + t] = make_float2((float)c, (float)s);
    }
}

// per-l preconditioner weights per packed index: (mean_all(M N^-1) D_l^2 + λ_eff)^-1
__global__ void k_pw(int L, const double *D, double mean_mninv, double lam_eff, double *pw64, float *pw32)
{
    const int m = blockIdx.x;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
        const double d = mean_mninv * D[l] * D[l] + lam_eff;
        const double w = d > 0 ? 1.0 / d : 0.0;
        pw64[mbase + l] = w;
        pw32[mbase + l] = (float)w;
    }
}

__global__ void k_iota(int n, int *out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = t;
}

// per ring: W = ω M N^-1 in both precisions; count of masked pixels, Σ N^-1 over them,
// and the number of invalid (negative or non-finite) entries
// W32r holds the FP32 weights in the order the FP32 ring FFT visits the pixels: slot k of a
// power-of-two ring (length 2^b) holds pixel brev_b(k), other rings are in pixel order.
__global__ void k_weights(const RingInfo *rings, const double *ninv, double omega, double *W64,
                          float *W32, float *W32r, double *ring_sum, double *ring_cnt, double *ring_bad)
{
    const RingInfo ri = rings[blockIdx.x];
    const bool pow2 = (ri.nphi & (ri.nphi - 1)) == 0;
    const int logn = 31 - __clz(ri.nphi);
    double s = 0, c = 0, bad = 0;
    for (int j = threadIdx.x; j < ri.nphi; j += blockDim.x) {
        const double v = ninv[ri.first + j];
        const bool ok = isfinite(v) && v >= 0;
        const double w = (ok && v > 0) ? omega * v : 0.0;
        W64[ri.first + j] = w;
        W32[ri.first + j] = (float)w;
        W32r[ri.first + (pow2 ? (int)(__brev((unsigned)j) >> (32 - logn)) : j)] = (float)w;
        if (!ok) bad += 1;
        if (ok && v > 0) {
            s += v;
            c += 1;
        }
    }
    __shared__ double sh[3][256];
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = c;
    sh[2][threadIdx.x] = bad;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off)
            for (int q = 0; q < 3; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ring_sum[blockIdx.x] = sh[0][0];
        ring_cnt[blockIdx.x] = sh[1][0];
        ring_bad[blockIdx.x] = sh[2][0];
    }
}

// radices of n = 4i: odd primes below kBluePrime first (direct passes, smallest Ns), then 4s
// and a 2; a prime >= kBluePrime (at most one: two would exceed 4 nside) is left for a last,
// Bluestein pass, where each of its length-p transforms reads and writes only its own strided
// positions of the ring
static FftFactors factorize(int n)
{
    FftFactors f{};
    int m = n;
    std::vector<int> small, big;
    while (m % 4 == 0) { small.push_back(4); m /= 4; }
    while (m % 2 == 0) { small.push_back(2); m /= 2; }
    for (int d = 3; (long long)d * d <= m; d += 2)
        while (m % d == 0) { big.push_back(d); m /= d; }
    if (m > 1) big.push_back(m);
    for (int d : big) {
        if (d >= kBluePrime) f.blue_p = d;
        else f.f[f.nf++] = d;
    }
    for (int d : small) f.f[f.nf++] = d;
    if (f.blue_p) {
        f.blue_M = 1;
        while (f.blue_M < 2 * f.blue_p - 1) f.blue_M *= 2;
    }
    return f;
}

// in-place radix-2 DFT on the host, out_k = Σ_j x_j e^{sign 2πi jk/M} (M a power of two)
static void host_fft(std::vector<std::complex<double>> &x, int sign)
{
    const int M = (int)x.size();
    for (int i = 1, j = 0; i < M; i++) {
        int bit = M >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    for (int len = 2; len <= M; len <<= 1) {
        for (int i = 0; i < M; i += len)
            for (int k = 0; k < len / 2; k++) {
                double sn, cs;
                sincospi(sign * 2.0 * k / len, &sn, &cs);
                const std::complex<double> w(cs, sn), u = x[i + k], v = x[i + k + len / 2] * w;
                x[i + k] = u + v;
                x[i + k + len / 2] = u - v;
            }
    }
}

// Bluestein tables of prime p with convolution length M: h_q = e^{iπ q²/p} (q < p) and, for
// each transform sign s = ±1, G_s = DFT^-_M(g_s) with g_s[k] = e^{-s iπ k²/p} at k and M - k
// (|k| < p), so that Σ_q z_q e^{s 2πi qr/p} = h_r^s · (1/M) DFT^+_M(DFT^-_M(z h^s) · G_s)[r]
// (h^+ = h, h^- = conj(h)).  Phases from q² mod 2p, exact in integers.
static void blue_tables(int p, int M, std::vector<double2> &out)
{
    auto cis = [&](long long t) {   // e^{iπ t / p}
        double sn, cs;
        sincospi((double)(t % (2LL * p)) / p, &sn, &cs);
        return std::complex<double>(cs, sn);
    };
    for (int q = 0; q < p; q++) {
        const std::complex<double> h = cis((long long)q * q);
        out.push_back(make_double2(h.real(), h.imag()));
    }
    for (int s : {1, -1}) {
        std::vector<std::complex<double>> g(M, 0.0);
        for (int k = 0; k < p; k++) {
            const std::complex<double> v = s > 0 ? std::conj(cis((long long)k * k)) : cis((long long)k * k);
            g[k] = v;
            if (k > 0) g[M - k] = v;
        }
        host_fft(g, -1);
        for (int k = 0; k < M; k++) out.push_back(make_double2(g[k].real(), g[k].imag()));
    }
}

akra_status ws_reserve(akra_plan p, Workspace &w, size_t bytes)
{
    if (bytes <= w.bytes) return AKRA_OK;
    if (w.ptr) {
        AKRA_CUDA_TRY(cudaDeviceSynchronize());
        cudaFree(w.ptr);
        w.ptr = nullptr;
        w.bytes = 0;
    }
    p->ws_gen++;   // captured CG graphs that refer to the old buffer are now stale
    if (cudaMalloc(&w.ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        w.ptr = nullptr;
        set_error("workspace allocation of %zu bytes failed", bytes);
        return AKRA_ENOMEM;
    }
    w.bytes = bytes;
    return AKRA_OK;
}

akra_status tc_error_check(akra_plan p)
{
    if (!p->d_tc_err) return AKRA_OK;
    int h = 0;
    AKRA_CUDA_TRY(cudaMemcpy(&h, p->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (!h) return AKRA_OK;
    AKRA_CUDA_TRY(cudaMemset(p->d_tc_err, 0, sizeof(int)));
    set_error("a bounded wait inside an FP32 Legendre kernel (tensor-core completion or the "
              "adjoint's tile hand-over) ran out: the FP32 operator results since the last "
              "blocking call are invalid");
    return AKRA_ECUDA;
}

size_t plan_device_bytes(akra_plan p)
{
    return p->bytes_tables + p->phi.bytes + p->partial.bytes + p->cg.bytes + p->red.bytes +
           p->xsave.bytes + p->red_cl.bytes + p->bpre.bytes;
}

LegShape leg_shape(akra_plan p, akra_prec prec, int R)
{
    const long long key = (long long)prec * 1000 + (R > 999 ? 999 : R);
    auto it = p->shapes.find(key);
    if (it != p->shapes.end()) return it->second;
    // defaults (measured on the DES-like footprint at Nside 1024-2048; akra_autotune refines):
    // FP32 synthesis one ring pair per thread, with up to 4 RHS per block, and the paired adjoint
    // at 5 pairs per thread, one RHS per block; FP64 synthesis up to 4 RHS per block, adjoint 2
    // pairs per thread and 2 RHS per block (4 pairs, 1 RHS at R = 1)
    if (prec == AKRA_F64) {
        if (R >= 4) return LegShape{1, 128, 4, 2, 0, 2};
        if (R >= 2) return LegShape{1, 128, 2, 2, 0, 2};
        return LegShape{1, 128, 1, 4};
    }
    if (R >= 4) return LegShape{1, 128, 4, 5, 0, 1};
    if (R >= 2) return LegShape{1, 128, 2, 5, 0, 1};
    return LegShape{1, 128, 1, 5};
}

template <typename T> static akra_prec prec_of();
template <> akra_prec prec_of<float>() { return AKRA_F32; }
template <> akra_prec prec_of<double>() { return AKRA_F64; }

static size_t phi_bytes(akra_plan p, size_t elem, int R)
{
    return (size_t)R * p->nring * (2 * (size_t)p->lmax + 1) * elem;
}

template <typename T>
akra_status op_synth(akra_plan p, LegMode mode, const void *alm, void *map, bool weighted, int R,
                     cudaStream_t st)
{
    if (is_flat(p)) return flat_op_A<T>(p, alm, map, weighted, R, st);
    AKRA_TRY(ws_reserve(p, p->phi, phi_bytes(p, sizeof(cx_t<T>), R)));
    const LegShape s = leg_shape(p, prec_of<T>(), R);
    AKRA_TRY(legendre_synth<T>(p, s, mode, alm, p->phi.ptr, R, p->d_all_units, p->nunit, st));
    return ring_fft<T>(p, FftMode::Synth, p->phi.ptr, nullptr, map, weighted, R, p->d_all_rings,
                       p->nring, st);
}



template <typename T>
akra_status op_adjoint(akra_plan p, LegMode mode, const void *map, void *alm, bool weighted, int R,
                       cudaStream_t st)
{
    if (is_flat(p)) return flat_op_At<T>(p, map, alm, weighted, R, st);
    const LegShape s = leg_shape(p, prec_of<T>(), R);
    // with weights, rings where W = 0 contribute exactly nothing: transform the active ones only
    const bool act = weighted && p->has_weights;
    const int *units = act ? p->d_active_units : p->d_all_units;
    const int nunits = act ? p->n_active_units : p->nunit;
    const int *rings = act ? p->d_active_rings : p->d_all_rings;
    const int nrings = act ? p->n_active_rings : p->nring;
    AKRA_TRY(ws_reserve(p, p->phi, phi_bytes(p, sizeof(cx_t<T>), R)));
    AKRA_TRY(ws_reserve(p, p->partial, (size_t)legendre_chunks(nunits, s) * R * p->ntri * 4 *
                                           sizeof(T)));
    AKRA_TRY(ring_fft<T>(p, FftMode::Adjoint, p->phi.ptr, map, nullptr, weighted, R, rings, nrings, st));
    int nch = 0;
    AKRA_TRY(legendre_adjoint<T>(p, s, p->phi.ptr, p->partial.ptr, R, units, nunits, &nch, st));
    return adjoint_epilogue<T>(p, mode, p->partial.ptr, nch, nullptr, 0.0, alm, R, st);
}

template <typename T>
akra_status op_H(akra_plan p, const void *x, void *y, int R, cudaStream_t st)
{
    if (is_flat(p)) return flat_op_H<T>(p, x, y, R, st);
    const LegShape s = leg_shape(p, prec_of<T>(), R);
    AKRA_TRY(ws_reserve(p, p->phi, phi_bytes(p, sizeof(cx_t<T>), R)));
    AKRA_TRY(ws_reserve(p, p->partial, (size_t)legendre_chunks(p->n_active_units, s) * R *
                                           p->ntri * 4 * sizeof(T)));
    AKRA_TRY(legendre_synth<T>(p, s, LegMode::KS, x, p->phi.ptr, R, p->d_active_units,
                               p->n_active_units, st));
    AKRA_TRY(ring_fft<T>(p, FftMode::Happly, p->phi.ptr, nullptr, nullptr, true, R,
                         p->d_active_rings, p->n_active_rings, st));
    int nch = 0;
    AKRA_TRY(legendre_adjoint<T>(p, s, p->phi.ptr, p->partial.ptr, R, p->d_active_units,
                                 p->n_active_units, &nch, st));
    return adjoint_epilogue<T>(p, LegMode::KS, p->partial.ptr, nch, x, p->lambda_eff, y, R, st,
                               p->fields);
}

template akra_status op_synth<float>(akra_plan, LegMode, const void *, void *, bool, int, cudaStream_t);
template akra_status op_synth<double>(akra_plan, LegMode, const void *, void *, bool, int, cudaStream_t);
template akra_status op_adjoint<float>(akra_plan, LegMode, const void *, void *, bool, int, cudaStream_t);
template akra_status op_adjoint<double>(akra_plan, LegMode, const void *, void *, bool, int, cudaStream_t);
template akra_status op_H<float>(akra_plan, const void *, void *, int, cudaStream_t);
template akra_status op_H<double>(akra_plan, const void *, void *, int, cudaStream_t);

}  // namespace akra

using namespace akra;

// ---------------------------------------------------------------------------
// C entry points
// ---------------------------------------------------------------------------
extern "C" const char *akra_last_error(void) { return g_err; }

extern "C" const char *akra_version(void) { return "akra-gb300 1.0 (sm_103a)"; }

template <typename P> static akra_status dev_alloc(akra_plan p, P **ptr, size_t bytes)
{
    if (cudaMalloc((void **)ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("plan table allocation of %zu bytes failed", bytes);
        return AKRA_ENOMEM;
    }
    p->bytes_tables += bytes;
    return AKRA_OK;
}

namespace akra { akra_status ring_fft_prepare(akra_plan p); }

static akra_status plan_build(akra_plan p)
{
    const int N = p->nside, L = p->lmax;
    AKRA_TRY(dev_alloc(p, &p->d_rings, sizeof(RingInfo) * p->nring));
    AKRA_TRY(dev_alloc(p, &p->d_units, sizeof(UnitInfo) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_factors, sizeof(FftFactors) * (N + 1)));
    AKRA_TRY(dev_alloc(p, &p->d_coef64, sizeof(double4_32a) * p->ntri));
    AKRA_TRY(dev_alloc(p, &p->d_coef32, sizeof(float4) * p->ntri));
    AKRA_TRY(dev_alloc(p, &p->d_seedC, sizeof(double) * (L + 1)));
    AKRA_TRY(dev_alloc(p, &p->d_D64, sizeof(double) * (L + 1)));
    AKRA_TRY(dev_alloc(p, &p->d_seed32, sizeof(float4) * (size_t)(L + 1) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_dseed32, sizeof(float2) * (size_t)(L + 1) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_seed64, sizeof(double4_32a) * (size_t)(L + 1) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_start32, sizeof(int2) * (size_t)(L + 1) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_start64, sizeof(int2) * (size_t)(L + 1) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_steps, sizeof(unsigned long long) * 2 * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_D32, sizeof(float) * (L + 1)));
    const size_t ntw = 4ull * N * (N + 1);
    AKRA_TRY(dev_alloc(p, &p->d_tw64, sizeof(double2) * ntw));
    AKRA_TRY(dev_alloc(p, &p->d_tw32, sizeof(float2) * ntw));
    AKRA_TRY(dev_alloc(p, &p->d_all_rings, sizeof(int) * p->nring));
    AKRA_TRY(dev_alloc(p, &p->d_all_units, sizeof(int) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_active_rings, sizeof(int) * p->nring));
    AKRA_TRY(dev_alloc(p, &p->d_active_units, sizeof(int) * p->nunit));
    AKRA_TRY(dev_alloc(p, &p->d_ring_active, p->nring));
    AKRA_TRY(dev_alloc(p, &p->d_W64, sizeof(double) * p->npix));
    AKRA_TRY(dev_alloc(p, &p->d_W32, sizeof(float) * p->npix));
    AKRA_TRY(dev_alloc(p, &p->d_W32r, sizeof(float) * p->npix));
    AKRA_TRY(dev_alloc(p, &p->d_pw64, sizeof(double) * p->ntri));
    AKRA_TRY(dev_alloc(p, &p->d_pw32, sizeof(float) * p->ntri));
    AKRA_TRY(dev_alloc(p, &p->d_tc_err, sizeof(int)));
    AKRA_CUDA_TRY(cudaMemset(p->d_tc_err, 0, sizeof(int)));

    std::vector<FftFactors> fac(N + 1);
    std::vector<double2> blue;
    std::map<int, long long> blue_at;   // prime -> table offset
    for (int i = 1; i <= N; i++) {
        fac[i] = factorize(4 * i);
        const int bp = fac[i].blue_p;
        if (!bp) continue;
        auto it = blue_at.find(bp);
        if (it == blue_at.end()) {
            it = blue_at.emplace(bp, (long long)blue.size()).first;
            blue_tables(bp, fac[i].blue_M, blue);
        }
        fac[i].blue_off = it->second;
    }
    AKRA_CUDA_TRY(cudaMemcpy(p->d_factors, fac.data(), sizeof(FftFactors) * (N + 1),
                             cudaMemcpyHostToDevice));
    if (!blue.empty()) {
        AKRA_TRY(dev_alloc(p, &p->d_blue64, sizeof(double2) * blue.size()));
        AKRA_CUDA_TRY(cudaMemcpy(p->d_blue64, blue.data(), sizeof(double2) * blue.size(),
                                 cudaMemcpyHostToDevice));
    }
    const int nthr = 256;
    k_geometry<<<(p->nring + nthr - 1) / nthr, nthr>>>(N, p->d_rings, p->d_units);
    AKRA_CUDA_TRY(cudaGetLastError());
    k_coef<<<(L + 1 + 127) / 128, 128>>>(L, p->d_coef64, p->d_coef32);
    AKRA_CUDA_TRY(cudaGetLastError());
    k_seed<<<(L + 1 + 127) / 128, 128>>>(L, p->d_seedC, p->d_D64, p->d_D32);
    AKRA_CUDA_TRY(cudaGetLastError());
    AKRA_CUDA_TRY(cudaMemset(p->d_steps, 0, sizeof(unsigned long long) * 2 * p->nunit));
    k_start_states<<<dim3((p->nunit + 127) / 128, L + 1), 128>>>(
        L, p->nunit, p->d_seedC, p->d_units, p->d_coef64, p->d_seed32, p->d_seed64, p->d_start32,
        p->d_start64, p->d_steps, p->d_dseed32);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->steps32.assign(p->nunit, 0);
    p->steps64.assign(p->nunit, 0);
    AKRA_CUDA_TRY(cudaMemcpy(p->steps32.data(), p->d_steps, sizeof(unsigned long long) * p->nunit,
                             cudaMemcpyDeviceToHost));
    AKRA_CUDA_TRY(cudaMemcpy(p->steps64.data(), p->d_steps + p->nunit,
                             sizeof(unsigned long long) * p->nunit, cudaMemcpyDeviceToHost));
    k_twiddles<<<dim3(4, N), 256>>>(N, p->d_tw64, p->d_tw32);
    AKRA_CUDA_TRY(cudaGetLastError());
    k_iota<<<(p->nring + 255) / 256, 256>>>(p->nring, p->d_all_rings);
    k_iota<<<(p->nunit + 255) / 256, 256>>>(p->nunit, p->d_all_units);
    AKRA_CUDA_TRY(cudaGetLastError());
    AKRA_CUDA_TRY(cudaMemset(p->d_ring_active, 1, p->nring));
    AKRA_TRY(ring_fft_prepare(p));
    AKRA_TRY(ring_fft32_build(p));
    AKRA_TRY(legendre_tc_prepare());
    {
        // 16-step l-tiles of every m (from l0 = max(m, 2)), the tensor-core synthesis' B operand grid
        std::vector<long long> tb(L + 1);
        long long acc = 0;
        for (int m = 0; m <= L; m++) {
            tb[m] = acc;
            acc += (L - std::max(m, 2)) / 16 + 1;
        }
        p->tc_tiles = acc;
        AKRA_TRY(dev_alloc(p, &p->d_tc_tilebase, sizeof(long long) * (L + 1)));
        AKRA_CUDA_TRY(cudaMemcpy(p->d_tc_tilebase, tb.data(), sizeof(long long) * (L + 1), cudaMemcpyHostToDevice));
    }
    AKRA_CUDA_TRY(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
    AKRA_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_a, cudaEventDisableTiming));
    AKRA_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_b, cudaEventDisableTiming));
    AKRA_CUDA_TRY(cudaDeviceSynchronize());
    return AKRA_OK;
}

extern "C" akra_status akra_plan_create(int nside, int lmax, akra_plan *out)
{
    if (!out) {
        set_error("akra_plan_create: out is NULL");
        return AKRA_EINVAL;
    }
    *out = nullptr;
    if (nside < 1 || nside > kMaxNside) {
        set_error("akra_plan_create: nside %d outside [1, %d]", nside, kMaxNside);
        return AKRA_EINVAL;
    }
    if (lmax < 2 || lmax > 4 * nside) {
        set_error("akra_plan_create: lmax %d outside [2, 4 nside = %d]", lmax, 4 * nside);
        return AKRA_EINVAL;
    }
    akra_plan p = new (std::nothrow) akra_plan_s();
    if (!p) {
        set_error("akra_plan_create: host allocation failed");
        return AKRA_ENOMEM;
    }
    p->nside = nside;
    p->lmax = lmax;
    p->nring = 4 * nside - 1;
    p->nunit = 2 * nside;
    p->npix = 12LL * nside * nside;
    p->ntri = (long long)(lmax + 1) * (lmax + 2) / 2;
    p->omega = 4.0 * 3.14159265358979323846 / (double)p->npix;
    cudaGetDevice(&p->device);
    akra_status s = plan_build(p);
    if (s != AKRA_OK) {
        akra_plan_destroy(p);
        return s;
    }
    *out = p;
    return AKRA_OK;
}



extern "C" void akra_plan_destroy(akra_plan p)
{
    if (!p) return;
    cudaDeviceSynchronize();
    cg_release_graphs(p);
    void *ptrs[] = {p->d_rings, p->d_units, p->d_factors, p->d_coef64, p->d_coef32, p->d_seedC,
                    p->d_D64, p->d_D32, p->d_tw64, p->d_tw32, p->d_all_rings, p->d_all_units,
                    p->d_active_rings, p->d_active_units, p->d_ring_active, p->d_W64, p->d_W32,
                    p->d_W32r, p->phi.ptr, p->partial.ptr, p->cg.ptr, p->red.ptr, p->xsave.ptr, p->red_cl.ptr,
                    p->d_fft32_M,
                    p->d_fft32_off, p->d_fft32_tw2, p->d_fft32_bhat, p->d_seed32, p->d_seed64,
                    p->d_start32, p->d_start64, p->d_steps, p->d_pw64, p->d_pw32, p->d_ftw64,
                    p->d_ftw32, p->d_fWt64, p->d_fWt32,
                    p->d_fft32_rings_all, p->d_fft32_rings_act, p->d_tc_err, p->d_dseed32, p->d_blue64,
                    p->bpre.ptr, p->d_tc_tilebase};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (p->stream) cudaStreamDestroy(p->stream);
    if (p->ev_a) cudaEventDestroy(p->ev_a);
    if (p->ev_b) cudaEventDestroy(p->ev_b);
    delete p;
}

extern "C" akra_status akra_debug_violations(long long *count, int *site, long long *index,
                                             long long *bound)
{
    if (!count) {
        set_error("akra_debug_violations: NULL count");
        return AKRA_EINVAL;
    }
#ifdef AKRA_DEBUG
    DebugRecord acc{};
    AKRA_CUDA_TRY(cudaDeviceSynchronize());
    AKRA_TRY(debug_collect_legendre(&acc));
    AKRA_TRY(debug_collect_legendre_tc(&acc));
    AKRA_TRY(debug_collect_batch(&acc));
    AKRA_TRY(debug_collect_ringfft(&acc));
    AKRA_TRY(debug_collect_ringfft32(&acc));
    *count = (long long)acc.count;
    if (site) *site = acc.site;
    if (index) *index = acc.index;
    if (bound) *bound = acc.bound;
#else
    *count = -1;   // release build: no checks compiled in
    if (site) *site = 0;
    if (index) *index = 0;
    if (bound) *bound = 0;
#endif
    return AKRA_OK;
}

extern "C" akra_status akra_plan_fill_workspaces(akra_plan p, int byte, void *stream)
{
    if (!p || byte < 0 || byte > 255) {
        set_error("akra_plan_fill_workspaces: NULL plan or byte outside [0, 255]");
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    akra::Workspace *ws[] = {&p->phi, &p->partial, &p->cg, &p->red, &p->xsave, &p->red_cl, &p->bpre};
    for (akra::Workspace *w : ws)
        if (w->ptr && w->bytes) AKRA_CUDA_TRY(cudaMemsetAsync(w->ptr, byte, w->bytes, st));
    return AKRA_OK;
}

extern "C" akra_status akra_plan_describe(akra_plan p, akra_plan_desc *out)
{
    if (!p || !out) {
        set_error("akra_plan_describe: NULL argument");
        return AKRA_EINVAL;
    }
    out->nside = p->nside;
    out->lmax = p->lmax;
    out->nring = p->nring;
    out->nunit = p->nunit;
    out->npix = p->npix;
    out->ntri = p->ntri;
    out->has_weights = p->has_weights ? 1 : 0;
    out->n_active_rings = p->n_active_rings;
    out->n_active_units = p->n_active_units;
    out->lambda = p->lambda;
    out->lambda_eff = p->lambda_eff;
    out->precond = p->precond;
    out->omega = p->omega;
    out->device_bytes = plan_device_bytes(p);
    out->kernel_launches = p->launches;
    long long s32 = 0, s64 = 0, o32 = 0, o64 = 0;
    if (p->has_weights) {
        for (size_t k = 0; k < p->h_active_units.size(); k++) {
            const int u = p->h_active_units[k];
            s32 += (long long)p->steps32[u];
            s64 += (long long)p->steps64[u];
            if (p->h_unit_one_ring[k]) {
                o32 += (long long)p->steps32[u];
                o64 += (long long)p->steps64[u];
            }
        }
    } else {
        for (int u = 0; u < p->nunit; u++) {
            s32 += (long long)p->steps32[u];
            s64 += (long long)p->steps64[u];
        }
    }
    out->legendre_steps_f32 = s32;
    out->legendre_steps_f64 = s64;
    out->legendre_steps_f32_one_ring = o32;
    out->legendre_steps_f64_one_ring = o64;
    return AKRA_OK;
}

extern "C" akra_status akra_plan_set_weights(akra_plan p, const double *d_ninv, double lambda,
                                             void *stream)
{
    if (!p || !d_ninv || !(lambda >= 0) || !std::isfinite(lambda)) {
        set_error("akra_plan_set_weights: NULL plan/ninv or invalid lambda");
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (is_flat(p)) return flat_set_weights(p, d_ninv, lambda, st);
    const int nr = p->nring;
    double *d_stats = nullptr;
    if (cudaMalloc(&d_stats, sizeof(double) * 3 * nr) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_plan_set_weights: scratch allocation failed");
        return AKRA_ENOMEM;
    }
    k_weights<<<nr, 256, 0, st>>>(p->d_rings, d_ninv, p->omega, p->d_W64, p->d_W32, p->d_W32r, d_stats,
                                  d_stats + nr, d_stats + 2 * nr);
    std::vector<double> h(3 * (size_t)nr);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaMemcpyAsync(h.data(), d_stats, sizeof(double) * 3 * nr,
                                     cudaMemcpyDeviceToHost, st);
    cudaError_t e3 = cudaStreamSynchronize(st);
    cudaFree(d_stats);
    if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
        set_error("akra_plan_set_weights: CUDA failure %s",
                  cudaGetErrorString(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3));
        return AKRA_ECUDA;
    }
    double sum = 0, cnt = 0, bad = 0;
    std::vector<unsigned char> active(nr);
    std::vector<int> rings;
    for (int r = 0; r < nr; r++) {
        sum += h[r];
        cnt += h[nr + r];
        bad += h[2 * nr + r];
        active[r] = h[nr + r] > 0 ? 1 : 0;
        if (active[r]) rings.push_back(r);
    }
    if (bad > 0) {
        set_error("akra_plan_set_weights: %.0f negative or non-finite N^-1 entries", bad);
        return AKRA_EINVAL;
    }
    std::vector<int> units;
    std::vector<unsigned char> one_ring;
    const int N = p->nside;
    int one = -1;   // the common single ring side of the active units (-1: none yet, 0: mixed)
    for (int u = 0; u < p->nunit; u++) {
        const int rn = u, rs = (u + 1 < 2 * N) ? 4 * N - (u + 1) - 1 : -1;
        const bool an = active[rn] != 0, as = rs >= 0 && active[rs] != 0;
        if (an || as) {
            units.push_back(u);
            one_ring.push_back(an && as ? 0 : 1);
            const int side = an && as ? 0 : an ? 1 : 2;
            one = one < 0 ? side : (one == side ? one : 0);
        }
    }
    p->one_side = one > 0 ? one : 0;
    AKRA_CUDA_TRY(cudaMemcpy(p->d_ring_active, active.data(), nr, cudaMemcpyHostToDevice));
    if (!rings.empty())
        AKRA_CUDA_TRY(cudaMemcpy(p->d_active_rings, rings.data(), sizeof(int) * rings.size(),
                                 cudaMemcpyHostToDevice));
    if (!units.empty())
        AKRA_CUDA_TRY(cudaMemcpy(p->d_active_units, units.data(), sizeof(int) * units.size(),
                                 cudaMemcpyHostToDevice));
    p->n_active_rings = (int)rings.size();
    p->n_active_units = (int)units.size();
    p->h_active_units = units;
    p->h_unit_one_ring = one_ring;
    p->lambda = lambda;
    p->lambda_eff = cnt > 0 ? lambda * sum / cnt : 0.0;
    p->precond = 1.0 / (sum / (double)p->npix + p->lambda_eff);
    if (!std::isfinite(p->precond)) p->precond = 1.0;
    k_pw<<<p->lmax + 1, 128, 0, st>>>(p->lmax, p->d_D64, sum / (double)p->npix, p->lambda_eff, p->d_pw64,
                                      p->d_pw32);
    AKRA_CUDA_TRY(cudaGetLastError());
    AKRA_CUDA_TRY(cudaStreamSynchronize(st));
    p->has_weights = true;
    p->ws_gen++;   // captured CG iterations hold the previous active lists and λ_eff
    return ring_fft32_order(p, rings, p->d_fft32_rings_act, &p->fft32_nsmall_act);
}

static akra_status check_common(akra_plan p, akra_prec prec, const void *a, const void *b, int R,
                                const char *who)
{
    if (!p || !a || !b) {
        set_error("%s: NULL plan or array", who);
        return AKRA_EINVAL;
    }
    if (prec != AKRA_F64 && prec != AKRA_F32) {
        set_error("%s: precision must be AKRA_F64 or AKRA_F32", who);
        return AKRA_EINVAL;
    }
    if (R < 1 || R > 65535) {
        set_error("%s: R = %d outside [1, 65535]", who, R);
        return AKRA_EINVAL;
    }
    return AKRA_OK;
}

extern "C" akra_status akra_synth_spin2(akra_plan p, akra_prec prec, const void *d_alm,
                                        void *d_map, int R, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_synth_spin2"));
    AKRA_TRY(check_common(p, prec, d_alm, d_map, R, "akra_synth_spin2"));
    cudaStream_t st = (cudaStream_t)stream;
    return prec == AKRA_F64 ? op_synth<double>(p, LegMode::Synth, d_alm, d_map, false, R, st)
                            : op_synth<float>(p, LegMode::Synth, d_alm, d_map, false, R, st);
}

extern "C" akra_status akra_adjoint_synth_spin2(akra_plan p, akra_prec prec, const void *d_map,
                                                void *d_alm, int R, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_adjoint_synth_spin2"));
    AKRA_TRY(check_common(p, prec, d_map, d_alm, R, "akra_adjoint_synth_spin2"));
    cudaStream_t st = (cudaStream_t)stream;
    return prec == AKRA_F64 ? op_adjoint<double>(p, LegMode::Synth, d_map, d_alm, false, R, st)
                            : op_adjoint<float>(p, LegMode::Synth, d_map, d_alm, false, R, st);
}

extern "C" akra_status akra_apply_A(akra_plan p, akra_prec prec, const void *d_x, void *d_map,
                                    int weighted, int R, void *stream)
{
    AKRA_TRY(check_common(p, prec, d_x, d_map, R, "akra_apply_A"));
    if (weighted && !p->has_weights) {
        set_error("akra_apply_A: weighted operator before akra_plan_set_weights");
        return AKRA_ENOWEIGHTS;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return prec == AKRA_F64 ? op_synth<double>(p, LegMode::KS, d_x, d_map, weighted != 0, R, st)
                            : op_synth<float>(p, LegMode::KS, d_x, d_map, weighted != 0, R, st);
}

extern "C" akra_status akra_apply_At(akra_plan p, akra_prec prec, const void *d_map, void *d_x,
                                     int weighted, int R, void *stream)
{
    AKRA_TRY(check_common(p, prec, d_map, d_x, R, "akra_apply_At"));
    if (weighted && !p->has_weights) {
        set_error("akra_apply_At: weighted operator before akra_plan_set_weights");
        return AKRA_ENOWEIGHTS;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return prec == AKRA_F64 ? op_adjoint<double>(p, LegMode::KS, d_map, d_x, weighted != 0, R, st)
                            : op_adjoint<float>(p, LegMode::KS, d_map, d_x, weighted != 0, R, st);
}

extern "C" akra_status akra_apply_H(akra_plan p, akra_prec prec, const void *d_x, void *d_y, int R,
                                    void *stream)
{
    AKRA_TRY(check_common(p, prec, d_x, d_y, R, "akra_apply_H"));
    if (!p->has_weights) {
        set_error("akra_apply_H: called before akra_plan_set_weights");
        return AKRA_ENOWEIGHTS;
    }
    if (d_x == d_y) {
        set_error("akra_apply_H: d_x and d_y must not overlap");
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    return prec == AKRA_F64 ? op_H<double>(p, d_x, d_y, R, st) : op_H<float>(p, d_x, d_y, R, st);
}

// ---------------------------------------------------------------------------
// autotuner: time every compiled Legendre tile shape over the units the operator will use,
// the synthesis and the adjoint separately, and keep for this (precision, R) the RHS grouping
// whose fastest synthesis + fastest adjoint is smallest
// ---------------------------------------------------------------------------
template <typename T>
static akra_status tune_one(akra_plan p, akra_prec prec, int R, cudaStream_t st)
{
    std::vector<LegShape> cands;
    if (R >= 4) cands.push_back({1, 128, 4});
    if (R >= 2) {
        cands.push_back({2, 128, 2});
        cands.push_back({1, 128, 2});
    }
    if (std::is_same<T, float>::value)
        for (int pp : {8, 6, 5, 3}) cands.push_back({pp, 128, 1});
    cands.push_back({4, 128, 1});
    cands.push_back({2, 128, 1});
    cands.push_back({1, 128, 1});
    const int *units = p->has_weights ? p->d_active_units : p->d_all_units;
    const int nunits = p->has_weights ? p->n_active_units : p->nunit;
    if (nunits == 0) return AKRA_OK;
    size_t max_part = 0;
    for (auto &c : cands)
        max_part = std::max(max_part, (size_t)legendre_chunks(nunits, c) * (size_t)R * (size_t)p->ntri * 4 * sizeof(T));
    AKRA_TRY(ws_reserve(p, p->phi, (size_t)R * p->nring * (2 * (size_t)p->lmax + 1) * sizeof(cx_t<T>)));
    AKRA_TRY(ws_reserve(p, p->partial, max_part));
    void *alm = nullptr;
    const size_t abytes = (size_t)R * 2 * p->ntri * sizeof(cx_t<T>);
    if (cudaMalloc(&alm, abytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_autotune: scratch allocation failed");
        return AKRA_ENOMEM;
    }
    cudaMemsetAsync(alm, 0, abytes, st);
    cudaMemsetAsync(p->phi.ptr, 0, p->phi.bytes, st);
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    std::vector<float> ts(cands.size(), 0.f), ta(cands.size(), 0.f);
    akra_status s = AKRA_OK;
    for (size_t k = 0; k < cands.size() && s == AKRA_OK; k++) {
        const LegShape &c = cands[k];
        for (int rep = 0; rep < 3 && s == AKRA_OK; rep++) {
            int nch = 0;
            cudaEventRecord(e0, st);
            s = legendre_synth<T>(p, c, LegMode::KS, alm, p->phi.ptr, R, units, nunits, st);
            cudaEventRecord(e1, st);
            if (s == AKRA_OK) s = legendre_adjoint<T>(p, c, p->phi.ptr, p->partial.ptr, R, units, nunits, &nch, st);
            cudaEventRecord(e2, st);
            cudaEventSynchronize(e2);
            float m1 = 0, m2 = 0;
            cudaEventElapsedTime(&m1, e0, e1);
            cudaEventElapsedTime(&m2, e1, e2);
            if (rep > 0) {   // the first run is a warm-up
                ts[k] += m1;
                ta[k] += m2;
            }
        }
    }
    // FP32: the tensor-core synthesis for every RHS group that R fills at least half
    std::vector<int> tcs;
    if (std::is_same<T, float>::value)
        for (int g : {4, 8, 16, 32})
            if (g == 4 || R > g / 2) tcs.push_back(g);
    std::vector<float> ttc(tcs.size(), 0.f);
    for (size_t q = 0; q < tcs.size() && s == AKRA_OK; q++) {
        for (int rep = 0; rep < 3 && s == AKRA_OK; rep++) {
            cudaEventRecord(e0, st);
            s = legendre_synth_tc(p, tcs[q], LegMode::KS, alm, p->phi.ptr, R, units, nunits, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float m1 = 0;
            cudaEventElapsedTime(&m1, e0, e1);
            if (rep > 0) ttc[q] += m1;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaFree(alm);
    if (s != AKRA_OK) return s;
    AKRA_TRY(tc_error_check(p));
    LegShape pick = cands.back();
    float best = 1e30f;
    for (size_t j = 0; j < cands.size(); j++) {      // adjoint shape j (its own RHS group) ...
        for (size_t k = 0; k < cands.size(); k++) {  // ... with a CUDA-core synthesis shape k
            if (ts[k] + ta[j] >= best) continue;
            best = ts[k] + ta[j];
            pick = LegShape{cands[k].P, cands[k].NT, cands[k].RG, cands[j].P, 0, cands[j].RG};
        }
        for (size_t q = 0; q < tcs.size(); q++) {    // ... or with the tensor-core synthesis
            if (ttc[q] + ta[j] >= best) continue;
            best = ttc[q] + ta[j];
            pick = LegShape{cands[j].P, cands[j].NT, cands[j].RG, cands[j].P, tcs[q], cands[j].RG};
        }
    }
    p->shapes[(long long)prec * 1000 + (R > 999 ? 999 : R)] = pick;
    p->ws_gen++;   // captured CG iterations used the previous shape
    return AKRA_OK;
}

static bool shape_compiled(akra_prec prec, int P, int RG)
{
    if (RG == 1) return P == 1 || P == 2 || P == 4 || (prec == AKRA_F32 && (P == 3 || P == 5 || P == 6 || P == 8));
    if (RG == 2) return P == 1 || P == 2;
    return RG == 4 && P == 1;
}

extern "C" akra_status akra_plan_get_shape(akra_plan p, akra_prec prec, int R, int *P, int *PA,
                                           int *RG)
{
    AKRA_TRY(reject_flat(p, "akra_plan_get_shape"));
    if (!p || !P || !PA || !RG || R < 1 || (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_plan_get_shape: invalid argument");
        return AKRA_EINVAL;
    }
    const LegShape s = leg_shape(p, prec, R);
    *P = s.P;
    *PA = s.adjP();
    *RG = s.RG;
    return AKRA_OK;
}

extern "C" akra_status akra_plan_set_preconditioner(akra_plan p, akra_precond kind)
{
    AKRA_TRY(reject_flat(p, "akra_plan_set_preconditioner"));
    if (!p || (kind != AKRA_PRECOND_SCALAR && kind != AKRA_PRECOND_PER_L)) {
        set_error("akra_plan_set_preconditioner: invalid argument");
        return AKRA_EINVAL;
    }
    p->precond_kind = kind == AKRA_PRECOND_PER_L ? 1 : 0;
    p->ws_gen++;   // captured CG iterations hold the previous weights
    return AKRA_OK;
}

extern "C" akra_status akra_plan_set_shape(akra_plan p, akra_prec prec, int R, int P, int PA, int RG)
{
    AKRA_TRY(reject_flat(p, "akra_plan_set_shape"));
    if (!p || R < 1 || R > 65535 || (prec != AKRA_F64 && prec != AKRA_F32) ||
        !shape_compiled(prec, P, RG) || !shape_compiled(prec, PA, RG)) {
        set_error("akra_plan_set_shape: invalid argument or no compiled kernel for P=%d PA=%d RG=%d",
                  P, PA, RG);
        return AKRA_EINVAL;
    }
    p->shapes[(long long)prec * 1000 + (R > 999 ? 999 : R)] = LegShape{P, 128, RG, PA};
    p->ws_gen++;   // captured CG iterations used the previous shape
    return AKRA_OK;
}

extern "C" akra_status akra_plan_set_adjoint_shape(akra_plan p, akra_prec prec, int R, int PA, int RGA)
{
    AKRA_TRY(reject_flat(p, "akra_plan_set_adjoint_shape"));
    if (!p || R < 1 || R > 65535 || (prec != AKRA_F64 && prec != AKRA_F32) || !shape_compiled(prec, PA, RGA)) {
        set_error("akra_plan_set_adjoint_shape: invalid argument or no compiled adjoint for P=%d RG=%d", PA, RGA);
        return AKRA_EINVAL;
    }
    LegShape s = leg_shape(p, prec, R);
    s.PA = PA;
    s.RGA = RGA;
    p->shapes[(long long)prec * 1000 + (R > 999 ? 999 : R)] = s;
    p->ws_gen++;   // captured CG iterations used the previous shape
    return AKRA_OK;
}

extern "C" akra_status akra_plan_get_adjoint_shape(akra_plan p, akra_prec prec, int R, int *PA, int *RGA)
{
    AKRA_TRY(reject_flat(p, "akra_plan_get_adjoint_shape"));
    if (!p || !PA || !RGA || R < 1 || (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_plan_get_adjoint_shape: invalid argument");
        return AKRA_EINVAL;
    }
    const LegShape s = leg_shape(p, prec, R);
    *PA = s.adjP();
    *RGA = s.adjRG();
    return AKRA_OK;
}

extern "C" akra_status akra_plan_set_tc_synthesis(akra_plan p, int R, int group)
{
    AKRA_TRY(reject_flat(p, "akra_plan_set_tc_synthesis"));
    if (!p || R < 1 || R > 65535 || !(group == 0 || group == 4 || group == 8 || group == 16 || group == 32)) {
        set_error("akra_plan_set_tc_synthesis: invalid argument (group must be 0, 4, 8, 16 or 32)");
        return AKRA_EINVAL;
    }
    LegShape s = leg_shape(p, AKRA_F32, R);
    s.TC = group;
    p->shapes[(long long)AKRA_F32 * 1000 + (R > 999 ? 999 : R)] = s;
    p->ws_gen++;   // captured CG iterations used the previous shape
    return AKRA_OK;
}

extern "C" akra_status akra_plan_get_tc_synthesis(akra_plan p, int R, int *group)
{
    AKRA_TRY(reject_flat(p, "akra_plan_get_tc_synthesis"));
    if (!p || !group || R < 1) {
        set_error("akra_plan_get_tc_synthesis: invalid argument");
        return AKRA_EINVAL;
    }
    *group = leg_shape(p, AKRA_F32, R).TC;
    return AKRA_OK;
}

extern "C" akra_status akra_autotune(akra_plan p, akra_prec prec, int R, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_autotune"));
    if (!p || R < 1 || R > 65535 || (prec != AKRA_F64 && prec != AKRA_F32 && prec != AKRA_MIXED)) {
        set_error("akra_autotune: invalid argument");
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (prec == AKRA_F64 || prec == AKRA_MIXED) AKRA_TRY(tune_one<double>(p, AKRA_F64, R, st));
    if (prec == AKRA_F32 || prec == AKRA_MIXED) AKRA_TRY(tune_one<float>(p, AKRA_F32, R, st));
    return AKRA_OK;
}

// ---------------------------------------------------------------------------
// stage timing of one H application (diagnostics for the roofline report)
// ---------------------------------------------------------------------------
template <typename T>
static akra_status time_stages(akra_plan p, int R, int reps, cudaStream_t st, double *ms)
{
    const akra_prec prec = prec_of<T>();
    const LegShape s = leg_shape(p, prec, R);
    const int nch = legendre_chunks(p->n_active_units, s);
    AKRA_TRY(ws_reserve(p, p->phi, phi_bytes(p, sizeof(cx_t<T>), R)));
    AKRA_TRY(ws_reserve(p, p->partial, (size_t)nch * R * p->ntri * 4 * sizeof(T)));
    void *x = nullptr, *y = nullptr;
    const size_t ab = (size_t)R * 2 * p->ntri * sizeof(cx_t<T>);
    if (cudaMalloc(&x, ab) != cudaSuccess || cudaMalloc(&y, ab) != cudaSuccess) {
        cudaGetLastError();
        if (x) cudaFree(x);
        set_error("akra_time_H_stages: scratch allocation failed");
        return AKRA_ENOMEM;
    }
    cudaMemsetAsync(x, 0, ab, st);
    cudaEvent_t ev[5];
    for (auto &e : ev) cudaEventCreate(&e);
    double acc[5] = {0, 0, 0, 0, 0};
    akra_status s1 = AKRA_OK;
    for (int rep = 0; rep <= reps && s1 == AKRA_OK; rep++) {
        int n2 = 0;
        cudaEventRecord(ev[0], st);
        s1 = legendre_synth<T>(p, s, LegMode::KS, x, p->phi.ptr, R, p->d_active_units, p->n_active_units, st);
        cudaEventRecord(ev[1], st);
        if (s1 == AKRA_OK)
            s1 = ring_fft<T>(p, FftMode::Happly, p->phi.ptr, nullptr, nullptr, true, R, p->d_active_rings,
                             p->n_active_rings, st);
        cudaEventRecord(ev[2], st);
        if (s1 == AKRA_OK)
            s1 = legendre_adjoint<T>(p, s, p->phi.ptr, p->partial.ptr, R, p->d_active_units,
                                     p->n_active_units, &n2, st);
        cudaEventRecord(ev[3], st);
        if (s1 == AKRA_OK) s1 = adjoint_epilogue<T>(p, LegMode::KS, p->partial.ptr, n2, x, p->lambda_eff, y, R, st);
        cudaEventRecord(ev[4], st);
        cudaEventSynchronize(ev[4]);
        if (rep == 0) continue;   // warm-up
        for (int k = 0; k < 4; k++) {
            float t = 0;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            acc[k] += t;
        }
        float t = 0;
        cudaEventElapsedTime(&t, ev[0], ev[4]);
        acc[4] += t;
    }
    for (auto &e : ev) cudaEventDestroy(e);
    cudaFree(x);
    cudaFree(y);
    if (s1 != AKRA_OK) return s1;
    AKRA_CUDA_TRY(cudaGetLastError());
    for (int k = 0; k < 5; k++) ms[k] = acc[k] / reps;
    return AKRA_OK;
}

extern "C" akra_status akra_time_H_stages(akra_plan p, akra_prec prec, int R, int reps, void *stream,
                                          double *ms_out)
{
    AKRA_TRY(reject_flat(p, "akra_time_H_stages"));
    if (!p || !ms_out || reps < 1 || R < 1 || (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_time_H_stages: invalid argument");
        return AKRA_EINVAL;
    }
    if (!p->has_weights) {
        set_error("akra_time_H_stages: called before akra_plan_set_weights");
        return AKRA_ENOWEIGHTS;
    }
    cudaStream_t st = (cudaStream_t)stream;
    AKRA_TRY(prec == AKRA_F64 ? time_stages<double>(p, R, reps, st, ms_out)
                              : time_stages<float>(p, R, reps, st, ms_out));
    return tc_error_check(p);
}
