// akra_ringfft.cu -- per-ring phase sums of the spin-2 synthesis and of its transpose
// (the φ half of SHT^-1 / SHT in Sec. II B), fused with the pixel-space diagonal
// W = ω M N^-1 (Sec. II B, "Pixel space (diagonal)").
//
// (This Stockham form serves the FP64 path; FP32 uses akra_ringfft32.cu.)
// Ring with n pixels at φ_j = π(2j+σ)/n.  Synthesis direction:
//   f_j = Σ_{m=-L}^{L} Φ(m) e^{imφ_j} = Σ_k e^{2πijk/n} F[k],
//   F[k] = e^{iπσk/n} Σ_{q: |k+nq|<=L} (-1)^{σq} Φ(k+nq)          (fold)
// Transpose direction (w_j = W_j f_j or the caller's map):
//   Φ'(m) = Σ_j w_j e^{-imφ_j} = e^{-iπσk/n} (-1)^{σq} Σ_j w_j e^{-2πijk/n},  m = k + nq.
// The length-n DFTs run in shared memory, one CTA per ring: a mixed-radix Stockham
// autosort with radices 4 and 2 as register butterflies and every odd prime factor below 67
// as a direct (output-oriented) pass; every pass reads all its inputs into registers,
// synchronises, then writes in place.  A prime factor p >= 67 (polar rings n = 4i with such a
// p in i) is the last pass, Bluestein's chirp-z form: each of its n/p length-p transforms reads
// and writes only the positions j + Ns r of the ring, and is a cyclic convolution of
// power-of-two length M >= 2p - 1 done with two length-M FFTs in a shared-memory scratch
// (O(p log p) instead of the direct pass's O(p^2)).  Twiddles come from the plan's per-length
// table e^{iπt/n}, t < 2n (the length-M ones from the table of the ring length M).
#include "akra_internal.cuh"

namespace akra {

constexpr int FFT_NT = 512;
constexpr int FFT_NMAX = 4 * kMaxNside;

template <typename T>
__device__ __forceinline__ cx_t<T> cmul(cx_t<T> a, cx_t<T> b)
{
    return cx_t<T>{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}

template <typename T, int DIR>
__device__ __forceinline__ cx_t<T> twid(const cx_t<T> *__restrict__ tw, int t)
{
    cx_t<T> w = tw[t];
    if (DIR < 0) w.y = -w.y;
    return w;
}

// R-point DFT in registers (R = 2, 4): out[r] = Σ_q v[q] e^{DIR 2πi qr/R}
template <typename T, int R, int DIR>
__device__ __forceinline__ void dft_small(cx_t<T> (&v)[R])
{
    using C2 = cx_t<T>;
    if constexpr (R == 2) {
        const C2 a = v[0], b = v[1];
        v[0] = C2{a.x + b.x, a.y + b.y};
        v[1] = C2{a.x - b.x, a.y - b.y};
    } else if constexpr (R == 4) {
        const C2 t0{v[0].x + v[2].x, v[0].y + v[2].y};
        const C2 t1{v[0].x - v[2].x, v[0].y - v[2].y};
        const C2 t2{v[1].x + v[3].x, v[1].y + v[3].y};
        const C2 d{v[1].x - v[3].x, v[1].y - v[3].y};
        const C2 t3 = DIR > 0 ? C2{-d.y, d.x} : C2{d.y, -d.x};   // DIR·i·d
        v[0] = C2{t0.x + t2.x, t0.y + t2.y};
        v[2] = C2{t0.x - t2.x, t0.y - t2.y};
        v[1] = C2{t1.x + t3.x, t1.y + t3.y};
        v[3] = C2{t1.x - t3.x, t1.y - t3.y};
    }
}

template <typename T, int R, int DIR>
__device__ void pass_small(cx_t<T> *data, int n, int Ns, const cx_t<T> *__restrict__ tw)
{
    constexpr int MB = (FFT_NMAX / R + FFT_NT - 1) / FFT_NT;
    cx_t<T> v[MB][R];
    const int nb = n / R;
    const int twstep = (2 * n) / (Ns * R);
#pragma unroll
    for (int b = 0; b < MB; b++) {
        const int j = threadIdx.x + b * FFT_NT;
        if (j < nb) {
            const int k = j % Ns;
#pragma unroll
            for (int q = 0; q < R; q++) v[b][q] = data[j + q * nb];
            if (Ns > 1) {
#pragma unroll
                for (int q = 1; q < R; q++) v[b][q] = cmul<T>(v[b][q], twid<T, DIR>(tw, twstep * q * k));
            }
            dft_small<T, R, DIR>(v[b]);
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MB; b++) {
        const int j = threadIdx.x + b * FFT_NT;
        if (j < nb) {
            const int k = j % Ns;
            const int base = (j / Ns) * Ns * R + k;
#pragma unroll
            for (int q = 0; q < R; q++) data[base + q * Ns] = v[b][q];
        }
    }
    __syncthreads();
}

// direct pass for an odd prime radix p (3, 5, 7 and larger): y[(j/Ns)Ns p + k + r Ns] = Σ_q x[j + q n/p] w_{Ns p}^{q(k + Ns r)}
template <typename T, int DIR>
__device__ void pass_generic(cx_t<T> *data, int n, int Ns, int p, const cx_t<T> *__restrict__ tw)
{
    constexpr int MO = (FFT_NMAX + FFT_NT - 1) / FFT_NT;
    cx_t<T> out[MO];
    const int NsP = Ns * p, nb = n / p, twstep = (2 * n) / NsP;
#pragma unroll
    for (int b = 0; b < MO; b++) {
        const int o = threadIdx.x + b * FFT_NT;
        if (o < n) {
            const int g = o / NsP, rem = o - g * NsP, rr = rem / Ns, k = rem - rr * Ns;
            const int j = g * Ns + k, step = k + Ns * rr;
            cx_t<T> acc{0, 0};
            int ex = 0;
            for (int q = 0; q < p; q++) {
                const cx_t<T> t = cmul<T>(data[j + q * nb], twid<T, DIR>(tw, twstep * ex));
                acc.x += t.x;
                acc.y += t.y;
                ex += step;
                if (ex >= NsP) ex -= NsP;
            }
            out[b] = acc;
        }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < MO; b++) {
        const int o = threadIdx.x + b * FFT_NT;
        if (o < n) data[o] = out[b];
    }
    __syncthreads();
}

// power-of-two length M in shared memory (radix 4 passes and a 2), twiddles of length M
template <typename T, int DIR>
__device__ void fft_pow2(cx_t<T> *data, int M, const cx_t<T> *__restrict__ twM)
{
    int Ns = 1;
    for (; Ns * 4 <= M; Ns *= 4) pass_small<T, 4, DIR>(data, M, Ns, twM);
    if (Ns < M) pass_small<T, 2, DIR>(data, M, Ns, twM);
}

// the last pass of length-n transform for a prime p = n / Ns >= kBluePrime: for each
// j < Ns, Z_r = Σ_q x[j + q Ns] e^{DIR 2πi qj/n} e^{DIR 2πi qr/p} -> x[j + r Ns], by
// Bluestein: with h_q = e^{DIR iπ q²/p}, Z_r = h_r (1/M) DFT+(DFT-(a) · G)[r], a_q = x' h_q
template <typename T, int DIR>
__device__ void pass_bluestein(cx_t<T> *data, int n, const FftFactors &fac, const cx_t<T> *__restrict__ tw,
                               const cx_t<T> *__restrict__ twM, const cx_t<T> *__restrict__ blue, cx_t<T> *scratch)
{
    using C2 = cx_t<T>;
    const int p = fac.blue_p, M = fac.blue_M, Ns = n / p;
    const C2 *h = blue + fac.blue_off;                     // h_q, q < p
    const C2 *G = h + p + (DIR > 0 ? 0 : M);               // G for this transform sign
    const T invM = T(1) / (T)M;
    for (int j = 0; j < Ns; j++) {
        for (int q = threadIdx.x; q < M; q += FFT_NT) {
            C2 v{0, 0};
            if (q < p) {
                v = data[j + q * Ns];
                if (j) v = cmul<T>(v, twid<T, DIR>(tw, (int)((2LL * q * j) % (2 * n))));
                C2 hq = h[q];
                if (DIR < 0) hq.y = -hq.y;
                v = cmul<T>(v, hq);
            }
            scratch[q] = v;
        }
        __syncthreads();
        fft_pow2<T, -1>(scratch, M, twM);
        for (int f = threadIdx.x; f < M; f += FFT_NT) scratch[f] = cmul<T>(scratch[f], G[f]);
        __syncthreads();
        fft_pow2<T, +1>(scratch, M, twM);
        for (int r = threadIdx.x; r < p; r += FFT_NT) {
            C2 hr = h[r];
            if (DIR < 0) hr.y = -hr.y;
            C2 v = cmul<T>(scratch[r], hr);
            v.x *= invM;
            v.y *= invM;
            data[j + r * Ns] = v;
        }
        __syncthreads();
    }
}

template <typename T, int DIR>
__device__ void fft_inplace(cx_t<T> *data, int n, const FftFactors &fac,
                            const cx_t<T> *__restrict__ tw, const cx_t<T> *__restrict__ tw_all,
                            const cx_t<T> *__restrict__ blue, cx_t<T> *scratch)
{
    int Ns = 1;
    for (int i = 0; i < fac.nf; i++) {
        const int R = fac.f[i];
        switch (R) {
        case 4: pass_small<T, 4, DIR>(data, n, Ns, tw); break;
        case 2: pass_small<T, 2, DIR>(data, n, Ns, tw); break;
        default: pass_generic<T, DIR>(data, n, Ns, R, tw); break;
        }
        Ns *= R;
    }
    if (fac.blue_p) {
        // twiddles of length M = 4i sit at offset 4 i (i - 1) of the plan's table
        const long long iM = fac.blue_M / 4;
        pass_bluestein<T, DIR>(data, n, fac, tw, tw_all + 4 * iM * (iM - 1), blue, scratch);
    }
}

__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <typename T, int MODE>
__global__ void __launch_bounds__(FFT_NT)
k_ring_fft(int L, int nring, long long npix, int nmax, const int *__restrict__ rings,
           const RingInfo *__restrict__ rinfo, const FftFactors *__restrict__ factors,
           const cx_t<T> *__restrict__ tw_all, const T *__restrict__ W, int weighted,
           cx_t<T> *__restrict__ phi, const T *__restrict__ map_in, T *__restrict__ map_out,
           const int *__restrict__ skip, const cx_t<T> *__restrict__ blue)
{
    using C2 = cx_t<T>;
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C2 *data = reinterpret_cast<C2 *>(smem_raw);
    C2 *red = data + nmax;
    C2 *scratch = red + FFT_NT;   // Bluestein convolution buffer (when the plan has one)
    const int ring = rings ? rings[blockIdx.x] : (int)blockIdx.x;
    const int r = blockIdx.y;
    const int tid = threadIdx.x;
    const RingInfo ri = rinfo[AKRA_IX(ring, nring, kDbgFftRing)];
    const int n = ri.nphi, sigma = ri.sigma;
    const long long first = ri.first;
    const FftFactors fac = factors[ri.ilen];
    const C2 *tw = tw_all + ri.tw_off;
    C2 *prow = phi + ((size_t)r * nring + ring) * (2 * (size_t)L + 1) + L;   // prow[m], |m| <= L
    // checked offsets within the ring's Φ row (|m| <= L) and within the map (pixel < npix)
#define AKRA_ROW(m) (AKRA_IX((long long)L + (m), 2LL * L + 1, kDbgFftPhi) - L)
#define AKRA_PIX(j, site) (AKRA_IX(first + (j), npix, site) - first)

    if (MODE != (int)FftMode::Adjoint) {
        // fold Φ(m) into n bins
        if (n >= FFT_NT) {
            for (int k = tid; k < n; k += FFT_NT) {
                const int qlo = -((L + k) / n), qhi = floordiv(L - k, n);
                C2 acc{0, 0};
                for (int q = qlo; q <= qhi; q++) {
                    const C2 v = prow[AKRA_ROW(k + n * q)];
                    if (sigma && (q & 1)) { acc.x -= v.x; acc.y -= v.y; }
                    else { acc.x += v.x; acc.y += v.y; }
                }
                data[k] = sigma ? cmul<T>(acc, tw[k]) : acc;
            }
        } else {
            const int G = FFT_NT / n, g = tid / n, k = tid - g * n;
            if (g < G) {
                const int qlo = -((L + k) / n), qhi = floordiv(L - k, n);
                C2 acc{0, 0};
                for (int q = qlo + g; q <= qhi; q += G) {
                    const C2 v = prow[AKRA_ROW(k + n * q)];
                    if (sigma && (q & 1)) { acc.x -= v.x; acc.y -= v.y; }
                    else { acc.x += v.x; acc.y += v.y; }
                }
                red[g * n + k] = acc;
            }
            __syncthreads();
            for (int kk = tid; kk < n; kk += FFT_NT) {
                C2 acc{0, 0};
                for (int gg = 0; gg < G; gg++) {
                    acc.x += red[gg * n + kk].x;
                    acc.y += red[gg * n + kk].y;
                }
                data[kk] = sigma ? cmul<T>(acc, tw[kk]) : acc;
            }
        }
        __syncthreads();
        fft_inplace<T, +1>(data, n, fac, tw, tw_all, blue, scratch);
        if (MODE == (int)FftMode::Synth) {
            T *o1 = map_out + ((size_t)r * 2 + 0) * npix + first;
            T *o2 = map_out + ((size_t)r * 2 + 1) * npix + first;
            for (int j = tid; j < n; j += FFT_NT) {
                C2 v = data[j];
                if (weighted) {
                    const T wj = W[AKRA_IX(first + j, npix, kDbgFftWeight)];
                    v.x *= wj;
                    v.y *= wj;
                }
                o1[AKRA_PIX(j, kDbgFftMapOut)] = v.x;
                o2[AKRA_PIX(j, kDbgFftMapOut)] = v.y;
            }
            return;
        }
        for (int j = tid; j < n; j += FFT_NT) {
            const T wj = W[AKRA_IX(first + j, npix, kDbgFftWeight)];
            data[j].x *= wj;
            data[j].y *= wj;
        }
        __syncthreads();
    } else {
        const T *u1 = map_in + ((size_t)r * 2 + 0) * npix + first;
        const T *u2 = map_in + ((size_t)r * 2 + 1) * npix + first;
        for (int j = tid; j < n; j += FFT_NT) {
            C2 v{u1[AKRA_PIX(j, kDbgFftMapIn)], u2[AKRA_PIX(j, kDbgFftMapIn)]};
            if (weighted) {
                const T wj = W[AKRA_IX(first + j, npix, kDbgFftWeight)];
                v.x *= wj;
                v.y *= wj;
            }
            data[j] = v;
        }
        __syncthreads();
    }
    fft_inplace<T, -1>(data, n, fac, tw, tw_all, blue, scratch);
    // unfold: Φ'(m) = e^{-iπσk/n} (-1)^{σq} Ŵ[k],  m = k + nq
    for (int mm = tid; mm < 2 * L + 1; mm += FFT_NT) {
        const int m = mm - L;
        const int q = floordiv(m, n), k = m - q * n;
        C2 v = data[k];
        if (sigma) {
            v = cmul<T>(v, twid<T, -1>(tw, k));
            if (q & 1) { v.x = -v.x; v.y = -v.y; }
        }
        prow[AKRA_ROW(m)] = v;
    }
#undef AKRA_ROW
#undef AKRA_PIX
}

template <typename T> const cx_t<T> *tw_ptr(akra_plan p);
template <> const float2 *tw_ptr<float>(akra_plan p) { return p->d_tw32; }
template <> const double2 *tw_ptr<double>(akra_plan p) { return p->d_tw64; }
template <typename T> const T *W_ptr(akra_plan p);
template <> const float *W_ptr<float>(akra_plan p) { return p->d_W32; }
template <> const double *W_ptr<double>(akra_plan p) { return p->d_W64; }

// largest Bluestein convolution length of the plan's ring lengths (0: none)
static int blue_maxM(akra_plan p)
{
    int mx = 0;
    for (int i = 1; i <= p->nside; i++) {
        const int n = 4 * i;
        int m = i;
        while (m % 2 == 0) m /= 2;
        int big = 0;
        for (int d = 3; d * d <= m; d += 2)
            while (m % d == 0) m /= d;
        if (m > 1) big = m;
        (void)n;
        if (big >= kBluePrime) {
            int M = 1;
            while (M < 2 * big - 1) M *= 2;
            mx = M > mx ? M : mx;
        }
    }
    return mx;
}

template <typename T, int MODE>
static akra_status launch_fft(akra_plan p, void *phi, const void *map_in, void *map_out,
                              bool weighted, int R, const int *rings, int nrings, cudaStream_t st)
{
    const int nmax = 4 * p->nside;
    const bool dbl = sizeof(T) == sizeof(double);
    const int mblue = dbl ? blue_maxM(p) : 0;
    const size_t smem = (size_t)(nmax + FFT_NT + mblue) * sizeof(cx_t<T>);
    auto kern = k_ring_fft<T, MODE>;
    dim3 grid(nrings, R);
    kern<<<grid, FFT_NT, smem, st>>>(p->lmax, p->nring, p->npix, nmax, rings, p->d_rings,
                                     p->d_factors, tw_ptr<T>(p), W_ptr<T>(p), weighted ? 1 : 0,
                                     (cx_t<T> *)phi, (const T *)map_in, (T *)map_out, p->cur_skip,
                                     dbl ? (const cx_t<T> *)p->d_blue64 : nullptr);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

template <typename T>
akra_status ring_fft(akra_plan p, FftMode mode, void *phi, const void *map_in, void *map_out,
                     bool weighted, int R, const int *rings, int nrings, cudaStream_t st)
{
    if (nrings <= 0) return AKRA_OK;
    if constexpr (sizeof(T) == sizeof(float))   // FP32: O(n log n) for every ring length
        return ring_fft32(p, mode, phi, map_in, map_out, weighted, R, rings, nrings, st);
    switch (mode) {
    case FftMode::Synth:
        return launch_fft<T, 0>(p, phi, map_in, map_out, weighted, R, rings, nrings, st);
    case FftMode::Adjoint:
        return launch_fft<T, 1>(p, phi, map_in, map_out, weighted, R, rings, nrings, st);
    default:
        return launch_fft<T, 2>(p, phi, map_in, map_out, weighted, R, rings, nrings, st);
    }
}

// raise the dynamic shared-memory limit of every ring-FFT kernel once (at plan creation,
// never inside a stream capture)
akra_status ring_fft_prepare(akra_plan p)
{
    // the attribute is per kernel, shared by every plan: clear the largest supported ring
    (void)p;
    const int nmax = FFT_NMAX;
    const int s32 = (nmax + FFT_NT) * (int)sizeof(float2);
    // FP64: + the Bluestein scratch of the largest prime below kMaxNside (M = 4096)
    const int s64 = (nmax + FFT_NT + 4096) * (int)sizeof(double2);
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64));
    return AKRA_OK;
}

template akra_status ring_fft<float>(akra_plan, FftMode, void *, const void *, void *, bool, int,
                                     const int *, int, cudaStream_t);
template akra_status ring_fft<double>(akra_plan, FftMode, void *, const void *, void *, bool, int,
                                      const int *, int, cudaStream_t);

AKRA_DEBUG_COLLECTOR(ringfft)

}  // namespace akra
