// akra_ringfft32_impl.cuh -- FP32 ring FFT bodies (see akra_ringfft32.cu for the method),
// shared by the per-plan launches and the multi-instance launches (akra_batch.cu).
#pragma once
#include "akra_internal.cuh"

namespace akra {

constexpr int F32_NT = 512;
constexpr int F32_MMAX = 8 * kMaxNside;   // largest convolution length (n <= 4 nside - 4)
constexpr int F32_KPT = 4 * kMaxNside / F32_NT;   // ring pixels per thread at most
static_assert(F32_KPT * F32_NT >= 4 * kMaxNside, "a ring must fit F32_KPT slots per thread");

__device__ __forceinline__ float2 cm(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmc(float2 a, float2 b)   // a * conj(b)
{
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// multiply by s·i (s = ±1)
template <int S> __device__ __forceinline__ float2 mul_si(float2 a)
{
    return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// e^{S 2πi t/L} from the table e^{-2πi u/MMAX}
template <int S>
__device__ __forceinline__ float2 w_pow2(const float2 *__restrict__ tw2, int t, int L)
{
    float2 w = tw2[t * (F32_MMAX / L)];
    if (S > 0) w.y = -w.y;
    return w;
}

// e^{S 2πi m/16} for 0 <= m < 16 (m is a compile-time constant after unrolling):
// cos(2πm/16) from cos 0, cos π/8, cos π/4, cos 3π/8, cos π/2 by symmetry, sin(2πm/16) =
// cos(2π(m-4)/16)
__device__ __forceinline__ constexpr float cos16(int m)
{
    constexpr float c[5] = {1.0f, 0.923879532511286756f, 0.707106781186547524f, 0.382683432365089772f, 0.0f};
    return m <= 4 ? c[m] : m <= 8 ? -c[8 - m] : m <= 12 ? -c[m - 8] : c[16 - m];
}
template <int S> __device__ __forceinline__ float2 root16(int m)
{
    return make_float2(cos16(m & 15), S * cos16((m + 12) & 15));
}

// radix-4 DIF butterfly on (a0..a3) = x[t + k q] of a length-L stage, in place: the outputs go
// where the in-place DIF keeps them (slot 1 holds the k = 2 output, slot 2 the k = 1 one),
// twiddled by w1 = w^i, w2 = w^{2i}, w3 = w^{3i} of length L
template <int S>
__device__ __forceinline__ void dif4(float2 &a0, float2 &a1, float2 &a2, float2 &a3, float2 w1, float2 w2,
                                     float2 w3)
{
    const float2 u0 = cadd(a0, a2), u1 = cadd(a1, a3), d0 = csub(a0, a2);
    const float2 d1 = mul_si<S>(csub(a1, a3));
    a0 = cadd(u0, u1);
    a1 = cm(csub(u0, u1), w2);
    a2 = cm(cadd(d0, d1), w1);
    a3 = cm(csub(d0, d1), w3);
}

// radix-4 DIT butterfly (the inverse arrangement of dif4), w1 = w^i, w2 = w^{2i} of length L
template <int S>
__device__ __forceinline__ void dit4(float2 &p0, float2 &p1, float2 &p2, float2 &p3, float2 w1, float2 w2)
{
    float2 u = cm(p1, w2);
    const float2 u0 = cadd(p0, u), u1 = csub(p0, u);
    u = cm(p3, w2);
    const float2 u2 = cadd(p2, u), u3 = csub(p2, u);
    const float2 v2 = cm(u2, w1), v3 = mul_si<S>(cm(u3, w1));
    p0 = cadd(u0, v2);
    p2 = csub(u0, v2);
    p1 = cadd(u1, v3);
    p3 = csub(u1, v3);
}

// Shared-memory slot of element i: one float2 of padding after every 16, so that the radix-4
// passes with element strides 1 and 4 (and every larger power of two) hit distinct banks.
__host__ __device__ constexpr int f32_slots(int m) { return m + (m >> 4); }
__device__ __forceinline__ int pd(int i) { return i + (i >> 4); }

// in-place DIF with DFT sign S: natural order in, bit-reversed out
template <int S>
__device__ void dif(float2 *x, int M, int logM, const float2 *__restrict__ tw2)
{
    int L = M;
    if (logM & 1) {
        const int h = M >> 1;
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const float2 a = x[pd(i)], b = x[pd(i + h)];
            x[pd(i)] = cadd(a, b);
            x[pd(i + h)] = cm(csub(a, b), w_pow2<S>(tw2, i, M));
        }
        __syncthreads();
        L = h;
    }
    // two radix-4 stages (lengths L and L/4) per pass: a thread holds the 16 elements t + j·L/16,
    // which form four groups of the first stage (j mod 4 fixed) and, after it, four groups of the
    // second (j div 4 fixed); results land where two separate passes would put them
    for (; L >= 16; L >>= 4) {
        const int q = L >> 4, lq = 31 - __clz(q);
        for (int b = threadIdx.x; b < (M >> 4); b += blockDim.x) {
            const int blk = b >> lq, i = b & (q - 1);
            const int t = blk * L + i;
            float2 v[16];
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = x[pd(t + j * q)];
            {
                // twiddles of group j1 (index i + j1·L/16): w^{k i} · e^{S 2πi k j1/16}
                const float2 b1 = w_pow2<S>(tw2, i, L), b2 = w_pow2<S>(tw2, 2 * i, L),
                             b3 = w_pow2<S>(tw2, 3 * i, L);
                dif4<S>(v[0], v[4], v[8], v[12], b1, b2, b3);
#pragma unroll
                for (int j1 = 1; j1 < 4; j1++)
                    dif4<S>(v[j1], v[j1 + 4], v[j1 + 8], v[j1 + 12], cm(b1, root16<S>(j1)),
                            cm(b2, root16<S>(2 * j1)), cm(b3, root16<S>(3 * j1)));
            }
            const int L2 = L >> 2;
            const float2 w1 = w_pow2<S>(tw2, i, L2), w2 = w_pow2<S>(tw2, 2 * i, L2),
                         w3 = w_pow2<S>(tw2, 3 * i, L2);
#pragma unroll
            for (int j2 = 0; j2 < 4; j2++) dif4<S>(v[4 * j2], v[4 * j2 + 1], v[4 * j2 + 2], v[4 * j2 + 3], w1, w2, w3);
#pragma unroll
            for (int j = 0; j < 16; j++) x[pd(t + j * q)] = v[j];
        }
        __syncthreads();
    }
    if (L == 4) {
        for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
            const int t = 4 * b;
            float2 a0 = x[pd(t)], a1 = x[pd(t + 1)], a2 = x[pd(t + 2)], a3 = x[pd(t + 3)];
            const float2 one = make_float2(1.f, 0.f);
            dif4<S>(a0, a1, a2, a3, one, one, one);
            x[pd(t)] = a0;
            x[pd(t + 1)] = a1;
            x[pd(t + 2)] = a2;
            x[pd(t + 3)] = a3;
        }
        __syncthreads();
    }
}

// in-place DIT with DFT sign S: bit-reversed order in, natural out (DIT<-S>(DIF<S>(x)) = M x)
template <int S>
__device__ void dit(float2 *x, int M, int logM, const float2 *__restrict__ tw2)
{
    const int Lmax = (logM & 1) ? (M >> 1) : M;
    int L = 4;
    // two radix-4 stages (lengths L and 4L) per pass: a thread holds the 16 elements t + j·L/4 of
    // one 4L block, four groups of the first stage (j div 4 fixed), then four of the second
    // (j mod 4 fixed)
    for (; 4 * L <= Lmax; L <<= 4) {
        const int q = L >> 2, lq = 31 - __clz(q);
        for (int b = threadIdx.x; b < (M >> 4); b += blockDim.x) {
            const int blk = b >> lq, i = b & (q - 1);
            const int t = blk * 4 * L + i;
            float2 v[16];
#pragma unroll
            for (int j = 0; j < 16; j++) v[j] = x[pd(t + j * q)];
            {
                const float2 w1 = w_pow2<S>(tw2, i, L), w2 = w_pow2<S>(tw2, 2 * i, L);
#pragma unroll
                for (int j2 = 0; j2 < 4; j2++) dit4<S>(v[4 * j2], v[4 * j2 + 1], v[4 * j2 + 2], v[4 * j2 + 3], w1, w2);
            }
            {
                // twiddles of group j1 (index i + j1·L/4 of length 4L): w^{k i} · e^{S 2πi k j1/16}
                const float2 b1 = w_pow2<S>(tw2, i, 4 * L), b2 = w_pow2<S>(tw2, 2 * i, 4 * L);
                dit4<S>(v[0], v[4], v[8], v[12], b1, b2);
#pragma unroll
                for (int j1 = 1; j1 < 4; j1++)
                    dit4<S>(v[j1], v[j1 + 4], v[j1 + 8], v[j1 + 12], cm(b1, root16<S>(j1)), cm(b2, root16<S>(2 * j1)));
            }
#pragma unroll
            for (int j = 0; j < 16; j++) x[pd(t + j * q)] = v[j];
        }
        __syncthreads();
    }
    if (L <= Lmax) {   // one radix-4 stage left (length L)
        const int q = L >> 2;
        for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
            const int blk = b / q, i = b - blk * q;
            const int t = blk * L + i;
            float2 p0 = x[pd(t)], p1 = x[pd(t + q)], p2 = x[pd(t + 2 * q)], p3 = x[pd(t + 3 * q)];
            dit4<S>(p0, p1, p2, p3, w_pow2<S>(tw2, i, L), w_pow2<S>(tw2, 2 * i, L));
            x[pd(t)] = p0;
            x[pd(t + q)] = p1;
            x[pd(t + 2 * q)] = p2;
            x[pd(t + 3 * q)] = p3;
        }
        __syncthreads();
    }
    if (logM & 1) {
        const int h = M >> 1;
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const float2 a = x[pd(i)], b = cm(x[pd(i + h)], w_pow2<S>(tw2, i, M));
            x[pd(i)] = cadd(a, b);
            x[pd(i + h)] = csub(a, b);
        }
        __syncthreads();
    }
}

// Bluestein DFT of x[0..n) in place (natural order in and out), sign S.
// chirp c_j = tw_ring[j^2 mod 2n] = e^{iπ j²/n}; bhat = DIF<-1> of the chirp filter.
template <int S>
__device__ void bluestein(float2 *x, int n, int M, int logM, const float2 *__restrict__ tw_ring,
                          const float2 *__restrict__ bhat, const float2 *__restrict__ tw2)
{
    const int n2 = 2 * n;
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        if (j < n) {
            const float2 c = tw_ring[(int)(((long long)j * j) % n2)];
            const float2 v = x[pd(j)];
            // forward: x conj(c);  backward: conj(x c) (conjugation trick)
            x[pd(j)] = S < 0 ? cmc(v, c) : make_float2(v.x * c.x - v.y * c.y, -(v.x * c.y + v.y * c.x));
        } else {
            x[pd(j)] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    dif<-1>(x, M, logM, tw2);
    for (int k = threadIdx.x; k < M; k += blockDim.x) x[pd(k)] = cm(x[pd(k)], bhat[k]);
    __syncthreads();
    dit<+1>(x, M, logM, tw2);
    const float inv = 1.0f / (float)M;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float2 c = tw_ring[(int)(((long long)k * k) % n2)];
        const float2 y = x[pd(k)];
        // forward: conj(c) y / M;  backward: c conj(y) / M
        const float2 r = S < 0 ? cmc(y, c) : cmc(c, y);
        x[pd(k)] = make_float2(r.x * inv, r.y * inv);
    }
    __syncthreads();
}

__device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int MODE>
__device__ __forceinline__ void ring_fft32_item(const Fft32Args &a, const int ring, const int r,
                                                float2 *buf, float2 *red)
{
    const int L = a.L, nring = a.nring;
    const long long npix = a.npix;
    const RingInfo *__restrict__ rinfo = a.rinfo;
    const int *__restrict__ fftM = a.fftM;
    const long long *__restrict__ bhat_off = a.bhat_off;
    const float2 *__restrict__ bhat_all = a.bhat_all;
    const float2 *__restrict__ tw2 = a.tw2;
    const float2 *__restrict__ tw_all = a.tw_all;
    const float *__restrict__ W = a.W;
    const int weighted = a.weighted;
    float2 *__restrict__ phi = a.phi;
    const float *__restrict__ map_in = a.map_in;
    float *__restrict__ map_out = a.map_out;
    const int tid = threadIdx.x;
    const RingInfo ri = rinfo[AKRA_IX(ring, nring, kDbgFftRing)];
    const int n = ri.nphi, sigma = ri.sigma;
    const long long first = ri.first;
    const float2 *tw = tw_all + ri.tw_off;         // e^{iπ t/n}, t < 2n
    const int M = fftM[ri.ilen];
    const bool pow2 = (M == n);
    const int logM = 31 - __clz(M), logn = 31 - __clz(n);
    const float2 *bhat = pow2 ? nullptr : bhat_all + bhat_off[ri.ilen];
    float2 *prow = phi + ((size_t)r * nring + ring) * (2 * (size_t)L + 1) + L;
    // checked offsets within the ring's Φ row (|m| <= L) and within the map (pixel < npix)
#define AKRA_ROW(m) (AKRA_IX((long long)L + (m), 2LL * L + 1, kDbgFftPhi) - L)
#define AKRA_PIX(j, site) (AKRA_IX(first + (j), npix, site) - first)

    if (MODE != (int)FftMode::Adjoint) {
        // fold Φ(m) into n bins: F[k] = e^{iπσk/n} Σ_q (-1)^{σq} Φ(k + nq)
        if (n >= F32_NT) {
            // a thread's bins k = tid + u·F32_NT (u < F32_KPT), each summed over q in increasing
            // order; the loads of one q are independent, so they are all in flight together
            float2 acc[F32_KPT];
#pragma unroll
            for (int u = 0; u < F32_KPT; u++) acc[u] = make_float2(0.f, 0.f);
            const int qmin = fdiv(-L, n), qmax = fdiv(L, n);
            for (int q = qmin; q <= qmax; q++) {
                const bool neg = sigma && (q & 1);
#pragma unroll
                for (int u = 0; u < F32_KPT; u++) {
                    const int k = tid + u * F32_NT, m = k + n * q;
                    if (k < n && m >= -L && m <= L) {
                        const float2 v = prow[AKRA_ROW(m)];
                        acc[u] = neg ? csub(acc[u], v) : cadd(acc[u], v);
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < F32_KPT; u++) {
                const int k = tid + u * F32_NT;
                if (k < n) buf[pd(k)] = sigma ? cm(acc[u], tw[k]) : acc[u];
            }
        } else {
            const int G = F32_NT / n, g = tid / n, k = tid - g * n;
            if (g < G) {
                const int qlo = -((L + k) / n), qhi = fdiv(L - k, n);
                float2 acc = make_float2(0.f, 0.f);
                for (int q = qlo + g; q <= qhi; q += G) {
                    const float2 v = prow[AKRA_ROW(k + n * q)];
                    if (sigma && (q & 1)) acc = csub(acc, v);
                    else acc = cadd(acc, v);
                }
                red[g * n + k] = acc;
            }
            __syncthreads();
            for (int kk = tid; kk < n; kk += F32_NT) {
                float2 acc = make_float2(0.f, 0.f);
                for (int gg = 0; gg < G; gg++) acc = cadd(acc, red[gg * n + kk]);
                buf[pd(kk)] = sigma ? cm(acc, tw[kk]) : acc;
            }
        }
        __syncthreads();
        // backward DFT: pixel values (bit-reversed order for power-of-two rings)
        if (pow2) dif<+1>(buf, n, logn, tw2);
        else bluestein<+1>(buf, n, M, logM, tw, bhat, tw2);
        if (MODE == (int)FftMode::Synth) {
            float *o1 = map_out + ((size_t)r * 2 + 0) * npix + first;
            float *o2 = map_out + ((size_t)r * 2 + 1) * npix + first;
            for (int k = tid; k < n; k += F32_NT) {
                const int j = pow2 ? (int)(__brev((unsigned)k) >> (32 - logn)) : k;
                float2 v = buf[pd(k)];
                if (weighted) {
                    const float wj = W[AKRA_IX(first + k, npix, kDbgFftWeight)];
                    v.x *= wj;
                    v.y *= wj;
                }
                o1[AKRA_PIX(j, kDbgFftMapOut)] = v.x;
                o2[AKRA_PIX(j, kDbgFftMapOut)] = v.y;
            }
            return;
        }
        // ×W: slot k's weight is W[first + k] (stored in this slot order), loads all in flight
#pragma unroll
        for (int u = 0; u < F32_KPT; u++) {
            const int k = tid + u * F32_NT;
            if (k < n) {
                const float wj = W[AKRA_IX(first + k, npix, kDbgFftWeight)];
                buf[pd(k)].x *= wj;
                buf[pd(k)].y *= wj;
            }
        }
        __syncthreads();
    } else {
        const float *u1 = map_in + ((size_t)r * 2 + 0) * npix + first;
        const float *u2 = map_in + ((size_t)r * 2 + 1) * npix + first;
        for (int k = tid; k < n; k += F32_NT) {
            const int j = pow2 ? (int)(__brev((unsigned)k) >> (32 - logn)) : k;
            float2 v = make_float2(u1[AKRA_PIX(j, kDbgFftMapIn)], u2[AKRA_PIX(j, kDbgFftMapIn)]);
            if (weighted) {
                const float wj = W[AKRA_IX(first + k, npix, kDbgFftWeight)];
                v.x *= wj;
                v.y *= wj;
            }
            buf[pd(k)] = v;
        }
        __syncthreads();
    }
    // forward DFT back to bins (natural order)
    if (pow2) dit<-1>(buf, n, logn, tw2);
    else bluestein<-1>(buf, n, M, logM, tw, bhat, tw2);
    // unfold: Φ'(m) = e^{-iπσk/n} (-1)^{σq} Ŵ[k],  m = k + nq
    for (int mm = tid; mm < 2 * L + 1; mm += F32_NT) {
        const int m = mm - L;
        const int q = fdiv(m, n), k = m - q * n;
        float2 v = buf[pd(k)];
        if (sigma) {
            v = cmc(v, tw[k]);
            if (q & 1) v = make_float2(-v.x, -v.y);
        }
        prow[AKRA_ROW(m)] = v;
    }
#undef AKRA_ROW
#undef AKRA_PIX
}


template <int MODE>
__global__ void __launch_bounds__(F32_NT, 2) k_ring_fft32(Fft32Args a)
{
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int ring = a.rings ? a.rings[blockIdx.x] : (int)blockIdx.x;
    ring_fft32_item<MODE>(a, ring, blockIdx.y, buf, buf + f32_slots(a.mmax));
}

// batched form over several plans: item = {instance, index into its ring list, RHS, 0}
template <int MODE>
__global__ void __launch_bounds__(F32_NT)
k_ring_fft32_batch(const Fft32Args *__restrict__ insts, const int4 *__restrict__ items, int mmax)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int4 w = items[blockIdx.x];
    const Fft32Args a = insts[w.x];
    if (a.skip && *a.skip) return;
    const int ring = a.rings ? a.rings[w.y] : w.y;
    ring_fft32_item<MODE>(a, ring, w.z, buf, buf + f32_slots(mmax));
}

}  // namespace akra
