// akra_ringfft32.cu -- FP32 ring phase sums (the φ half of SHT^-1 / SHT, Sec. II B) with the
// pixel diagonal W fused between them: O(n log n) for every ring length.
//
// The ring sums are the same as in akra_ringfft.cu (fold Φ(m) into n bins with phase
// e^{iπσk/n}, length-n DFT, ×W, DFT back, unfold).  Here the length-n DFTs are
//   * n a power of two: in-place radix-4/2 decimation in frequency (natural -> bit-reversed)
//     for the backward DFT and decimation in time (bit-reversed -> natural) for the forward
//     one, so W is applied to the bit-reversed pixel order and no permutation pass is needed;
//   * any other n (polar rings n = 4i): Bluestein's chirp-z form,
//       X_k = conj(c_k) Σ_j [x_j conj(c_j)] c_{k-j},  c_j = e^{iπ j²/n},
//     a cyclic convolution of length M = 2^⌈log2(2n-1)⌉ done by the same DIF/DIT pair, with
//     the chirp's spectrum precomputed per ring length (stored in DIF output order).
//     The backward DFT is conj(forward(conj x)).
#include "akra_internal.cuh"

namespace akra {

constexpr int F32_NT = 1024;
constexpr int F32_MMAX = 8 * kMaxNside;   // largest convolution length (n <= 4 nside - 4)

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

// in-place DIF with DFT sign S: natural order in, bit-reversed out
template <int S>
__device__ void dif(float2 *x, int M, int logM, const float2 *__restrict__ tw2)
{
    int L = M;
    if (logM & 1) {
        const int h = M >> 1;
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const float2 a = x[i], b = x[i + h];
            x[i] = cadd(a, b);
            x[i + h] = cm(csub(a, b), w_pow2<S>(tw2, i, M));
        }
        __syncthreads();
        L = h;
    }
    for (; L >= 4; L >>= 2) {
        const int q = L >> 2;
        for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
            const int blk = b / q, i = b - blk * q;
            float2 *p = x + blk * L + i;
            const float2 a0 = p[0], a1 = p[q], a2 = p[2 * q], a3 = p[3 * q];
            const float2 w1 = w_pow2<S>(tw2, i, L), w2 = w_pow2<S>(tw2, 2 * i, L),
                         w3 = w_pow2<S>(tw2, 3 * i, L);
            const float2 u0 = cadd(a0, a2), u1 = cadd(a1, a3), d0 = csub(a0, a2);
            const float2 d1 = mul_si<S>(csub(a1, a3));
            p[0] = cadd(u0, u1);
            p[q] = cm(csub(u0, u1), w2);
            p[2 * q] = cm(cadd(d0, d1), w1);
            p[3 * q] = cm(csub(d0, d1), w3);
        }
        __syncthreads();
    }
}

// in-place DIT with DFT sign S: bit-reversed order in, natural out (DIT<-S>(DIF<S>(x)) = M x)
template <int S>
__device__ void dit(float2 *x, int M, int logM, const float2 *__restrict__ tw2)
{
    const int Lmax = (logM & 1) ? (M >> 1) : M;
    for (int L = 4; L <= Lmax; L <<= 2) {
        const int q = L >> 2;
        for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
            const int blk = b / q, i = b - blk * q;
            float2 *p = x + blk * L + i;
            const float2 p0 = p[0], p1 = p[q], p2 = p[2 * q], p3 = p[3 * q];
            const float2 w1 = w_pow2<S>(tw2, i, L), w2 = w_pow2<S>(tw2, 2 * i, L);
            float2 t = cm(p1, w2);
            const float2 u0 = cadd(p0, t), u1 = csub(p0, t);
            t = cm(p3, w2);
            const float2 u2 = cadd(p2, t), u3 = csub(p2, t);
            const float2 v2 = cm(u2, w1), v3 = mul_si<S>(cm(u3, w1));
            p[0] = cadd(u0, v2);
            p[2 * q] = csub(u0, v2);
            p[q] = cadd(u1, v3);
            p[3 * q] = csub(u1, v3);
        }
        __syncthreads();
    }
    if (logM & 1) {
        const int h = M >> 1;
        for (int i = threadIdx.x; i < h; i += blockDim.x) {
            const float2 a = x[i], b = cm(x[i + h], w_pow2<S>(tw2, i, M));
            x[i] = cadd(a, b);
            x[i + h] = csub(a, b);
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
            const float2 v = x[j];
            // forward: x conj(c);  backward: conj(x c) (conjugation trick)
            x[j] = S < 0 ? cmc(v, c) : make_float2(v.x * c.x - v.y * c.y, -(v.x * c.y + v.y * c.x));
        } else {
            x[j] = make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    dif<-1>(x, M, logM, tw2);
    for (int k = threadIdx.x; k < M; k += blockDim.x) x[k] = cm(x[k], bhat[k]);
    __syncthreads();
    dit<+1>(x, M, logM, tw2);
    const float inv = 1.0f / (float)M;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const float2 c = tw_ring[(int)(((long long)k * k) % n2)];
        const float2 y = x[k];
        // forward: conj(c) y / M;  backward: c conj(y) / M
        const float2 r = S < 0 ? cmc(y, c) : cmc(c, y);
        x[k] = make_float2(r.x * inv, r.y * inv);
    }
    __syncthreads();
}

__device__ __forceinline__ int fdiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int MODE>
__global__ void __launch_bounds__(F32_NT)
k_ring_fft32(int L, int nring, long long npix, int mmax, const int *__restrict__ rings,
             const RingInfo *__restrict__ rinfo, const int *__restrict__ fftM,
             const long long *__restrict__ bhat_off, const float2 *__restrict__ bhat_all,
             const float2 *__restrict__ tw2, const float2 *__restrict__ tw_all,
             const float *__restrict__ W, int weighted, float2 *__restrict__ phi,
             const float *__restrict__ map_in, float *__restrict__ map_out,
             const int *__restrict__ skip)
{
    if (skip && *skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *red = buf + mmax;
    const int ring = rings ? rings[blockIdx.x] : (int)blockIdx.x;
    const int r = blockIdx.y, tid = threadIdx.x;
    const RingInfo ri = rinfo[ring];
    const int n = ri.nphi, sigma = ri.sigma;
    const long long first = ri.first;
    const float2 *tw = tw_all + ri.tw_off;         // e^{iπ t/n}, t < 2n
    const int M = fftM[ri.ilen];
    const bool pow2 = (M == n);
    const int logM = 31 - __clz(M), logn = 31 - __clz(n);
    const float2 *bhat = pow2 ? nullptr : bhat_all + bhat_off[ri.ilen];
    float2 *prow = phi + ((size_t)r * nring + ring) * (2 * (size_t)L + 1) + L;

    if (MODE != (int)FftMode::Adjoint) {
        // fold Φ(m) into n bins: F[k] = e^{iπσk/n} Σ_q (-1)^{σq} Φ(k + nq)
        if (n >= F32_NT) {
            for (int k = tid; k < n; k += F32_NT) {
                const int qlo = -((L + k) / n), qhi = fdiv(L - k, n);
                float2 acc = make_float2(0.f, 0.f);
                for (int q = qlo; q <= qhi; q++) {
                    const float2 v = prow[k + n * q];
                    if (sigma && (q & 1)) acc = csub(acc, v);
                    else acc = cadd(acc, v);
                }
                buf[k] = sigma ? cm(acc, tw[k]) : acc;
            }
        } else {
            const int G = F32_NT / n, g = tid / n, k = tid - g * n;
            if (g < G) {
                const int qlo = -((L + k) / n), qhi = fdiv(L - k, n);
                float2 acc = make_float2(0.f, 0.f);
                for (int q = qlo + g; q <= qhi; q += G) {
                    const float2 v = prow[k + n * q];
                    if (sigma && (q & 1)) acc = csub(acc, v);
                    else acc = cadd(acc, v);
                }
                red[g * n + k] = acc;
            }
            __syncthreads();
            for (int kk = tid; kk < n; kk += F32_NT) {
                float2 acc = make_float2(0.f, 0.f);
                for (int gg = 0; gg < G; gg++) acc = cadd(acc, red[gg * n + kk]);
                buf[kk] = sigma ? cm(acc, tw[kk]) : acc;
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
                float2 v = buf[k];
                if (weighted) {
                    const float wj = W[first + j];
                    v.x *= wj;
                    v.y *= wj;
                }
                o1[j] = v.x;
                o2[j] = v.y;
            }
            return;
        }
        for (int k = tid; k < n; k += F32_NT) {
            const int j = pow2 ? (int)(__brev((unsigned)k) >> (32 - logn)) : k;
            const float wj = W[first + j];
            buf[k].x *= wj;
            buf[k].y *= wj;
        }
        __syncthreads();
    } else {
        const float *u1 = map_in + ((size_t)r * 2 + 0) * npix + first;
        const float *u2 = map_in + ((size_t)r * 2 + 1) * npix + first;
        for (int k = tid; k < n; k += F32_NT) {
            const int j = pow2 ? (int)(__brev((unsigned)k) >> (32 - logn)) : k;
            float2 v = make_float2(u1[j], u2[j]);
            if (weighted) {
                const float wj = W[first + j];
                v.x *= wj;
                v.y *= wj;
            }
            buf[k] = v;
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
        float2 v = buf[k];
        if (sigma) {
            v = cmc(v, tw[k]);
            if (q & 1) v = make_float2(-v.x, -v.y);
        }
        prow[m] = v;
    }
}

// chirp-filter spectra: for each non-power-of-two ring length n = 4i,
// b_j = c_j (|j| < n, indices mod M), bhat = DIF<-1>(b)
__global__ void __launch_bounds__(F32_NT)
k_bhat32(int N, const int *__restrict__ fftM, const long long *__restrict__ bhat_off,
         const double2 *__restrict__ tw64_all, const float2 *__restrict__ tw2, float2 *bhat_all)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    const int i = blockIdx.x + 1;
    const int n = 4 * i, M = fftM[i];
    if (M == n) return;
    const double2 *tw = tw64_all + 4LL * i * (i - 1);
    for (int j = threadIdx.x; j < M; j += blockDim.x) {
        const int jj = j < n ? j : (j > M - n ? M - j : -1);
        float2 v = make_float2(0.f, 0.f);
        if (jj >= 0) {
            const double2 c = tw[(int)(((long long)jj * jj) % (2 * n))];
            v = make_float2((float)c.x, (float)c.y);
        }
        buf[j] = v;
    }
    __syncthreads();
    dif<-1>(buf, M, 31 - __clz(M), tw2);
    float2 *out = bhat_all + bhat_off[i];
    for (int j = threadIdx.x; j < M; j += blockDim.x) out[j] = buf[j];
}

__global__ void k_tw2(float2 *tw2)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < F32_MMAX) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)F32_MMAX, &s, &c);
        tw2[t] = make_float2((float)c, (float)s);
    }
}

static int next_pow2(int v)
{
    int m = 1;
    while (m < v) m <<= 1;
    return m;
}

// plan tables of the FP32 ring FFT (convolution lengths, chirp spectra, pow2 twiddles)
akra_status ring_fft32_build(akra_plan p)
{
    const int N = p->nside;
    std::vector<int> M(N + 1, 0);
    std::vector<long long> off(N + 1, -1);
    long long total = 0;
    int mmax = 4;
    for (int i = 1; i <= N; i++) {
        const int n = 4 * i;
        if ((n & (n - 1)) == 0) {
            M[i] = n;
        } else {
            M[i] = next_pow2(2 * n - 1);
            off[i] = total;
            total += M[i];
        }
        mmax = std::max(mmax, M[i]);
    }
    p->fft32_mmax = mmax;
    size_t bytes = sizeof(int) * (N + 1) + sizeof(long long) * (N + 1) + sizeof(float2) * F32_MMAX +
                   sizeof(float2) * (size_t)std::max(total, 1LL);
    if (cudaMalloc(&p->d_fft32_M, sizeof(int) * (N + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_off, sizeof(long long) * (N + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_tw2, sizeof(float2) * F32_MMAX) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_bhat, sizeof(float2) * (size_t)std::max(total, 1LL)) != cudaSuccess) {
        cudaGetLastError();
        set_error("ring FFT table allocation failed");
        return AKRA_ENOMEM;
    }
    p->bytes_tables += bytes;
    AKRA_CUDA_TRY(cudaMemcpy(p->d_fft32_M, M.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
    AKRA_CUDA_TRY(cudaMemcpy(p->d_fft32_off, off.data(), sizeof(long long) * (N + 1), cudaMemcpyHostToDevice));
    k_tw2<<<(F32_MMAX + 255) / 256, 256>>>(p->d_fft32_tw2);
    AKRA_CUDA_TRY(cudaGetLastError());
    const int smem_b = mmax * (int)sizeof(float2);
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_bhat32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_b));
    k_bhat32<<<N, F32_NT, smem_b>>>(N, p->d_fft32_M, p->d_fft32_off, p->d_tw64, p->d_fft32_tw2,
                                    p->d_fft32_bhat);
    AKRA_CUDA_TRY(cudaGetLastError());
    const int smem = (mmax + F32_NT) * (int)sizeof(float2);
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return AKRA_OK;
}

akra_status ring_fft32(akra_plan p, FftMode mode, void *phi, const void *map_in, void *map_out,
                       bool weighted, int R, const int *rings, int nrings, cudaStream_t st)
{
    if (nrings <= 0) return AKRA_OK;
    const int mmax = p->fft32_mmax;
    const size_t smem = (size_t)(mmax + F32_NT) * sizeof(float2);
    dim3 grid(nrings, R);
#define AKRA_F32_LAUNCH(MD)                                                                        \
    k_ring_fft32<MD><<<grid, F32_NT, smem, st>>>(p->lmax, p->nring, p->npix, mmax, rings, p->d_rings, \
                                                 p->d_fft32_M, p->d_fft32_off, p->d_fft32_bhat,       \
                                                 p->d_fft32_tw2, p->d_tw32, p->d_W32, weighted ? 1 : 0, \
                                                 (float2 *)phi, (const float *)map_in, (float *)map_out, \
                                                 p->cur_skip)
    switch (mode) {
    case FftMode::Synth: AKRA_F32_LAUNCH(0); break;
    case FftMode::Adjoint: AKRA_F32_LAUNCH(1); break;
    default: AKRA_F32_LAUNCH(2); break;
    }
#undef AKRA_F32_LAUNCH
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

}  // namespace akra
