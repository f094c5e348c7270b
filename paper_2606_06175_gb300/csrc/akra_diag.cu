// akra_diag.cu -- measured FMA rates of this GPU, the denominators of the Legendre kernels'
// pipe fractions (the recurrence and contraction steps are plain FP32 / FP64 FMA work).
#include <algorithm>
#include <chrono>

#include "akra_internal.cuh"

namespace akra {

// Every thread runs NC independent FMA chains, either sharing one multiplier and addend
// (operands the register reuse caches serve) or each with its own (DISTINCT); the values stay
// bounded (|b| < 1) and the sum is stored only under a condition that never holds, so no FMA
// can be removed.
template <typename T, int NC, bool DISTINCT>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, T b, T c, T *sink)
{
    T a[NC], bb[NC], cc[NC];
#pragma unroll
    for (int i = 0; i < NC; i++) {
        a[i] = (T)threadIdx.x * (T)1e-3 + (T)i;
        bb[i] = DISTINCT ? b - (T)i * (T)1e-7 : b;
        cc[i] = DISTINCT ? c + (T)i * (T)1e-9 : c;
    }
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < 16; u++)
#pragma unroll
            for (int i = 0; i < NC; i++) a[i] = fma(a[i], bb[i], cc[i]);
    }
    T s = 0;
#pragma unroll
    for (int i = 0; i < NC; i++) s += a[i];
    if (s == (T)-12345) sink[0] = s;
}

template <typename T, int NC, bool DISTINCT>
static akra_status fma_rate_one(int nb, int iters, T *sink, double *tflops)
{
    const int nt = 256;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_rate<T, NC, DISTINCT><<<nb, nt>>>(iters / 8, (T)0.999999, (T)1e-7, sink);   // warm-up
    cudaEventRecord(e0);
    k_fma_rate<T, NC, DISTINCT><<<nb, nt>>>(iters, (T)0.999999, (T)1e-7, sink);
    cudaEventRecord(e1);
    const cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    AKRA_CUDA_TRY(err);
    AKRA_CUDA_TRY(cudaGetLastError());
    *tflops = 2.0 * NC * 16 * (double)iters * nt * nb / (ms * 1e-3) / 1e12;
    return AKRA_OK;
}

// the best of 4 and 8 chains per thread with shared or distinct operands (FP32 runs fastest
// with shared ones, FP64 with distinct ones and the shorter register footprint)
template <typename T>
static akra_status fma_rate(double *tflops)
{
    int dev = 0, sms = 0;
    AKRA_CUDA_TRY(cudaGetDevice(&dev));
    AKRA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    T *sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_fma_rate: allocation failed");
        return AKRA_ENOMEM;
    }
    const int nb = sms * 8;
    const int iters = sizeof(T) == 4 ? 32768 : 512;   // about 30 ms per variant
    double r[4] = {0, 0, 0, 0};
    akra_status s = fma_rate_one<T, 4, false>(nb, 2 * iters, sink, &r[0]);
    if (s == AKRA_OK) s = fma_rate_one<T, 8, false>(nb, iters, sink, &r[1]);
    if (s == AKRA_OK) s = fma_rate_one<T, 4, true>(nb, 2 * iters, sink, &r[2]);
    if (s == AKRA_OK) s = fma_rate_one<T, 8, true>(nb, iters, sink, &r[3]);
    cudaFree(sink);
    if (s != AKRA_OK) return s;
    *tflops = std::max(std::max(r[0], r[1]), std::max(r[2], r[3]));
    return AKRA_OK;
}

// Lane-steps a Legendre launch executes against the steps it counts.  One block per (m, chunk)
// with the kernels' layout of ring pairs: synthesis pair (chunk P + k) NT + tid; adjoint pair
// chunk P NT + warp 32 P + k 32 + lane.  A warp computes all 32 P of its slots from the first
// l-tile (64-step tiles from the block's earliest start) that holds its earliest start, to lmax;
// the counted steps are each live pair's own, from its start to lmax.
__global__ void k_lane_steps(const int2 *__restrict__ start, const int *__restrict__ units, int nunits,
                             int nunit_all, int L, int P, int nchunks, int adjoint, int tile,
                             unsigned long long *out)
{
    __shared__ int s_first;
    const int m = blockIdx.x / nchunks, chunk = blockIdx.x - m * nchunks;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, NT = blockDim.x;
    if (tid == 0) s_first = kNeverLive;
    __syncthreads();
    int my_first = kNeverLive;
    unsigned long long counted = 0;
    for (int k = 0; k < P; k++) {
        const long long iu = adjoint ? (long long)chunk * P * NT + warp * 32 * P + k * 32 + lane
                                     : ((long long)chunk * P + k) * NT + tid;
        int g = kNeverLive;
        if (iu < nunits) g = start[(size_t)m * nunit_all + units[iu]].x;
        if (g <= L) counted += (unsigned long long)(L - g + 1);
        my_first = min(my_first, g);
    }
    const int warp_first = __reduce_min_sync(0xffffffffu, my_first);
    atomicMin(&s_first, my_first);
    __syncthreads();
    const int l_first = s_first;
    for (int o = 16; o > 0; o >>= 1) counted += __shfl_xor_sync(0xffffffffu, counted, o);
    if (lane == 0) {
        atomicAdd(&out[1], counted);
        if (warp_first <= L) {
            const int t0 = l_first + (warp_first - l_first) / tile * tile;
            atomicAdd(&out[0], 32ull * P * (unsigned long long)(L - t0 + 1));
        }
    }
}

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_legendre_lane_steps(akra_plan p, akra_prec prec, int adjoint, int P, int NT,
                                                long long *lane_steps, long long *steps)
{
    if (!p || !lane_steps || !steps || (prec != AKRA_F64 && prec != AKRA_F32) || P < 1 || P > 64 ||
        NT < 32 || NT > 1024 || NT % 32 != 0) {
        set_error("akra_legendre_lane_steps: invalid argument");
        return AKRA_EINVAL;
    }
    AKRA_TRY(reject_flat(p, "akra_legendre_lane_steps"));
    *lane_steps = *steps = 0;
    const int *units = p->has_weights ? p->d_active_units : p->d_all_units;
    const int nunits = p->has_weights ? p->n_active_units : p->nunit;
    if (nunits <= 0) return AKRA_OK;
    const int nchunks = (nunits + P * NT - 1) / (P * NT);
    unsigned long long *d = nullptr, h[2] = {0, 0};
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_legendre_lane_steps: allocation failed");
        return AKRA_ENOMEM;
    }
    cudaMemset(d, 0, sizeof(h));
    k_lane_steps<<<(p->lmax + 1) * nchunks, NT>>>(prec == AKRA_F32 ? p->d_start32 : p->d_start64, units, nunits,
                                                 p->nunit, p->lmax, P, nchunks, adjoint ? 1 : 0, 64, d);
    const cudaError_t e1 = cudaGetLastError();
    const cudaError_t e2 = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    AKRA_CUDA_TRY(e1);
    AKRA_CUDA_TRY(e2);
    *lane_steps = (long long)h[0];
    *steps = (long long)h[1];
    return AKRA_OK;
}

extern "C" akra_status akra_fma_rate(akra_prec prec, double *tflops)
{
    if (!tflops || (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_fma_rate: invalid argument");
        return AKRA_EINVAL;
    }
    return prec == AKRA_F32 ? fma_rate<float>(tflops) : fma_rate<double>(tflops);
}
