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

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_fma_rate(akra_prec prec, double *tflops)
{
    if (!tflops || (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_fma_rate: invalid argument");
        return AKRA_EINVAL;
    }
    return prec == AKRA_F32 ? fma_rate<float>(tflops) : fma_rate<double>(tflops);
}
