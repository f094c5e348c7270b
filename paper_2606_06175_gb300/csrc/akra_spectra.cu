// akra_spectra.cu -- the noise-realisation pipeline's device steps (Sec. IV, "Power spectrum
// results"): shuffling the observed shear among the unmasked pixels, and the E/B auto and
// cross power spectra of reconstructed convergence alm with their band powers.
#include "akra_internal.cuh"

namespace akra {

// out[r][c][p] = shear[c][perm[r][p]]; an index outside [0, npix) yields 0 and is counted
template <typename T>
__global__ void k_shuffle(long long npix, int R, const T *__restrict__ shear,
                          const int *__restrict__ perm, T *__restrict__ out, int *bad)
{
    const long long n = (long long)R * npix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / npix, p = i - r * npix;
        const int q = perm[i];
        T g1 = 0, g2 = 0;
        if (q >= 0 && q < npix) {
            g1 = shear[q];
            g2 = shear[npix + q];
        } else {
            atomicAdd(bad, 1);
        }
        out[(r * 2 + 0) * npix + p] = g1;
        out[(r * 2 + 1) * npix + p] = g2;
    }
}

// C_l^{XY} = [Re a_X,l0 Re b_Y,l0 + 2 Re Σ_{m>0} a_X,lm conj(b_Y,lm)] / (2l + 1), X, Y in {E, B},
// accumulated in FP64; one thread per (l, r): for a fixed m the threads read consecutive l
template <typename T>
__global__ void k_cl(int L, long long ntri, int R, const cx_t<T> *__restrict__ a,
                     const cx_t<T> *__restrict__ b, double *__restrict__ cl)
{
    const int l = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (l > L) return;
    const cx_t<T> *aE = a + ((size_t)r * 2 + 0) * ntri, *aB = a + ((size_t)r * 2 + 1) * ntri;
    const cx_t<T> *bE = b + ((size_t)r * 2 + 0) * ntri, *bB = b + ((size_t)r * 2 + 1) * ntri;
    double s[4] = {0, 0, 0, 0};
    for (int m = 0; m <= l; m++) {
        const long long ix = (long long)m * (2 * L + 1 - m) / 2 + l;
        const cx_t<T> xe = aE[ix], xb = aB[ix], ye = bE[ix], yb = bB[ix];
        if (m == 0) {
            s[0] += (double)xe.x * ye.x;
            s[1] += (double)xe.x * yb.x;
            s[2] += (double)xb.x * ye.x;
            s[3] += (double)xb.x * yb.x;
        } else {
            s[0] += 2.0 * ((double)xe.x * ye.x + (double)xe.y * ye.y);
            s[1] += 2.0 * ((double)xe.x * yb.x + (double)xe.y * yb.y);
            s[2] += 2.0 * ((double)xb.x * ye.x + (double)xb.y * ye.y);
            s[3] += 2.0 * ((double)xb.x * yb.x + (double)xb.y * yb.y);
        }
    }
    const double inv = 1.0 / (2.0 * l + 1.0);
    for (int k = 0; k < 4; k++) cl[((size_t)r * 4 + k) * (L + 1) + l] = s[k] * inv;
}

constexpr int kMaxBins = 64;
struct Edges {
    int nb;
    double e[kMaxBins + 1];
};

// band power b = mean of C_l over l in (e_b, e_{b+1}] (0 for a bin holding no l)
__global__ void k_bands(int L, int R, const double *__restrict__ cl, Edges ed, double *__restrict__ out)
{
    const int bin = blockIdx.x, k = blockIdx.y % 4, r = blockIdx.y / 4;
    __shared__ double s_sum[256];
    __shared__ int s_cnt[256];
    double sum = 0;
    int cnt = 0;
    for (int l = threadIdx.x; l <= L; l += blockDim.x) {
        if ((double)l > ed.e[bin] && (double)l <= ed.e[bin + 1]) {
            sum += cl[((size_t)r * 4 + k) * (L + 1) + l];
            cnt++;
        }
    }
    s_sum[threadIdx.x] = sum;
    s_cnt[threadIdx.x] = cnt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s_sum[threadIdx.x] += s_sum[threadIdx.x + o];
            s_cnt[threadIdx.x] += s_cnt[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) out[((size_t)r * 4 + k) * ed.nb + bin] = s_cnt[0] ? s_sum[0] / s_cnt[0] : 0.0;
}

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_shuffle_shear(akra_plan p, akra_prec prec, const void *d_shear,
                                          const int *d_perm, void *d_out, int R, void *stream)
{
    if (!p || !d_shear || !d_perm || !d_out || R < 1 || (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_shuffle_shear: invalid argument");
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    int *bad = nullptr;
    if (cudaMalloc(&bad, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_shuffle_shear: allocation failed");
        return AKRA_ENOMEM;
    }
    cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (prec == AKRA_F64)
        k_shuffle<double><<<1216, 256, 0, st>>>(p->npix, R, (const double *)d_shear, d_perm, (double *)d_out, bad);
    else
        k_shuffle<float><<<1216, 256, 0, st>>>(p->npix, R, (const float *)d_shear, d_perm, (float *)d_out, bad);
    cudaError_t e = cudaGetLastError();
    int h_bad = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(bad);
    AKRA_CUDA_TRY(e);
    p->launches++;
    if (h_bad) {
        set_error("akra_shuffle_shear: %d permutation entries outside [0, npix)", h_bad);
        return AKRA_EINVAL;
    }
    return AKRA_OK;
}

extern "C" akra_status akra_cl_spectra(akra_plan p, akra_prec prec, const void *d_a, const void *d_b,
                                       int R, int nbins, const double *edges, double *d_out, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_cl_spectra"));
    if (!p || !d_a || !d_b || !d_out || R < 1 || R > 65535 || (prec != AKRA_F64 && prec != AKRA_F32) ||
        nbins < 0 || nbins > kMaxBins || (nbins > 0 && !edges)) {
        set_error("akra_cl_spectra: invalid argument (at most %d bins)", kMaxBins);
        return AKRA_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int L = p->lmax;
    double *cl = d_out;
    if (nbins > 0) {
        AKRA_TRY(ws_reserve(p, p->red_cl, (size_t)R * 4 * (L + 1) * sizeof(double)));
        cl = (double *)p->red_cl.ptr;
    }
    dim3 grid((L + 1 + 127) / 128, R);
    if (prec == AKRA_F64)
        k_cl<double><<<grid, 128, 0, st>>>(L, p->ntri, R, (const double2 *)d_a, (const double2 *)d_b, cl);
    else
        k_cl<float><<<grid, 128, 0, st>>>(L, p->ntri, R, (const float2 *)d_a, (const float2 *)d_b, cl);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    if (nbins > 0) {
        Edges ed{};
        ed.nb = nbins;
        for (int i = 0; i <= nbins; i++) ed.e[i] = edges[i];
        k_bands<<<dim3(nbins, 4 * R), 256, 0, st>>>(L, R, cl, ed, d_out);
        AKRA_CUDA_TRY(cudaGetLastError());
        p->launches++;
    }
    return AKRA_OK;
}
