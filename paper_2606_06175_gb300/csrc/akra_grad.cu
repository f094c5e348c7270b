// akra_grad.cu -- pieces of the gradient of a loss through the CG solve x̂ = H^{-1} A^T W y.
//
// With g the gradient of the loss w.r.t. the stored (re, im) components of x̂, and G the
// real-dof metric (1 on the real part at m = 0, 0 on its ignored imaginary part, 2 at m > 0)
// in which H is self-adjoint:
//   u = H^{-1} G^{-1} g                       (implicit adjoint solve, same H and CG)
//   dL/dy_p     = W_p (A u)_p                 (akra_apply_A with weights)
//   dL/dN^-1_p  = ω M_p <(A u)_p, y_p - (A x̂)_p>   (λ_eff held fixed)
#include "akra_internal.cuh"

namespace akra {

// out = G^{-1} in: halve m > 0 entries, keep the real part at m = 0 and zero its imaginary part
template <typename T>
__global__ void k_metric_inverse(int L, long long ntri, long long n, const cx_t<T> *in, cx_t<T> *out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long idx = i % ntri;
        cx_t<T> v = in[i];
        if (idx <= L) v.y = 0;
        else {
            v.x *= T(0.5);
            v.y *= T(0.5);
        }
        out[i] = v;
    }
}

// grad_p = ω M_p Σ_r Σ_c Au[r][c][p] (y[r][c][p] - Ax[r][c][p]),  M_p = [W_p > 0]
template <typename T>
__global__ void k_weight_grad(long long npix, int R, double omega, const double *W, const T *Au,
                              const T *y, const T *Ax, T *grad)
{
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < npix;
         p += (long long)gridDim.x * blockDim.x) {
        double s = 0;
        for (int r = 0; r < R; r++)
            for (int c = 0; c < 2; c++) {
                const size_t o = ((size_t)r * 2 + c) * npix + p;
                s += (double)Au[o] * ((double)y[o] - (double)Ax[o]);
            }
        grad[p] = (T)(W[p] > 0 ? omega * s : 0.0);
    }
}

akra_status metric_inverse(akra_plan p, bool dbl, const void *in, void *out, int R, cudaStream_t st)
{
    const long long n = (long long)R * 2 * p->ntri;
    const int nb = (int)std::min<long long>((n + 255) / 256, 4096);
    if (dbl)
        k_metric_inverse<double><<<nb, 256, 0, st>>>(p->lmax, p->ntri, n, (const double2 *)in, (double2 *)out);
    else
        k_metric_inverse<float><<<nb, 256, 0, st>>>(p->lmax, p->ntri, n, (const float2 *)in, (float2 *)out);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_weight_grad(akra_plan p, akra_prec prec, const void *d_Au, const void *d_y,
                                        const void *d_Ax, void *d_grad, int R, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_weight_grad"));
    if (!p || !d_Au || !d_y || !d_Ax || !d_grad || R < 1 || R > 65535 ||
        (prec != AKRA_F64 && prec != AKRA_F32)) {
        set_error("akra_weight_grad: invalid argument");
        return AKRA_EINVAL;
    }
    if (!p->has_weights) {
        set_error("akra_weight_grad: called before akra_plan_set_weights");
        return AKRA_ENOWEIGHTS;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)std::min<long long>((p->npix + 255) / 256, 8192);
    if (prec == AKRA_F64)
        k_weight_grad<double><<<nb, 256, 0, st>>>(p->npix, R, p->omega, p->d_W64, (const double *)d_Au,
                                                  (const double *)d_y, (const double *)d_Ax, (double *)d_grad);
    else
        k_weight_grad<float><<<nb, 256, 0, st>>>(p->npix, R, p->omega, p->d_W64, (const float *)d_Au,
                                                 (const float *)d_y, (const float *)d_Ax, (float *)d_grad);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}
