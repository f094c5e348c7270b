// akra_ringfft32.cu -- FP32 ring phase sums (the φ half of SHT^-1 / SHT, Sec. II B) with the
// pixel diagonal W fused between them: O(n log n) for every ring length.
//
// The ring sums are the same as in akra_ringfft.cu (fold Φ(m) into n bins with phase
// e^{iπσk/n}, length-n DFT, ×W, DFT back, unfold).  Here the length-n DFTs are
//   * n a power of two: in-place radix-4/2 decimation in frequency (natural -> bit-reversed)
//     for the backward DFT and decimation in time (bit-reversed -> natural) for the forward
//     one, so W is applied to the bit-reversed pixel order and no permutation pass is needed;
//     pairs of radix-4 stages run as one pass through shared memory (each thread keeps the
//     16 elements of both stages in registers), so n = 8192 takes 4 passes instead of 7;
//   * any other n (polar rings n = 4i): Bluestein's chirp-z form,
//       X_k = conj(c_k) Σ_j [x_j conj(c_j)] c_{k-j},  c_j = e^{iπ j²/n},
//     a cyclic convolution of length M = 2^⌈log2(2n-1)⌉ done by the same DIF/DIT pair, with
//     the chirp's spectrum precomputed per ring length (stored in DIF output order).
//     The backward DFT is conj(forward(conj x)).
#include "akra_ringfft32_impl.cuh"

namespace akra {

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
        buf[pd(j)] = v;
    }
    __syncthreads();
    dif<-1>(buf, M, 31 - __clz(M), tw2);
    float2 *out = bhat_all + bhat_off[i];
    for (int j = threadIdx.x; j < M; j += blockDim.x) out[j] = buf[pd(j)];
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
    p->fft32_M_host = M;
    p->fft32_msmall = 0;
    for (int i = 1; i <= N; i++)
        if (M[i] < mmax) p->fft32_msmall = std::max(p->fft32_msmall, M[i]);
    size_t bytes = sizeof(int) * (N + 1) + sizeof(long long) * (N + 1) + sizeof(float2) * F32_MMAX +
                   sizeof(float2) * (size_t)std::max(total, 1LL);
    if (cudaMalloc(&p->d_fft32_M, sizeof(int) * (N + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_off, sizeof(long long) * (N + 1)) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_tw2, sizeof(float2) * F32_MMAX) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_bhat, sizeof(float2) * (size_t)std::max(total, 1LL)) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_rings_all, sizeof(int) * p->nring) != cudaSuccess ||
        cudaMalloc(&p->d_fft32_rings_act, sizeof(int) * p->nring) != cudaSuccess) {
        cudaGetLastError();
        set_error("ring FFT table allocation failed");
        return AKRA_ENOMEM;
    }
    p->bytes_tables += bytes + 2 * sizeof(int) * (size_t)p->nring;
    std::vector<int> all(p->nring);
    for (int r = 0; r < p->nring; r++) all[r] = r;
    AKRA_TRY(ring_fft32_order(p, all, p->d_fft32_rings_all, &p->fft32_nsmall_all));
    AKRA_TRY(ring_fft32_order(p, all, p->d_fft32_rings_act, &p->fft32_nsmall_act));
    AKRA_CUDA_TRY(cudaMemcpy(p->d_fft32_M, M.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
    AKRA_CUDA_TRY(cudaMemcpy(p->d_fft32_off, off.data(), sizeof(long long) * (N + 1), cudaMemcpyHostToDevice));
    k_tw2<<<(F32_MMAX + 255) / 256, 256>>>(p->d_fft32_tw2);
    AKRA_CUDA_TRY(cudaGetLastError());
    // kernel attributes are shared by every plan: clear the largest supported length
    const int smem_b = f32_slots(mmax) * (int)sizeof(float2);
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_bhat32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       f32_slots(F32_MMAX) * (int)sizeof(float2)));
    k_bhat32<<<N, F32_NT, smem_b>>>(N, p->d_fft32_M, p->d_fft32_off, p->d_tw64, p->d_fft32_tw2,
                                    p->d_fft32_bhat);
    AKRA_CUDA_TRY(cudaGetLastError());
    const int smem = (f32_slots(F32_MMAX) + F32_NT) * (int)sizeof(float2);
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (f32_slots(F32_MMAX) + F32_NT) * (int)sizeof(float2)));
    return AKRA_OK;
}

// Order a ring list for the FP32 FFT launches: rings whose convolution length M is at most
// fft32_msmall first (their launch reserves less shared memory, so two blocks
// fit on an SM), then those with M = fft32_mmax.  Writes the list to d_out (device).
akra_status ring_fft32_order(akra_plan p, const std::vector<int> &rings, int *d_out, int *nsmall)
{
    const int N = p->nside;
    std::vector<int> lo, hi;
    for (int r : rings) {
        const int i = r + 1;                                   // 1-based ring index
        const int n = i < N ? 4 * i : (i <= 3 * N ? 4 * N : 4 * (4 * N - i));
        const int M = p->fft32_M_host[n / 4];
        (p->fft32_msmall > 0 && M <= p->fft32_msmall ? lo : hi).push_back(r);
    }
    *nsmall = (int)lo.size();
    lo.insert(lo.end(), hi.begin(), hi.end());
    if (!lo.empty())
        AKRA_CUDA_TRY(cudaMemcpy(d_out, lo.data(), sizeof(int) * lo.size(), cudaMemcpyHostToDevice));
    return AKRA_OK;
}

Fft32Args fft32_args(akra_plan p, bool weighted, const int *rings)
{
    Fft32Args a{};
    a.L = p->lmax;
    a.nring = p->nring;
    a.mmax = p->fft32_mmax;
    a.npix = p->npix;
    a.rings = rings;
    a.rinfo = p->d_rings;
    a.fftM = p->d_fft32_M;
    a.bhat_off = p->d_fft32_off;
    a.bhat_all = p->d_fft32_bhat;
    a.tw2 = p->d_fft32_tw2;
    a.tw_all = p->d_tw32;
    a.W = p->d_W32r;
    a.weighted = weighted ? 1 : 0;
    a.skip = p->cur_skip;
    return a;
}

akra_status ring_fft32(akra_plan p, FftMode mode, void *phi, const void *map_in, void *map_out,
                       bool weighted, int R, const int *rings, int nrings, cudaStream_t st)
{
    if (nrings <= 0) return AKRA_OK;
    // the plan's own ring lists go out in two launches by convolution length
    const int *list = rings;
    int nsmall = 0;
    if (p->fft32_msmall > 0 && rings == p->d_active_rings && nrings == p->n_active_rings) {
        list = p->d_fft32_rings_act;
        nsmall = p->fft32_nsmall_act;
    } else if (p->fft32_msmall > 0 && rings == p->d_all_rings && nrings == p->nring) {
        list = p->d_fft32_rings_all;
        nsmall = p->fft32_nsmall_all;
    }
    Fft32Args a = fft32_args(p, weighted, list);
    a.phi = (float2 *)phi;
    a.map_in = (const float *)map_in;
    a.map_out = (float *)map_out;
    for (int part = 0; part < 2; part++) {
        const int cnt = part == 0 ? nsmall : nrings - nsmall;
        if (cnt <= 0) continue;
        a.rings = list + (part == 0 ? 0 : nsmall);
        a.mmax = part == 0 ? p->fft32_msmall : p->fft32_mmax;   // buffer length; scratch follows it
        const size_t smem = (size_t)(f32_slots(a.mmax) + F32_NT) * sizeof(float2);
        dim3 grid(cnt, R);
#define AKRA_F32_LAUNCH(MD) k_ring_fft32<MD><<<grid, F32_NT, smem, st>>>(a)
        switch (mode) {
        case FftMode::Synth: AKRA_F32_LAUNCH(0); break;
        case FftMode::Adjoint: AKRA_F32_LAUNCH(1); break;
        default: AKRA_F32_LAUNCH(2); break;
        }
#undef AKRA_F32_LAUNCH
        AKRA_CUDA_TRY(cudaGetLastError());
        p->launches++;
    }
    return AKRA_OK;
}

AKRA_DEBUG_COLLECTOR(ringfft32)

}  // namespace akra
