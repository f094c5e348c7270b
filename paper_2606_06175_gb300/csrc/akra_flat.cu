// akra_flat.cu -- the flat-sky variant of the operator (Sec. II B: each SHT replaced by a 2D
// FFT, the four-step structure of A and the CG solver unchanged).
//
// On an n x n periodic patch the unknown is x = F z, the unitary 2D Fourier transform of the
// complex field z = κ_E + i κ_B (rows k2, columns k1, FFT frequency order), and
//   A x   = F^-1 (D x)            γ1 + i γ2 at the pixels,  D(k) = (k1² - k2² + 2i k1 k2)/|k|²
//   A^T u = conj(D) F (u1 + i u2) (the exact adjoint: F is unitary and |D| <= 1)
//   H x   = conj(D) F (W F^-1 (D x)) + λ_eff x,   W = M N^-1 on the pixels,
// the flat-sky Kaiser-Squires kernel (D(0) = 0) in place of D_l and the spin-2 SHTs.
//
// A 2D transform is a pass of row FFTs, a transpose, and a second pass of row FFTs; for H the
// second and third passes (inverse along y, ×W, forward along y) are one kernel per row of the
// transposed field, as the ring FFT fuses W between its two DFTs.  Row FFTs run in shared memory
// (radix-4/2, decimation in frequency for the inverse, in time for the forward transform);
// permutations are folded into the loads and stores.
#include "akra_internal.cuh"

namespace akra {
namespace flat {

constexpr int NT = 512;            // threads per row-FFT block
constexpr int kMaxN = 8192;        // largest grid side (FP64 rows: 139 KB of shared memory)

__host__ __device__ constexpr int slots(int n) { return n + (n >> 4); }
__device__ __forceinline__ int pd(int i) { return i + (i >> 4); }   // bank-conflict padding

// complex helpers on float2 / double2 (C)
template <typename C> __device__ __forceinline__ C cmul(C a, C b)
{
    return C{fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x)};
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <int S, typename C> __device__ __forceinline__ C mul_si(C a)   // S i a
{
    return S > 0 ? C{-a.y, a.x} : C{a.y, -a.x};
}
// e^{S 2πi t/len} from the table e^{-2πi u/n}
template <int S, typename C>
__device__ __forceinline__ C tw(const C *__restrict__ w, int t, int len, int n)
{
    C v = w[t * (n / len)];
    if (S > 0) v.y = -v.y;
    return v;
}

// in-place DIF, sign S: natural order in, bit-reversed out
template <int S, typename T>
__device__ void dif(cx_t<T> *x, int n, int logn, const cx_t<T> *__restrict__ w)
{
    int L = n;
    if (logn & 1) {
        const int h = n >> 1;
        for (int i = threadIdx.x; i < h; i += NT) {
            const cx_t<T> a = x[pd(i)], b = x[pd(i + h)];
            x[pd(i)] = cadd(a, b);
            x[pd(i + h)] = cmul(csub(a, b), tw<S>(w, i, n, n));
        }
        __syncthreads();
        L = h;
    }
    for (; L >= 4; L >>= 2) {
        const int q = L >> 2;
        for (int b = threadIdx.x; b < (n >> 2); b += NT) {
            const int blk = b / q, i = b - blk * q, t = blk * L + i;
            const cx_t<T> a0 = x[pd(t)], a1 = x[pd(t + q)], a2 = x[pd(t + 2 * q)], a3 = x[pd(t + 3 * q)];
            const cx_t<T> u0 = cadd(a0, a2), u1 = cadd(a1, a3), d0 = csub(a0, a2);
            const cx_t<T> d1 = mul_si<S>(csub(a1, a3));
            x[pd(t)] = cadd(u0, u1);
            x[pd(t + q)] = cmul(csub(u0, u1), tw<S>(w, 2 * i, L, n));
            x[pd(t + 2 * q)] = cmul(cadd(d0, d1), tw<S>(w, i, L, n));
            x[pd(t + 3 * q)] = cmul(csub(d0, d1), tw<S>(w, 3 * i, L, n));
        }
        __syncthreads();
    }
}

// in-place DIT, sign S: bit-reversed order in, natural out
template <int S, typename T>
__device__ void dit(cx_t<T> *x, int n, int logn, const cx_t<T> *__restrict__ w)
{
    const int Lmax = (logn & 1) ? (n >> 1) : n;
    for (int L = 4; L <= Lmax; L <<= 2) {
        const int q = L >> 2;
        for (int b = threadIdx.x; b < (n >> 2); b += NT) {
            const int blk = b / q, i = b - blk * q, t = blk * L + i;
            const cx_t<T> p0 = x[pd(t)], p1 = x[pd(t + q)], p2 = x[pd(t + 2 * q)], p3 = x[pd(t + 3 * q)];
            const cx_t<T> w1 = tw<S>(w, i, L, n), w2 = tw<S>(w, 2 * i, L, n);
            cx_t<T> u = cmul(p1, w2);
            const cx_t<T> u0 = cadd(p0, u), u1 = csub(p0, u);
            u = cmul(p3, w2);
            const cx_t<T> u2 = cadd(p2, u), u3 = csub(p2, u);
            const cx_t<T> v2 = cmul(u2, w1), v3 = mul_si<S>(cmul(u3, w1));
            x[pd(t)] = cadd(u0, v2);
            x[pd(t + 2 * q)] = csub(u0, v2);
            x[pd(t + q)] = cadd(u1, v3);
            x[pd(t + 3 * q)] = csub(u1, v3);
        }
        __syncthreads();
    }
    if (logn & 1) {
        const int h = n >> 1;
        for (int i = threadIdx.x; i < h; i += NT) {
            const cx_t<T> a = x[pd(i)], b = cmul(x[pd(i + h)], tw<S>(w, i, n, n));
            x[pd(i)] = cadd(a, b);
            x[pd(i + h)] = csub(a, b);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ int brev(int k, int logn) { return (int)(__brev((unsigned)k) >> (32 - logn)); }
__device__ __forceinline__ int freq(int i, int n) { return i < n / 2 ? i : i - n; }

// flat-sky Kaiser-Squires kernel at frequency indices (k1, k2)
template <typename T>
__device__ __forceinline__ cx_t<T> ks(int k1, int k2, int n)
{
    const T a = (T)freq(k1, n), b = (T)freq(k2, n);
    const T q = a * a + b * b;
    if (q == T(0)) return cx_t<T>{0, 0};
    const T inv = T(1) / q;
    return cx_t<T>{(a * a - b * b) * inv, T(2) * a * b * inv};
}

template <typename T>
struct Args {
    int n, logn;
    const cx_t<T> *w;        // twiddles e^{-2πi t/n}
    const cx_t<T> *in;       // [R][n][n]
    cx_t<T> *out;            // [R][n][n] (may equal in)
    const T *Wt;             // middle pass: [n][n] weights, transposed, scaled by 1/n^2
    const cx_t<T> *xreg;     // mode 2: x for the λ_eff term (nullptr: none)
    T lam, scale;
    const int *skip;         // device flag: return at once if set
};

// One row of one RHS per block.  MODE
//   0: ×D(k1 = column, k2 = row), inverse FFT along the row
//   1: inverse FFT, ×Wt[row][y], forward FFT (the transposed middle of H)
//   2: forward FFT, then ×conj(D(k1 = column, k2 = row)) × scale + λ x
//   3: inverse FFT, × scale
//   4: forward FFT
template <typename T, int MODE>
__global__ void __launch_bounds__(NT) k_rows(Args<T> a)
{
    if (a.skip && *a.skip) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cx_t<T> *buf = reinterpret_cast<cx_t<T> *>(smem_raw);
    const int n = a.n, logn = a.logn, row = blockIdx.x;
    const size_t base = ((size_t)blockIdx.y * n + row) * n;
    const cx_t<T> *src = a.in + base;
    cx_t<T> *dst = a.out + base;
    constexpr bool fwd_first = MODE == 2 || MODE == 4;
    for (int k = threadIdx.x; k < n; k += NT) {
        cx_t<T> v = src[k];
        if (MODE == 0) v = cmul(ks<T>(k, row, n), v);
        buf[pd(fwd_first ? brev(k, logn) : k)] = v;   // DIT reads bit-reversed order
    }
    __syncthreads();
    if (fwd_first) {
        dit<-1, T>(buf, n, logn, a.w);
    } else {
        dif<+1, T>(buf, n, logn, a.w);
        if (MODE == 1) {
            for (int k = threadIdx.x; k < n; k += NT) {
                const T wy = a.Wt[(size_t)row * n + brev(k, logn)];
                buf[pd(k)].x *= wy;
                buf[pd(k)].y *= wy;
            }
            __syncthreads();
            dit<-1, T>(buf, n, logn, a.w);
        }
    }
    for (int k = threadIdx.x; k < n; k += NT) {
        // after an inverse-only pass element k sits in bit-reversed slot brev(k)
        cx_t<T> v = buf[pd((MODE == 0 || MODE == 3) ? brev(k, logn) : k)];
        if (MODE == 2) {
            const cx_t<T> d = ks<T>(k, row, n);
            v = cmul(cx_t<T>{d.x, -d.y}, v);
            v.x *= a.scale;
            v.y *= a.scale;
            if (a.xreg) {
                const cx_t<T> xr = a.xreg[base + k];
                v.x = fma(a.lam, xr.x, v.x);
                v.y = fma(a.lam, xr.y, v.y);
            }
        } else if (MODE == 3) {
            v.x *= a.scale;
            v.y *= a.scale;
        }
        dst[k] = v;
    }
}

// out[r][j][i] = in[r][i][j] in 32 x 32 tiles
template <typename T>
__global__ void k_transpose(int n, const cx_t<T> *__restrict__ in, cx_t<T> *__restrict__ out, const int *skip)
{
    if (skip && *skip) return;
    __shared__ cx_t<T> tile[32][33];
    const size_t off = (size_t)blockIdx.z * n * n;
    const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int y = y0 + j, x = x0 + threadIdx.x;
        if (y < n && x < n) tile[j][threadIdx.x] = in[off + (size_t)y * n + x];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int y = x0 + j, x = y0 + threadIdx.x;
        if (y < n && x < n) out[off + (size_t)y * n + x] = tile[threadIdx.x][j];
    }
}

// complex [R][n²] <-> maps [R][2][n²] (γ1 = real part, γ2 = imaginary part), optional ×W
template <typename T>
__global__ void k_split(long long npix, int R, const cx_t<T> *__restrict__ z, const T *__restrict__ W, T *__restrict__ map)
{
    const long long tot = (long long)R * npix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / npix, pix = i - r * npix;
        const cx_t<T> v = z[i];
        const T wv = W ? W[pix] : T(1);
        map[(2 * r) * npix + pix] = wv * v.x;
        map[(2 * r + 1) * npix + pix] = wv * v.y;
    }
}

template <typename T>
__global__ void k_join(long long npix, int R, const T *__restrict__ map, const T *__restrict__ W, cx_t<T> *__restrict__ z)
{
    const long long tot = (long long)R * npix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / npix, pix = i - r * npix;
        const T wv = W ? W[pix] : T(1);
        z[i] = cx_t<T>{wv * map[(2 * r) * npix + pix], wv * map[(2 * r + 1) * npix + pix]};
    }
}

// per-device statistics of N^-1 and the weight tables
__global__ void k_weights(int n, const double *ninv, double *W64, float *W32, double *Wt64, float *Wt32,
                          double *stats)
{
    const long long npix = (long long)n * n;
    double s = 0, c = 0, bad = 0;
    const double scale = 1.0 / (double)npix;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix; i += (long long)gridDim.x * blockDim.x) {
        const double v = ninv[i];
        const bool ok = isfinite(v) && v >= 0;
        const double w = (ok && v > 0) ? v : 0.0;
        W64[i] = w;
        W32[i] = (float)w;
        const long long y = i / n, x = i - y * n;
        Wt64[x * n + y] = w * scale;
        Wt32[x * n + y] = (float)(w * scale);
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
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; q++) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; q++) atomicAdd(&stats[q], sh[q][0]);
}

__global__ void k_twiddles(int n, double2 *w64, float2 *w32)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) {
        double s, c;
        sincospi(-2.0 * (double)t / (double)n, &s, &c);
        w64[t] = make_double2(c, s);
        w32[t] = make_float2((float)c, (float)s);
    }
}

template <typename T> const cx_t<T> *twiddles(akra_plan p);
template <> const double2 *twiddles<double>(akra_plan p) { return p->d_ftw64; }
template <> const float2 *twiddles<float>(akra_plan p) { return p->d_ftw32; }
template <typename T> const T *wt(akra_plan p);
template <> const double *wt<double>(akra_plan p) { return p->d_fWt64; }
template <> const float *wt<float>(akra_plan p) { return p->d_fWt32; }
template <typename T> const T *wmap(akra_plan p);
template <> const double *wmap<double>(akra_plan p) { return p->d_W64; }
template <> const float *wmap<float>(akra_plan p) { return p->d_W32; }

template <typename T, int MODE>
static akra_status rows(akra_plan p, const void *in, void *out, int R, const void *xreg, double lam,
                        double scale, cudaStream_t st)
{
    Args<T> a{};
    a.n = p->nside;
    a.logn = p->flat_logn;
    a.w = twiddles<T>(p);
    a.in = (const cx_t<T> *)in;
    a.out = (cx_t<T> *)out;
    a.Wt = wt<T>(p);
    a.xreg = (const cx_t<T> *)xreg;
    a.lam = (T)lam;
    a.scale = (T)scale;
    a.skip = p->cur_skip;
    const size_t smem = (size_t)slots(a.n) * sizeof(cx_t<T>);
    k_rows<T, MODE><<<dim3(a.n, R), NT, smem, st>>>(a);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

template <typename T>
static akra_status transpose(akra_plan p, const void *in, void *out, int R, cudaStream_t st)
{
    const int n = p->nside, g = (n + 31) / 32;
    k_transpose<T><<<dim3(g, g, R), dim3(32, 8), 0, st>>>(n, (const cx_t<T> *)in, (cx_t<T> *)out, p->cur_skip);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

template <typename T>
static akra_status buffers(akra_plan p, int R, cx_t<T> **b1, cx_t<T> **b2)
{
    const size_t v = (size_t)R * p->npix;
    AKRA_TRY(ws_reserve(p, p->phi, 2 * v * sizeof(cx_t<T>)));
    *b1 = (cx_t<T> *)p->phi.ptr;
    *b2 = *b1 + v;
    return AKRA_OK;
}

}  // namespace flat

template <typename T>
akra_status flat_op_A(akra_plan p, const void *x, void *map, bool weighted, int R, cudaStream_t st)
{
    cx_t<T> *b1, *b2;
    AKRA_TRY(flat::buffers<T>(p, R, &b1, &b2));
    const double s = 1.0 / (double)p->nside;
    AKRA_TRY((flat::rows<T, 0>(p, x, b1, R, nullptr, 0.0, 1.0, st)));   // ×D, inverse along k1
    AKRA_TRY(flat::transpose<T>(p, b1, b2, R, st));
    AKRA_TRY((flat::rows<T, 3>(p, b2, b2, R, nullptr, 0.0, s, st)));   // inverse along k2, × 1/n
    AKRA_TRY(flat::transpose<T>(p, b2, b1, R, st));
    flat::k_split<T><<<1216, 256, 0, st>>>(p->npix, R, b1, weighted ? flat::wmap<T>(p) : nullptr, (T *)map);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

template <typename T>
akra_status flat_op_At(akra_plan p, const void *map, void *x, bool weighted, int R, cudaStream_t st)
{
    cx_t<T> *b1, *b2;
    AKRA_TRY(flat::buffers<T>(p, R, &b1, &b2));
    flat::k_join<T><<<1216, 256, 0, st>>>(p->npix, R, (const T *)map, weighted ? flat::wmap<T>(p) : nullptr, b1);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    AKRA_TRY(flat::transpose<T>(p, b1, b2, R, st));                            // [x][y]
    AKRA_TRY((flat::rows<T, 4>(p, b2, b2, R, nullptr, 0.0, 1.0, st)));        // forward along y
    AKRA_TRY(flat::transpose<T>(p, b2, b1, R, st));                            // [k2][x]
    return flat::rows<T, 2>(p, b1, x, R, nullptr, 0.0, 1.0 / (double)p->nside, st);   // along x, ×conj D / n
}

template <typename T>
akra_status flat_op_H(akra_plan p, const void *x, void *y, int R, cudaStream_t st)
{
    cx_t<T> *b1, *b2;
    AKRA_TRY(flat::buffers<T>(p, R, &b1, &b2));
    AKRA_TRY((flat::rows<T, 0>(p, x, b1, R, nullptr, 0.0, 1.0, st)));        // ×D, inverse along k1
    AKRA_TRY(flat::transpose<T>(p, b1, b2, R, st));
    AKRA_TRY((flat::rows<T, 1>(p, b2, b2, R, nullptr, 0.0, 1.0, st)));       // along k2: F^-1, ×W/n², F
    AKRA_TRY(flat::transpose<T>(p, b2, b1, R, st));
    return flat::rows<T, 2>(p, b1, y, R, x, p->lambda_eff, 1.0, st);          // along x, ×conj D, + λ x
}

template akra_status flat_op_A<float>(akra_plan, const void *, void *, bool, int, cudaStream_t);
template akra_status flat_op_A<double>(akra_plan, const void *, void *, bool, int, cudaStream_t);
template akra_status flat_op_At<float>(akra_plan, const void *, void *, bool, int, cudaStream_t);
template akra_status flat_op_At<double>(akra_plan, const void *, void *, bool, int, cudaStream_t);
template akra_status flat_op_H<float>(akra_plan, const void *, void *, int, cudaStream_t);
template akra_status flat_op_H<double>(akra_plan, const void *, void *, int, cudaStream_t);

akra_status flat_set_weights(akra_plan p, const double *d_ninv, double lambda, cudaStream_t st)
{
    double *d_stats = nullptr;
    if (cudaMalloc(&d_stats, 3 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_plan_set_weights: allocation failed");
        return AKRA_ENOMEM;
    }
    double h[3] = {0, 0, 0};
    cudaError_t e = cudaMemsetAsync(d_stats, 0, 3 * sizeof(double), st);
    if (e == cudaSuccess) {
        flat::k_weights<<<1216, 256, 0, st>>>(p->nside, d_ninv, p->d_W64, p->d_W32, p->d_fWt64, p->d_fWt32, d_stats);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_stats, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_stats);
    AKRA_CUDA_TRY(e);
    if (h[2] > 0) {
        set_error("akra_plan_set_weights: %.0f negative or non-finite N^-1 entries", h[2]);
        return AKRA_EINVAL;
    }
    p->lambda = lambda;
    p->omega = 1.0;
    p->lambda_eff = h[1] > 0 ? lambda * h[0] / h[1] : 0.0;
    p->precond = 1.0 / (h[0] / (double)p->npix + p->lambda_eff);
    if (!std::isfinite(p->precond)) p->precond = 1.0;
    p->has_weights = true;
    p->ws_gen++;   // captured CG iterations hold the previous λ_eff
    return AKRA_OK;
}

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_flat_plan_create(int n, akra_plan *out)
{
    if (!out) {
        set_error("akra_flat_plan_create: out is NULL");
        return AKRA_EINVAL;
    }
    *out = nullptr;
    if (n < 16 || n > flat::kMaxN || (n & (n - 1))) {
        set_error("akra_flat_plan_create: n = %d must be a power of two in [16, %d]", n, flat::kMaxN);
        return AKRA_EINVAL;
    }
    akra_plan p = new (std::nothrow) akra_plan_s();
    if (!p) {
        set_error("akra_flat_plan_create: host allocation failed");
        return AKRA_ENOMEM;
    }
    p->kind = 1;
    p->nside = n;
    p->lmax = -1;
    p->npix = (long long)n * n;
    p->ntri = p->npix / 2;
    int lg = 0;
    while ((1 << lg) < n) lg++;
    p->flat_logn = lg;
    cudaGetDevice(&p->device);
    const size_t np = (size_t)p->npix;
    auto fail = [&](const char *what) {
        cudaGetLastError();
        set_error("akra_flat_plan_create: %s", what);
        akra_plan_destroy(p);
        return AKRA_ENOMEM;
    };
    if (cudaMalloc(&p->d_ftw64, sizeof(double2) * n) != cudaSuccess ||
        cudaMalloc(&p->d_ftw32, sizeof(float2) * n) != cudaSuccess ||
        cudaMalloc(&p->d_W64, sizeof(double) * np) != cudaSuccess ||
        cudaMalloc(&p->d_W32, sizeof(float) * np) != cudaSuccess ||
        cudaMalloc(&p->d_fWt64, sizeof(double) * np) != cudaSuccess ||
        cudaMalloc(&p->d_fWt32, sizeof(float) * np) != cudaSuccess)
        return fail("table allocation failed");
    p->bytes_tables = (sizeof(double2) + sizeof(float2)) * n + 2 * (sizeof(double) + sizeof(float)) * np;
    flat::k_twiddles<<<(n + 255) / 256, 256>>>(n, p->d_ftw64, p->d_ftw32);
    cudaError_t e = cudaGetLastError();
    // row kernels: shared memory for the largest supported row, set once for every plan
    const int s64 = flat::slots(flat::kMaxN) * (int)sizeof(double2), s32 = flat::slots(flat::kMaxN) * (int)sizeof(float2);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<double, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<double, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<double, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<double, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<double, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s64);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<float, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<float, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<float, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<float, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(flat::k_rows<float, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_a, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_b, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        set_error("akra_flat_plan_create: %s", cudaGetErrorString(e));
        akra_plan_destroy(p);
        return AKRA_ECUDA;
    }
    *out = p;
    return AKRA_OK;
}
