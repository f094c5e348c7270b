// akra_cg.cu -- (preconditioned) conjugate gradients on H = A^T W A + λ_eff I
// (Sec. II B "The inversion problem"; Eq. 14 regulariser; Eq. 15 scalar preconditioner),
// plain FP64 / FP32 and FP32-inner with FP64 iterative refinement.
//
// One CG iteration is a fixed kernel sequence captured once into a CUDA graph:
//   q = H p  (Legendre synthesis, ring FFT x W x FFT, Legendre adjoint, epilogue + λ_eff p)
//   <p,q>  -> α = <r,z>/<p,q>                               (FP64 accumulation)
//   x += α p, r -= α q, <r,r> -> stop test, β                (FP64 accumulation)
//   p = P r + β p
// Every kernel returns at once when the device flag `all_done` is set, so the host can
// launch iterations ahead and only polls the flag (bounded by a wall-clock budget).
// Dot products use the real-dof metric: <x,y> = Σ_l [x_l0 y_l0 + 2 Re Σ_{m>0} x conj(y)].
#include <algorithm>
#include <chrono>
#include <mutex>
#include <thread>

#include "akra_cg_impl.cuh"

namespace akra {

// ---------------------------------------------------------------------------
// vector kernels
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ double wdot(bool m0, cx_t<T> a, cx_t<T> b)
{
    // m = 0 entries count once and are real; m > 0 twice
    return m0 ? (double)a.x * (double)b.x : 2.0 * ((double)a.x * (double)b.x + (double)a.y * (double)b.y);
}

// FP32 vectors: the element's product in FP32 (relative rounding 2^-24, far below the FP32 CG's
// inner tolerances), the sums in FP64 -- one conversion per element instead of four, which the
// FP64 pipe executes
template <>
__device__ __forceinline__ double wdot<float>(bool m0, float2 a, float2 b)
{
    return (double)(m0 ? a.x * b.x : 2.f * fmaf(a.x, b.x, a.y * b.y));
}

// block-reduce one double per slot into scratch[k * RED_NB + blockIdx.x]; returns true on the
// last block to finish (which may then read every partial)
__device__ bool block_partials(double *vals, int nslots, double *scratch, CgCtl *ctl)
{
    __shared__ double sh[RED_NT];
    __shared__ bool last;
    for (int r = 0; r < nslots; r++) {
        sh[threadIdx.x] = vals[r];
        __syncthreads();
        for (int off = RED_NT / 2; off > 0; off >>= 1) {
            if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) scratch[(size_t)r * RED_NB + blockIdx.x] = sh[0];
        __syncthreads();
    }
    __threadfence();
    if (threadIdx.x == 0) last = atomicAdd(&ctl->counter, 1) == (int)gridDim.x - 1;
    __syncthreads();
    return last;
}

// in the last block: the total of every slot, summed by all threads in a fixed order (the
// partials are read past L1, they were written by other blocks), into tot[0..nslots)
__device__ void block_totals(const double *scratch, int nslots, double *tot)
{
    __shared__ double sh[RED_NT];
    for (int r = 0; r < nslots; r++) {
        double s = 0;
        for (int b = threadIdx.x; b < RED_NB; b += RED_NT) s += __ldcg(scratch + (size_t)r * RED_NB + b);
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int off = RED_NT / 2; off > 0; off >>= 1) {
            if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) tot[r] = sh[0];
        __syncthreads();
    }
}

constexpr int kMaxRhsLocal = 64;

// per-element preconditioner weights when the plan uses the per-l diagonal, else nullptr
template <typename T> static const T *pw_ptr(akra_plan p);
template <> const double *pw_ptr<double>(akra_plan p) { return p->precond_kind ? p->d_pw64 : nullptr; }
template <> const float *pw_ptr<float>(akra_plan p) { return p->precond_kind ? p->d_pw32 : nullptr; }

// Grid-stride walk over the packed index j of both fields of RHS r: element o = (2r + f) ntri + j
// (no division per element); j <= L are the m = 0 entries.
#define AKRA_FOR_RHS_ELEMENTS(r)                                                                     \
    for (int f_ = 0; f_ < 2; f_++)                                                                   \
        _Pragma("unroll 4") for (long long j = blockIdx.x * (long long)RED_NT + threadIdx.x, o = ((long long)(r) * 2 + f_) * ntri + j; \
             j < ntri; j += (long long)gridDim.x * RED_NT, o += (long long)gridDim.x * RED_NT)

// preconditioner weight of packed index j: the scalar P of Eq. 15, or a per-l diagonal
template <typename T>
__device__ __forceinline__ T pweight(const T *pw, long long j, T P)
{
    return pw ? pw[j] : P;
}

// initial state: x = 0, r = b, p = z = P r, rz = <r, z>, bnorm2 = <b,b>
template <typename T>
__global__ void __launch_bounds__(RED_NT)
k_cg_init(int L, long long ntri, const cx_t<T> *b, cx_t<T> *x, cx_t<T> *r, cx_t<T> *p, CgState *st,
          CgCtl *ctl, double *scratch, double tol, int maxiter, const T *pw)
{
    const int R = ctl->R;
    const T P = (T)ctl->precond;
    double acc[2 * kMaxRhsLocal];
    for (int q = 0; q < R; q++) {
        double bb = 0, rz = 0;
        AKRA_FOR_RHS_ELEMENTS(q) {
            const cx_t<T> v = b[o];
            const T w = pweight(pw, j, P);
            const cx_t<T> z{w * v.x, w * v.y};
            x[o] = cx_t<T>{0, 0};
            r[o] = v;
            p[o] = z;
            bb += wdot<T>(j <= L, v, v);
            rz += wdot<T>(j <= L, v, z);
        }
        acc[2 * q] = bb;
        acc[2 * q + 1] = rz;
    }
    if (block_partials(acc, 2 * R, scratch, ctl)) {
        __shared__ double tot[2 * kMaxRhsLocal];
        block_totals(scratch, 2 * R, tot);
        for (int q = threadIdx.x; q < R; q += RED_NT) {
            const double bb = tot[2 * q];
            CgState s{};
            s.bnorm2 = bb;
            s.rr = bb;
            s.rz = tot[2 * q + 1];
            s.tol = tol;
            s.relres = bb > 0 ? 1.0 : 0.0;
            s.done = bb > 0 ? 0 : 1;
            s.status = AKRA_OK;
            if (!isfinite(bb)) {
                s.done = 1;
                s.status = AKRA_ENUMERIC;
            }
            st[q] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int q = 0; q < R; q++) all &= st[q].done;
            ctl->all_done = all;
            ctl->maxiter = maxiter;
            ctl->counter = 0;
        }
    }
}

// <p, q> -> α
template <typename T>
__global__ void __launch_bounds__(RED_NT)
k_cg_dot_pq(int L, long long ntri, const cx_t<T> *p, const cx_t<T> *q, CgState *st, CgCtl *ctl,
            double *scratch)
{
    if (ctl->all_done) return;
    const int R = ctl->R;
    double acc[kMaxRhsLocal];
    for (int r = 0; r < R; r++) {
        double a = 0;
        if (!st[r].done) {
            AKRA_FOR_RHS_ELEMENTS(r) a += wdot<T>(j <= L, p[o], q[o]);
        }
        acc[r] = a;
    }
    if (block_partials(acc, R, scratch, ctl)) {
        __shared__ double tot[kMaxRhsLocal];
        block_totals(scratch, R, tot);
        for (int r = threadIdx.x; r < R; r += RED_NT) {
            if (st[r].done) continue;
            const double pq = tot[r];
            st[r].pq = pq;
            if (!(pq > 0) || !isfinite(pq)) {
                st[r].status = AKRA_ENUMERIC;
                st[r].done = 1;
                st[r].alpha = 0;
            } else {
                st[r].alpha = st[r].rz / pq;
            }
        }
        if (threadIdx.x == 0) ctl->counter = 0;
    }
}

// x += α p, r -= α q, <r,r> -> relres, stop test, <r, P r> -> β
template <typename T>
__global__ void __launch_bounds__(RED_NT)
k_cg_update_xr(int L, long long ntri, const cx_t<T> *p, const cx_t<T> *q, cx_t<T> *x, cx_t<T> *rv,
               CgState *st, CgCtl *ctl, double *scratch, const T *pw)
{
    if (ctl->all_done) return;
    const int R = ctl->R;
    double acc[2 * kMaxRhsLocal];
    for (int r = 0; r < R; r++) {
        double a = 0, az = 0;
        if (!st[r].done) {
            const T al = (T)st[r].alpha;
            AKRA_FOR_RHS_ELEMENTS(r) {
                const cx_t<T> pv = p[o], qv = q[o];
                cx_t<T> xv = x[o], rr = rv[o];
                xv.x = fma(al, pv.x, xv.x);
                xv.y = fma(al, pv.y, xv.y);
                rr.x = fma(-al, qv.x, rr.x);
                rr.y = fma(-al, qv.y, rr.y);
                x[o] = xv;
                rv[o] = rr;
                const double d = wdot<T>(j <= L, rr, rr);
                a += d;
                if (pw) az += (double)pw[j] * d;
            }
        }
        acc[2 * r] = a;
        acc[2 * r + 1] = az;
    }
    if (block_partials(acc, 2 * R, scratch, ctl)) {
        __shared__ double tot[2 * kMaxRhsLocal];
        block_totals(scratch, 2 * R, tot);
        const double P = ctl->precond;
        for (int r = threadIdx.x; r < R; r += RED_NT) {
            CgState s = st[r];
            if (s.done) continue;
            const double rr = tot[2 * r];
            s.rr = rr;
            s.iters += 1;
            s.relres = sqrt(rr / s.bnorm2);
            const double rz_new = pw ? tot[2 * r + 1] : P * rr;
            s.beta = rz_new / s.rz;
            s.rz = rz_new;
            if (!isfinite(rr)) {
                s.status = AKRA_ENUMERIC;
                s.done = 1;
            } else if (s.relres < s.tol) {
                s.done = 1;
            } else if (s.iters >= ctl->maxiter) {
                s.status = AKRA_ENOCONV;
                s.done = 1;
            }
            st[r] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int all = 1;
            for (int r = 0; r < R; r++) all &= st[r].done;
            ctl->all_done = all;
            ctl->counter = 0;
        }
    }
}

// p = P r + β p
template <typename T>
__global__ void __launch_bounds__(RED_NT)
k_cg_update_p(long long ntri, const cx_t<T> *rv, cx_t<T> *p, const CgState *st, const CgCtl *ctl,
              const T *pw)
{
    if (ctl->all_done) return;
    const int R = ctl->R;
    const T P = (T)ctl->precond;
    for (int r = 0; r < R; r++) {
        if (st[r].done) continue;
        const T b = (T)st[r].beta;
        AKRA_FOR_RHS_ELEMENTS(r) {
            const T w = pweight(pw, j, P);
            const cx_t<T> rr = rv[o];
            cx_t<T> pv = p[o];
            pv.x = fma(b, pv.x, w * rr.x);
            pv.y = fma(b, pv.y, w * rr.y);
            p[o] = pv;
        }
    }
}

// out = b - h; per-RHS ||out||^2 and ||b||^2 into res[2r], res[2r+1] (FP64 accumulation)
template <typename T>
__global__ void __launch_bounds__(RED_NT)
k_residual(int L, long long ntri, int R, const cx_t<T> *b, const cx_t<T> *h, cx_t<T> *out,
           double *res, CgCtl *ctl, double *scratch)
{
    double acc[2 * kMaxRhsLocal];
    for (int r = 0; r < R; r++) {
        double a = 0, ab = 0;
        AKRA_FOR_RHS_ELEMENTS(r) {
            const cx_t<T> bv = b[o], hv = h[o];
            const cx_t<T> d{bv.x - hv.x, bv.y - hv.y};
            if (out) out[o] = d;
            a += wdot<T>(j <= L, d, d);
            ab += wdot<T>(j <= L, bv, bv);
        }
        acc[2 * r] = a;
        acc[2 * r + 1] = ab;
    }
    if (block_partials(acc, 2 * R, scratch, ctl)) {
        __shared__ double tot[2 * kMaxRhsLocal];
        block_totals(scratch, 2 * R, tot);
        for (int q = threadIdx.x; q < 2 * R; q += RED_NT) res[q] = tot[q];
        if (threadIdx.x == 0) ctl->counter = 0;
    }
}

// r32 = (float) (r64 * s_r), s_r = 1/||r64_r||  (per RHS scale from res[2r])
__global__ void k_cast_scaled(long long n, int R, const double2 *r64, const double *res, float2 *r32)
{
    for (int r = 0; r < R; r++) {
        const double nr = sqrt(res[2 * r]);
        const double s = nr > 0 ? 1.0 / nr : 0.0;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const double2 v = r64[(size_t)r * n + i];
            r32[(size_t)r * n + i] = make_float2((float)(v.x * s), (float)(v.y * s));
        }
    }
}

// x64 += ||r64_r|| * d32
__global__ void k_axpy_mixed(long long n, int R, const float2 *d32, const double *res, double2 *x64)
{
    for (int r = 0; r < R; r++) {
        const double nr = sqrt(res[2 * r]);
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
             i += (long long)gridDim.x * blockDim.x) {
            const float2 d = d32[(size_t)r * n + i];
            double2 x = x64[(size_t)r * n + i];
            x.x += nr * (double)d.x;
            x.y += nr * (double)d.y;
            x64[(size_t)r * n + i] = x;
        }
    }
}

akra_status cg_reserve(akra_plan p, int R, CgBufs &b)
{
    if (R > kMaxRhsLocal) {
        set_error("CG: at most %d right-hand sides per solve", kMaxRhsLocal);
        return AKRA_EINVAL;
    }
    const size_t V64 = (size_t)R * 2 * p->ntri * sizeof(double2);
    const size_t V32 = (size_t)R * 2 * p->ntri * sizeof(float2);
    AKRA_TRY(ws_reserve(p, p->cg, 5 * V64 + 5 * V32));
    const size_t nst = (size_t)kMaxRhsLocal;
    const size_t red = 2 * nst * sizeof(CgState) + 2 * 64 + (size_t)RED_NB * 2 * nst * sizeof(double) +
                       2 * nst * sizeof(double);
    AKRA_TRY(ws_reserve(p, p->red, red));
    char *c = (char *)p->cg.ptr;
    for (int i = 0; i < 5; i++) b.v64[i] = c + i * V64;
    for (int i = 0; i < 5; i++) b.v32[i] = c + 5 * V64 + i * V32;
    char *d = (char *)p->red.ptr;
    b.st[0] = (CgState *)d;
    b.st[1] = (CgState *)(d + nst * sizeof(CgState));
    b.ctl[0] = (CgCtl *)(d + 2 * nst * sizeof(CgState));
    b.ctl[1] = (CgCtl *)(d + 2 * nst * sizeof(CgState) + 64);
    b.scratch = (double *)(d + 2 * nst * sizeof(CgState) + 128);
    b.res = b.scratch + (size_t)RED_NB * 2 * nst;
    if (!p->h_pinned) {
        if (cudaMallocHost(&p->h_pinned, 2 * nst * sizeof(CgState) + 256 + 2 * nst * sizeof(double)) !=
            cudaSuccess) {
            cudaGetLastError();
            set_error("CG: pinned host allocation failed");
            return AKRA_ENOMEM;
        }
    }
    return AKRA_OK;
}


// capture (or reuse) the graph of one CG iteration for precision T and R RHS
template <typename T>
static akra_status cg_graph(akra_plan p, int R, CgBufs &b, cudaGraphExec_t *out)
{
    const long long key = ((long long)p->fields << 40) | ((long long)PrecIdx<T>::v << 32) | (long long)R;
    CgGraph *g = p->graphs.count(key) ? p->graphs[key] : nullptr;
    if (g && g->exec && g->gen == p->ws_gen) {
        *out = g->exec;
        return AKRA_OK;
    }
    if (!g) {
        g = new CgGraph();
        p->graphs[key] = g;
    }
    if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    // reserve the operator workspaces before capture (no allocation may happen inside)
    const LegShape s = leg_shape(p, PrecIdx<T>::v == 0 ? AKRA_F64 : AKRA_F32, R);
    if (is_flat(p))   // the flat-sky operator's two transpose buffers
        AKRA_TRY(ws_reserve(p, p->phi, 2 * (size_t)R * p->npix * sizeof(cx_t<T>)));
    else
        AKRA_TRY(ws_reserve(p, p->phi, (size_t)R * p->nring * (2 * (size_t)p->lmax + 1) * sizeof(cx_t<T>)));
    const int nch = legendre_chunks(p->n_active_units, s);
    AKRA_TRY(ws_reserve(p, p->partial, (size_t)nch * R * p->ntri * 4 * sizeof(T)));
    if (PrecIdx<T>::v == 1 && !is_flat(p)) AKRA_TRY(tc_reserve(p, s.TC, R));
    AKRA_TRY(cg_reserve(p, R, b));   // pointers are stable now (nothing grows below)
    void **v = vecs<T>(b);
    CgState *st = b.st[PrecIdx<T>::v];
    CgCtl *ctl = b.ctl[PrecIdx<T>::v];
    cudaStream_t cs = p->stream;
    AKRA_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    p->cur_skip = &ctl->all_done;
    const long long launched_before = p->launches;   // capturing launches nothing
    akra_status s1 = op_H<T>(p, v[3], v[4], R, cs);
    p->cur_skip = nullptr;
    p->launches = launched_before;
    if (s1 == AKRA_OK) s1 = cg_launch_tail<T>(p, b, cs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (s1 != AKRA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s1;
    }
    AKRA_CUDA_TRY(e);
    size_t nnodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nnodes);
    g->kernels = (long long)nnodes;   // every captured node is a kernel launch
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    AKRA_CUDA_TRY(e);
    g->gen = p->ws_gen;
    *out = g->exec;
    return AKRA_OK;
}

// process-wide solver settings
static std::mutex g_settings_mu;
static double g_timeout_s = 3600.0;
static MixedPolicy g_mixed{0.0, 0.5};
constexpr double kMaxTimeout = 1e9;   // seconds (about 32 years)

MixedPolicy mixed_policy()
{
    std::lock_guard<std::mutex> lock(g_settings_mu);
    return g_mixed;
}

void set_mixed_policy(MixedPolicy mp)
{
    std::lock_guard<std::mutex> lock(g_settings_mu);
    g_mixed = mp;
}

std::chrono::steady_clock::time_point solve_deadline()
{
    double s;
    {
        std::lock_guard<std::mutex> lock(g_settings_mu);
        s = g_timeout_s;
    }
    // s is finite and in (0, 1e9] (akra_set_timeout), so the microsecond count fits
    return std::chrono::steady_clock::now() + std::chrono::microseconds((long long)(s * 1e6));
}

// MIXED inner tolerance: max(floor, min(0.1, factor · tol / current FP64 residual)).
// floor <= 0 selects the automatic floor, the FP32 operator's own accuracy (below it the FP32
// CG gains nothing on the FP64 residual): 0.1 · 2^-24 · lmax, within [5e-6, 1e-3].
double inner_tol(const MixedPolicy &mp, int lmax, double tol, double worst)
{
    const double fl = mp.floor > 0 ? mp.floor
                                   : std::min(1e-3, std::max(5e-6, 0.1 * 0x1p-24 * (double)lmax));
    return std::max(fl, std::min(0.1, mp.factor * tol / worst));
}

// wait for the event with a wall-clock budget (no unbounded device wait)
akra_status bounded_wait(cudaEvent_t ev, std::chrono::steady_clock::time_point deadline)
{
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return AKRA_OK;
        if (e != cudaErrorNotReady) {
            set_error("CG: %s", cudaGetErrorString(e));
            return AKRA_ECUDA;
        }
        if (std::chrono::steady_clock::now() > deadline) {
            set_error("CG: wall-clock budget exhausted");
            return AKRA_ETIMEOUT;
        }
        std::this_thread::yield();
    }
}

// run CG for precision T on the plan-owned vectors (b already in slot 0); returns the per-RHS
// states in host memory hst[R]
template <typename T>
static akra_status cg_run(akra_plan p, int R, CgBufs &b, double tol, int maxiter, CgState *hst,
                          std::chrono::steady_clock::time_point deadline)
{
    cudaGraphExec_t exec;
    AKRA_TRY(cg_graph<T>(p, R, b, &exec));
    const long long per_iter =
        p->graphs[((long long)p->fields << 40) | ((long long)PrecIdx<T>::v << 32) | (long long)R]->kernels;
    void **v = vecs<T>(b);
    CgState *st = b.st[PrecIdx<T>::v];
    CgCtl *ctl = b.ctl[PrecIdx<T>::v];
    cudaStream_t cs = p->stream;
    AKRA_TRY(cg_launch_init<T>(p, R, b, tol, maxiter, cs));
    int *h_done = (int *)p->h_pinned;
    int launched = 0;
    int chunk = 2;
    while (launched < maxiter) {
        const int k = std::min(chunk, maxiter - launched);
        for (int i = 0; i < k; i++) AKRA_CUDA_TRY(cudaGraphLaunch(exec, cs));
        p->launches += per_iter * k;
        launched += k;
        AKRA_CUDA_TRY(cudaMemcpyAsync(h_done, &ctl->all_done, sizeof(int), cudaMemcpyDeviceToHost, cs));
        AKRA_CUDA_TRY(cudaEventRecord(p->ev_a, cs));
        AKRA_TRY(bounded_wait(p->ev_a, deadline));
        if (*h_done) break;
        chunk = std::min(chunk * 2, 16);
    }
    AKRA_CUDA_TRY(cudaMemcpyAsync(hst, st, sizeof(CgState) * R, cudaMemcpyDeviceToHost, cs));
    AKRA_CUDA_TRY(cudaEventRecord(p->ev_a, cs));
    AKRA_TRY(bounded_wait(p->ev_a, deadline));
    return AKRA_OK;
}

// FP64 (or FP32) true residual of x against b: res[2r] = ||b - Hx||^2, res[2r+1] = ||b||^2
template <typename T>
static akra_status true_residual(akra_plan p, int R, CgBufs &b, const void *bv, const void *xv,
                                 void *tmp, void *rout, double *hres,
                                 std::chrono::steady_clock::time_point deadline)
{
    cudaStream_t cs = p->stream;
    AKRA_TRY(op_H<T>(p, xv, tmp, R, cs));
    k_residual<T><<<RED_NB, RED_NT, 0, cs>>>(p->lmax, p->ntri, R, (const cx_t<T> *)bv,
                                             (const cx_t<T> *)tmp, (cx_t<T> *)rout, b.res,
                                             b.ctl[PrecIdx<T>::v], b.scratch);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    AKRA_CUDA_TRY(cudaMemcpyAsync(hres, b.res, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, cs));
    AKRA_CUDA_TRY(cudaEventRecord(p->ev_a, cs));
    return bounded_wait(p->ev_a, deadline);
}

static void fill_info(akra_cg_info *info, int R, const std::vector<double> &relres,
                      const std::vector<int> &iters, const std::vector<int> &status)
{
    if (!info) return;
    double mx = 0;
    int worst = AKRA_OK;
    for (int r = 0; r < R; r++) {
        mx = std::max(mx, relres[r]);
        if (status[r] != AKRA_OK && (worst == AKRA_OK || status[r] > worst)) worst = status[r];
        if (info->relres_rhs) info->relres_rhs[r] = relres[r];
        if (info->iters_rhs) info->iters_rhs[r] = iters[r];
    }
    info->relres = mx;
    info->status = worst;
}

// solve H x = b; `bsrc` is the caller's harmonic b, or nullptr when b is already in place
static akra_status solve_b(akra_plan p, akra_prec prec, const void *bsrc, void *d_x, int R, double tol,
                           int maxiter, akra_cg_info *info, cudaStream_t user, bool b_in_place,
                           CgBufs &b, int h64_already)
{
    const auto deadline = solve_deadline();
    cudaStream_t cs = p->stream;
    const size_t V64 = (size_t)R * 2 * p->ntri * sizeof(double2);
    const size_t V32 = (size_t)R * 2 * p->ntri * sizeof(float2);
    std::vector<double> relres(R, 0.0);
    std::vector<int> iters(R, 0), status(R, AKRA_OK);
    std::vector<CgState> hst(R);
    std::vector<double> hres(2 * R);
    int h64 = h64_already, h32 = 0, outer = 0, total_iters = 0;

    if (prec == AKRA_F64 || prec == AKRA_F32) {
        const bool d = prec == AKRA_F64;
        void **v = d ? b.v64 : b.v32;
        const size_t V = d ? V64 : V32;
        if (!b_in_place) AKRA_CUDA_TRY(cudaMemcpyAsync(v[0], bsrc, V, cudaMemcpyDeviceToDevice, cs));
        akra_status s = d ? cg_run<double>(p, R, b, tol, maxiter, hst.data(), deadline)
                          : cg_run<float>(p, R, b, tol, maxiter, hst.data(), deadline);
        if (s != AKRA_OK) return s;
        for (int r = 0; r < R; r++) {
            iters[r] = hst[r].iters;
            status[r] = hst[r].status;
            relres[r] = hst[r].relres;
            total_iters = std::max(total_iters, hst[r].iters);
        }
        (d ? h64 : h32) += total_iters;
        if (d) {
            // report the true FP64 residual at exit
            AKRA_TRY(true_residual<double>(p, R, b, v[0], v[1], v[4], nullptr, hres.data(), deadline));
            h64 += 1;
            for (int r = 0; r < R; r++) relres[r] = hres[2 * r + 1] > 0 ? sqrt(hres[2 * r] / hres[2 * r + 1]) : 0;
        }
        AKRA_CUDA_TRY(cudaMemcpyAsync(d_x, v[1], V, cudaMemcpyDeviceToDevice, cs));
    } else {
        // MIXED: FP64 outer residual, FP32 inner CG (iterative refinement)
        void *b64 = b.v64[0], *x64 = b.v64[1], *r64 = b.v64[2], *t64 = b.v64[3];
        if (!b_in_place) AKRA_CUDA_TRY(cudaMemcpyAsync(b64, bsrc, V64, cudaMemcpyDeviceToDevice, cs));
        AKRA_CUDA_TRY(cudaMemsetAsync(x64, 0, V64, cs));
        AKRA_CUDA_TRY(cudaMemsetAsync(t64, 0, V64, cs));
        // r = b - H·0 = b  (residual kernel with h = 0 gives ||r||, ||b||)
        k_residual<double><<<RED_NB, RED_NT, 0, cs>>>(p->lmax, p->ntri, R, (const double2 *)b64,
                                                     (const double2 *)t64, (double2 *)r64, b.res,
                                                     b.ctl[0], b.scratch);
        AKRA_CUDA_TRY(cudaGetLastError());
        p->launches++;
        // the ctl counter must be zero before the first last-block reduction
        AKRA_CUDA_TRY(cudaMemcpyAsync(hres.data(), b.res, sizeof(double) * 2 * R, cudaMemcpyDeviceToHost, cs));
        AKRA_CUDA_TRY(cudaEventRecord(p->ev_a, cs));
        AKRA_TRY(bounded_wait(p->ev_a, deadline));
        const int max_outer = 30;
        double worst = 0;
        for (int r = 0; r < R; r++) {
            relres[r] = hres[2 * r + 1] > 0 ? sqrt(hres[2 * r] / hres[2 * r + 1]) : 0;
            worst = std::max(worst, relres[r]);
        }
        int inner_budget = maxiter;
        while (worst >= tol) {
            if (outer >= max_outer || inner_budget <= 0) {
                for (int r = 0; r < R; r++)
                    if (relres[r] >= tol) status[r] = AKRA_ENOCONV;
                break;
            }
            // inner tolerance: what this outer step must gain, but not below FP32 reach
            const double tin = inner_tol(mixed_policy(), p->lmax, tol, worst);
            k_cast_scaled<<<RED_NB, RED_NT, 0, cs>>>(2 * p->ntri, R, (const double2 *)r64, b.res,
                                                     (float2 *)b.v32[0]);
            AKRA_CUDA_TRY(cudaGetLastError());
            p->launches++;
            AKRA_TRY(cg_run<float>(p, R, b, tin, inner_budget, hst.data(), deadline));
            int it = 0;
            for (int r = 0; r < R; r++) {
                it = std::max(it, hst[r].iters);
                iters[r] += hst[r].iters;
                if (hst[r].status == AKRA_ENUMERIC) status[r] = AKRA_ENUMERIC;
            }
            total_iters += it;
            h32 += it;
            inner_budget -= it;
            k_axpy_mixed<<<RED_NB, RED_NT, 0, cs>>>(2 * p->ntri, R, (const float2 *)b.v32[1], b.res,
                                                    (double2 *)x64);
            AKRA_CUDA_TRY(cudaGetLastError());
            p->launches++;
            AKRA_TRY(true_residual<double>(p, R, b, b64, x64, t64, r64, hres.data(), deadline));
            h64 += 1;
            outer += 1;
            worst = 0;
            for (int r = 0; r < R; r++) {
                relres[r] = hres[2 * r + 1] > 0 ? sqrt(hres[2 * r] / hres[2 * r + 1]) : 0;
                if (!std::isfinite(relres[r])) status[r] = AKRA_ENUMERIC;
                worst = std::max(worst, relres[r]);
            }
            bool bad = false;
            for (int r = 0; r < R; r++) bad |= status[r] == AKRA_ENUMERIC;
            if (bad) break;
        }
        AKRA_CUDA_TRY(cudaMemcpyAsync(d_x, x64, V64, cudaMemcpyDeviceToDevice, cs));
    }
    // the caller's stream continues after the copies on the internal stream
    AKRA_CUDA_TRY(cudaEventRecord(p->ev_b, cs));
    AKRA_CUDA_TRY(cudaStreamWaitEvent(user, p->ev_b, 0));
    AKRA_CUDA_TRY(cudaEventRecord(p->ev_a, cs));
    AKRA_TRY(bounded_wait(p->ev_a, deadline));
    AKRA_TRY(tc_error_check(p));
    if (info) {
        info->iters = total_iters;
        info->outer = outer;
        info->h_applies_f64 = h64;
        info->h_applies_f32 = h32;
    }
    fill_info(info, R, relres, iters, status);
    int worst = AKRA_OK;
    for (int r = 0; r < R; r++)
        if (status[r] != AKRA_OK && (worst == AKRA_OK || status[r] > worst)) worst = status[r];
    if (worst != AKRA_OK) set_error("CG: %s", worst == AKRA_ENOCONV ? "maxiter reached before tol"
                                                                    : "non-finite or non-positive curvature");
    return (akra_status)worst;
}

template <typename T>
akra_status cg_launch_init(akra_plan p, int R, CgBufs &b, double tol, int maxiter, cudaStream_t cs)
{
    void **v = vecs<T>(b);
    CgState *st = b.st[PrecIdx<T>::v];
    CgCtl *ctl = b.ctl[PrecIdx<T>::v];
    CgCtl hctl{};
    hctl.R = R;
    hctl.precond = p->precond;
    hctl.maxiter = maxiter;
    // pageable-to-device copies are staged and ordered on the stream
    AKRA_CUDA_TRY(cudaMemcpyAsync(ctl, &hctl, sizeof(CgCtl), cudaMemcpyHostToDevice, cs));
    k_cg_init<T><<<RED_NB, RED_NT, 0, cs>>>(p->lmax, p->ntri, (const cx_t<T> *)v[0], (cx_t<T> *)v[1],
                                            (cx_t<T> *)v[2], (cx_t<T> *)v[3], st, ctl, b.scratch, tol,
                                            maxiter, pw_ptr<T>(p));
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

template <typename T>
akra_status cg_launch_tail(akra_plan p, CgBufs &b, cudaStream_t cs)
{
    void **v = vecs<T>(b);
    CgState *st = b.st[PrecIdx<T>::v];
    CgCtl *ctl = b.ctl[PrecIdx<T>::v];
    k_cg_dot_pq<T><<<RED_NB, RED_NT, 0, cs>>>(p->lmax, p->ntri, (const cx_t<T> *)v[3],
                                              (const cx_t<T> *)v[4], st, ctl, b.scratch);
    k_cg_update_xr<T><<<RED_NB, RED_NT, 0, cs>>>(p->lmax, p->ntri, (const cx_t<T> *)v[3],
                                                 (const cx_t<T> *)v[4], (cx_t<T> *)v[1],
                                                 (cx_t<T> *)v[2], st, ctl, b.scratch, pw_ptr<T>(p));
    k_cg_update_p<T><<<RED_NB, RED_NT, 0, cs>>>(p->ntri, (const cx_t<T> *)v[2], (cx_t<T> *)v[3], st, ctl,
                                                pw_ptr<T>(p));
    AKRA_CUDA_TRY(cudaGetLastError());
    return AKRA_OK;
}

akra_status launch_residual64(akra_plan p, int R, CgBufs &b, const void *bv, const void *hv, void *out,
                              cudaStream_t cs)
{
    k_residual<double><<<RED_NB, RED_NT, 0, cs>>>(p->lmax, p->ntri, R, (const double2 *)bv,
                                                 (const double2 *)hv, (double2 *)out, b.res, b.ctl[0],
                                                 b.scratch);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

akra_status launch_cast_scaled(akra_plan p, int R, CgBufs &b, cudaStream_t cs)
{
    k_cast_scaled<<<RED_NB, RED_NT, 0, cs>>>(2 * p->ntri, R, (const double2 *)b.v64[2], b.res,
                                             (float2 *)b.v32[0]);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

akra_status launch_axpy_mixed(akra_plan p, int R, CgBufs &b, cudaStream_t cs)
{
    k_axpy_mixed<<<RED_NB, RED_NT, 0, cs>>>(2 * p->ntri, R, (const float2 *)b.v32[1], b.res,
                                            (double2 *)b.v64[1]);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

template akra_status cg_launch_init<float>(akra_plan, int, CgBufs &, double, int, cudaStream_t);
template akra_status cg_launch_init<double>(akra_plan, int, CgBufs &, double, int, cudaStream_t);
template akra_status cg_launch_tail<float>(akra_plan, CgBufs &, cudaStream_t);
template akra_status cg_launch_tail<double>(akra_plan, CgBufs &, cudaStream_t);

void cg_release_graphs(akra_plan p)
{
    for (auto &kv : p->graphs) {
        if (kv.second) {
            if (kv.second->exec) cudaGraphExecDestroy(kv.second->exec);
            delete kv.second;
        }
    }
    p->graphs.clear();
    if (p->h_pinned) {
        cudaFreeHost(p->h_pinned);
        p->h_pinned = nullptr;
    }
}

static akra_status check_cg(akra_plan p, akra_prec prec, const void *a, const void *x, int R, double tol,
                            int maxiter, const char *who)
{
    if (!p || !a || !x) {
        set_error("%s: NULL plan or array", who);
        return AKRA_EINVAL;
    }
    if (prec != AKRA_F64 && prec != AKRA_F32 && prec != AKRA_MIXED) {
        set_error("%s: unknown precision", who);
        return AKRA_EINVAL;
    }
    if (R < 1 || R > kMaxRhsLocal) {
        set_error("%s: R = %d outside [1, %d]", who, R, kMaxRhsLocal);
        return AKRA_EINVAL;
    }
    if (!(tol > 0) || maxiter < 1) {
        set_error("%s: tol must be > 0 and maxiter >= 1", who);
        return AKRA_EINVAL;
    }
    if (!p->has_weights) {
        set_error("%s: called before akra_plan_set_weights", who);
        return AKRA_ENOWEIGHTS;
    }
    return AKRA_OK;
}

// out = a - b over n complex entries
template <typename T>
__global__ void k_sub(long long n, const cx_t<T> *__restrict__ a, const cx_t<T> *__restrict__ b,
                      cx_t<T> *__restrict__ out)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const cx_t<T> u = a[i], v = b[i];
        out[i] = cx_t<T>{u.x - v.x, u.y - v.y};
    }
}

// zero field f (0 = E, 1 = B) of an [R][2][ntri] complex array
static akra_status zero_field(akra_plan p, void *v, size_t elem, int R, int f, cudaStream_t st)
{
    const size_t fb = (size_t)p->ntri * elem;
    AKRA_CUDA_TRY(cudaMemset2DAsync((char *)v + f * fb, 2 * fb, 0, fb, R, st));
    return AKRA_OK;
}

// copy field f of an [R][2][ntri] complex array to / from a packed [R][ntri] one
static akra_status copy_field(akra_plan p, void *dst, const void *src, size_t elem, int R, int f,
                              bool to_packed, cudaStream_t st)
{
    const size_t fb = (size_t)p->ntri * elem;
    if (to_packed)
        AKRA_CUDA_TRY(cudaMemcpy2DAsync(dst, fb, (const char *)src + f * fb, 2 * fb, fb, R,
                                        cudaMemcpyDeviceToDevice, st));
    else
        AKRA_CUDA_TRY(cudaMemcpy2DAsync((char *)dst + f * fb, 2 * fb, src, fb, fb, R,
                                        cudaMemcpyDeviceToDevice, st));
    return AKRA_OK;
}

// H acts on the given fields for the lifetime of the guard (field-restricted solves)
struct FieldGuard {
    akra_plan p;
    FieldGuard(akra_plan q, int fields) : p(q) { p->fields = fields; }
    ~FieldGuard() { p->fields = 3; }
};

// the internal stream starts after everything already queued on the caller's stream
static akra_status join_user(akra_plan p, cudaStream_t user, CgBufs &b)
{
    AKRA_CUDA_TRY(cudaEventRecord(p->ev_b, user));
    AKRA_CUDA_TRY(cudaStreamWaitEvent(p->stream, p->ev_b, 0));
    // last-block tickets start at zero
    AKRA_CUDA_TRY(cudaMemsetAsync(b.ctl[0], 0, sizeof(CgCtl), p->stream));
    AKRA_CUDA_TRY(cudaMemsetAsync(b.ctl[1], 0, sizeof(CgCtl), p->stream));
    return AKRA_OK;
}

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_set_mixed_policy(double inner_floor, double inner_factor)
{
    if (!(inner_floor >= 0) || !(inner_floor < 0.1) || !(inner_factor > 0) || !(inner_factor <= 1)) {
        set_error("akra_set_mixed_policy: need 0 <= inner_floor < 0.1 and 0 < inner_factor <= 1");
        return AKRA_EINVAL;
    }
    set_mixed_policy(MixedPolicy{inner_floor, inner_factor});
    return AKRA_OK;
}

extern "C" akra_status akra_set_timeout(double seconds)
{
    if (!(seconds > 0) || !(seconds <= kMaxTimeout)) {   // also rejects NaN and +inf
        set_error("akra_set_timeout: seconds must be finite, > 0 and <= 1e9");
        return AKRA_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_settings_mu);
    g_timeout_s = seconds;
    return AKRA_OK;
}

extern "C" akra_status akra_cg_solve_b(akra_plan p, akra_prec prec, const void *d_b, void *d_x, int R,
                                       double tol, int maxiter, akra_cg_info *info, void *stream)
{
    AKRA_TRY(check_cg(p, prec, d_b, d_x, R, tol, maxiter, "akra_cg_solve_b"));
    cudaStream_t user = (cudaStream_t)stream;
    CgBufs b;
    AKRA_TRY(cg_reserve(p, R, b));
    AKRA_TRY(join_user(p, user, b));
    StreamJoinGuard leave{p->stream, user, p->ev_b};
    return solve_b(p, prec, d_b, d_x, R, tol, maxiter, info, user, false, b, 0);
}

extern "C" akra_status akra_cg_solve(akra_plan p, akra_prec prec, const void *d_shear, void *d_x, int R,
                                     double tol, int maxiter, akra_cg_info *info, void *stream)
{
    AKRA_TRY(check_cg(p, prec, d_shear, d_x, R, tol, maxiter, "akra_cg_solve"));
    cudaStream_t user = (cudaStream_t)stream;
    CgBufs b;
    AKRA_TRY(cg_reserve(p, R, b));
    AKRA_TRY(join_user(p, user, b));
    StreamJoinGuard leave{p->stream, user, p->ev_b};
    // b = A^T W y, in FP64 unless the whole solve is FP32
    akra_status s;
    int h64 = 0;
    if (prec == AKRA_F32) {
        // the caller's shear is FP32 for an F32 solve
        s = op_adjoint<float>(p, LegMode::KS, d_shear, b.v32[0], true, R, p->stream);
    } else {
        s = op_adjoint<double>(p, LegMode::KS, d_shear, b.v64[0], true, R, p->stream);
        h64 = 1;
    }
    if (s != AKRA_OK) return s;
    // the adjoint may have grown a workspace; refresh the buffer pointers
    AKRA_TRY(cg_reserve(p, R, b));
    return solve_b(p, prec, nullptr, d_x, R, tol, maxiter, info, user, true, b, h64);
}

extern "C" akra_status akra_cg_solve_adjoint(akra_plan p, akra_prec prec, const void *d_g, void *d_u, int R,
                                             double tol, int maxiter, akra_cg_info *info, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_cg_solve_adjoint"));
    AKRA_TRY(check_cg(p, prec, d_g, d_u, R, tol, maxiter, "akra_cg_solve_adjoint"));
    cudaStream_t user = (cudaStream_t)stream;
    CgBufs b;
    AKRA_TRY(cg_reserve(p, R, b));
    AKRA_TRY(join_user(p, user, b));
    StreamJoinGuard leave{p->stream, user, p->ev_b};
    // right-hand side G^{-1} g in the solve's own precision region
    const bool dbl = prec != AKRA_F32;
    AKRA_TRY(metric_inverse(p, dbl, d_g, dbl ? b.v64[0] : b.v32[0], R, p->stream));
    return solve_b(p, prec, nullptr, d_u, R, tol, maxiter, info, user, true, b, 0);
}

extern "C" akra_status akra_cg_solve_fields(akra_plan p, akra_prec prec, akra_fields fields,
                                            const void *d_shear, void *d_x, int R, double tol,
                                            int maxiter, akra_cg_info *info, void *stream)
{
    AKRA_TRY(reject_flat(p, "akra_cg_solve_fields"));
    AKRA_TRY(check_cg(p, prec, d_shear, d_x, R, tol, maxiter, "akra_cg_solve_fields"));
    if (fields != AKRA_SOLVE_E && fields != AKRA_SOLVE_B_GIVEN_E) {
        set_error("akra_cg_solve_fields: fields must be AKRA_SOLVE_E or AKRA_SOLVE_B_GIVEN_E");
        return AKRA_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    CgBufs b;
    AKRA_TRY(cg_reserve(p, R, b));
    AKRA_TRY(join_user(p, user, b));
    StreamJoinGuard leave{p->stream, user, p->ev_b};
    cudaStream_t cs = p->stream;
    const bool dbl = prec != AKRA_F32;
    const size_t elem = dbl ? sizeof(double2) : sizeof(float2);
    // b = A^T W y (the joint right-hand side; FP64 unless the whole solve is FP32)
    akra_status s = dbl ? op_adjoint<double>(p, LegMode::KS, d_shear, b.v64[0], true, R, cs)
                        : op_adjoint<float>(p, LegMode::KS, d_shear, b.v32[0], true, R, cs);
    if (s != AKRA_OK) return s;
    AKRA_TRY(cg_reserve(p, R, b));
    void **v = dbl ? b.v64 : b.v32;
    int h64 = dbl ? 1 : 0;
    if (fields == AKRA_SOLVE_E) {
        // E-mode normal equations H_EE κ_E = b_E: B rows dropped, κ_B held at zero
        AKRA_TRY(zero_field(p, v[0], elem, R, 1, cs));
        FieldGuard guard(p, 1);
        return solve_b(p, prec, nullptr, d_x, R, tol, maxiter, info, user, true, b, h64);
    }
    // reduced B-mode equation (Eq. A8): b~_B = b_B - H_BE κ_E = [b - H (κ_E, 0)]_B
    AKRA_CUDA_TRY(cudaMemcpyAsync(v[1], d_x, (size_t)R * 2 * p->ntri * elem, cudaMemcpyDeviceToDevice, cs));
    AKRA_TRY(zero_field(p, v[1], elem, R, 1, cs));
    s = dbl ? op_H<double>(p, v[1], v[4], R, cs) : op_H<float>(p, v[1], v[4], R, cs);
    if (s != AKRA_OK) return s;
    h64 += dbl ? 1 : 0;
    const long long n = (long long)R * 2 * p->ntri;
    if (dbl)
        k_sub<double><<<RED_NB, RED_NT, 0, cs>>>(n, (const double2 *)v[0], (const double2 *)v[4], (double2 *)v[0]);
    else
        k_sub<float><<<RED_NB, RED_NT, 0, cs>>>(n, (const float2 *)v[0], (const float2 *)v[4], (float2 *)v[0]);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    AKRA_TRY(zero_field(p, v[0], elem, R, 0, cs));
    // keep κ_E aside: the solve writes the whole of d_x
    AKRA_TRY(ws_reserve(p, p->xsave, (size_t)R * p->ntri * elem));
    AKRA_TRY(cg_reserve(p, R, b));
    AKRA_TRY(copy_field(p, p->xsave.ptr, d_x, elem, R, 0, true, cs));
    {
        FieldGuard guard(p, 2);
        s = solve_b(p, prec, nullptr, d_x, R, tol, maxiter, info, user, true, b, h64);
    }
    if (s != AKRA_OK) return s;
    // the caller's stream already waits for the solve: put κ_E back after it
    return copy_field(p, d_x, p->xsave.ptr, elem, R, 0, false, user);
}
