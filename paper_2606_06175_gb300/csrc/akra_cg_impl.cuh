// akra_cg_impl.cuh -- CG state, workspace layout and the launchers shared by the per-plan
// solver (akra_cg.cu) and the multi-instance solver (akra_batch.cu).
#pragma once
#include <chrono>

#include "akra_internal.cuh"

namespace akra {

struct CgState {          // one per RHS (device)
    double rz, pq, alpha, beta, rr, bnorm2, relres, tol;
    int done, iters, status, pad;
};

struct CgCtl {            // one per solver precision (device)
    int all_done;         // read by every iteration kernel
    int counter;          // last-block ticket
    int maxiter;
    int R;
    double precond;
};

constexpr int RED_NB = 608;    // vector-kernel blocks (4 per SM on 152 SMs)
constexpr int RED_NT = 256;

struct CgGraph {
    cudaGraphExec_t exec = nullptr;
    unsigned gen = 0;
    long long kernels = 0;   // kernel nodes of one captured iteration
};

// ---------------------------------------------------------------------------
// workspace layout (plan->cg): FP64 region of 5 vectors, FP32 region of 5 vectors
//   F64 CG:  b x r p q in the FP64 region
//   F32 CG and the MIXED inner CG: b x r p q in the FP32 region
//   MIXED outer: b64 x64 r64 t64 in the FP64 region (slots 0..3)
// plan->red: [CgState R] x 2 precisions, CgCtl x 2, scratch doubles, residual doubles
// ---------------------------------------------------------------------------
struct CgBufs {
    void *v64[5];
    void *v32[5];
    CgState *st[2];
    CgCtl *ctl[2];
    double *scratch;
    double *res;
};

template <typename T> struct PrecIdx;
template <> struct PrecIdx<double> { static constexpr int v = 0; };
template <> struct PrecIdx<float> { static constexpr int v = 1; };

template <typename T>
inline void **vecs(CgBufs &b) { return PrecIdx<T>::v == 0 ? b.v64 : b.v32; }

// process-wide settings (set from any thread).  The mixed-precision policy is one pair,
// written and read under a lock, so a solve never sees a floor from one call of
// akra_set_mixed_policy with the factor of another; a solve reads it once per outer step.
struct MixedPolicy {
    double floor;    // <= 0: the automatic floor (the FP32 operator's own accuracy)
    double factor;
};
MixedPolicy mixed_policy();
void set_mixed_policy(MixedPolicy mp);
// inner FP32 tolerance of an outer step: max(floor, min(0.1, factor tol / worst))
double inner_tol(const MixedPolicy &mp, int lmax, double tol, double worst);
// the wall-clock deadline of a blocking solve that starts now (budget of akra_set_timeout)
std::chrono::steady_clock::time_point solve_deadline();

// Orders the caller's stream after everything queued so far on an internal stream, on every
// return path (normal, error or ETIMEOUT) of a blocking call that queued work there: the
// caller may then free or reuse its buffers in stream order, even while copies or CG
// iterations launched before an early return are still running.
struct StreamJoinGuard {
    cudaStream_t from, to;
    cudaEvent_t ev;
    ~StreamJoinGuard()
    {
        if (cudaEventRecord(ev, from) == cudaSuccess) cudaStreamWaitEvent(to, ev, 0);
    }
};
akra_status cg_reserve(akra_plan p, int R, CgBufs &b);
akra_status bounded_wait(cudaEvent_t ev, std::chrono::steady_clock::time_point deadline);
// x = 0, r = b (slot 0), p = P r, state and ctl initialised (precision T region)
template <typename T>
akra_status cg_launch_init(akra_plan p, int R, CgBufs &b, double tol, int maxiter, cudaStream_t cs);
// the three vector kernels that follow q = H p in one iteration
template <typename T> akra_status cg_launch_tail(akra_plan p, CgBufs &b, cudaStream_t cs);
// res[2r] = ||b - h||^2, res[2r+1] = ||b||^2 (FP64), out = b - h (may be nullptr)
akra_status launch_residual64(akra_plan p, int R, CgBufs &b, const void *bv, const void *hv, void *out,
                              cudaStream_t cs);
// FP32 right-hand side r64/||r64|| into slot 0 of the FP32 region; x64 += ||r64|| d32
akra_status launch_cast_scaled(akra_plan p, int R, CgBufs &b, cudaStream_t cs);
akra_status launch_axpy_mixed(akra_plan p, int R, CgBufs &b, cudaStream_t cs);

}  // namespace akra
