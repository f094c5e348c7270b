// akra_batch.cu -- several plans (uneven Nside / lmax, several RHS each) solved together:
// every FP32 H application of the inner CG is one persistent Legendre-synthesis launch over
// the work items of all instances (a queue of (instance, m, chunk, RHS group) items ordered
// by cost, heaviest first), one ring-FFT launch over all instances' rings, one persistent
// Legendre-adjoint launch, then each instance's epilogue and CG vector kernels -- all in one
// CUDA graph per iteration.  The synthesis can instead run on the tensor cores (its own queue of
// (instance, m, 128-pair chunk, RHS group) items; the adjoint keeps the CUDA-core items).  The FP64 outer refinement of the mixed-precision form runs per
// instance between inner solves.  (Motivated by the paper's noise realisations and
// tomographic bins, Sec. III; the batching itself is not in the paper.)
#include <algorithm>
#include <chrono>
#include <cstring>

#include "akra_cg_impl.cuh"
#include "akra_legendre_impl.cuh"
#include "akra_ringfft32_impl.cuh"

struct akra_batch_s {
    int ninst = 0;
    std::vector<akra_plan> plans;
    std::vector<int> R;
    akra::LegShape shape{1, 128, 4};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    akra::LegArgs<float> *d_syn = nullptr, *d_adj = nullptr;
    akra::Fft32Args *d_fft = nullptr;
    int4 *d_items = nullptr, *d_fitems = nullptr;
    int nitems = 0, nfitems = 0;
    int *d_counter = nullptr;             // queue heads: synthesis, adjoint, tensor-core synthesis
    int tcg = 0;                          // tensor-core synthesis RHS group (0: CUDA-core synthesis)
    akra::LegArgs<float> *d_syn_tc = nullptr;
    std::vector<akra::LegArgs<float>> h_syn_tc;   // host copies: the B-operand staging launches
    int4 *d_titems = nullptr;
    int ntitems = 0, titems_tcg = 0;
    int fft_mmax = 0;
    size_t fft_smem_set = 48 * 1024;     // dynamic shared memory the FFT kernel is cleared for
    akra::LegShape items_shape{0, 0, 0};
    std::vector<int> nch;                 // Legendre chunks per instance (current shape)
    cudaGraphExec_t graph = nullptr;
    std::vector<unsigned> graph_gens;
    long long graph_kernels = 0;
    akra::LegShape graph_shape{0, 0, 0};
    int graph_tcg = 0;
    int *h_flags = nullptr;               // pinned: one done flag per instance
    long long launches = 0;
};

namespace akra {

static int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// (re)build the work-item lists for the batch's Legendre shape
static akra_status batch_items(akra_batch b)
{
    const LegShape s = b->shape;
    if (b->d_items && s.P == b->items_shape.P && s.RG == b->items_shape.RG && s.NT == b->items_shape.NT)
        return AKRA_OK;
    struct It { long long cost; int4 v; };
    std::vector<It> items;
    std::vector<int4> fitems;
    b->nch.assign(b->ninst, 0);
    b->fft_mmax = 0;
    for (int i = 0; i < b->ninst; i++) {
        akra_plan p = b->plans[i];
        const int nu = p->n_active_units, per = s.NT * s.P;
        const int nch = (nu + per - 1) / per, ng = (b->R[i] + s.RG - 1) / s.RG;
        b->nch[i] = nch;
        for (int m = 0; m <= p->lmax; m++)
            for (int c = 0; c < nch; c++)
                for (int g = 0; g < ng; g++) {
                    const long long units = std::min(per, nu - c * per);
                    const long long rg = std::min(s.RG, b->R[i] - g * s.RG);
                    const long long steps = p->lmax - std::max(m, 2) + 1;
                    items.push_back({steps * units * (6 + 8 * rg), make_int4(i, m, c, g)});
                }
        for (int k = 0; k < p->n_active_rings; k++)
            for (int r = 0; r < b->R[i]; r++) fitems.push_back(make_int4(i, k, r, 0));
        b->fft_mmax = std::max(b->fft_mmax, p->fft32_mmax);
    }
    std::stable_sort(items.begin(), items.end(), [](const It &a, const It &c) { return a.cost > c.cost; });
    std::vector<int4> hv(items.size());
    for (size_t k = 0; k < items.size(); k++) hv[k] = items[k].v;
    if (b->d_items) cudaFree(b->d_items);
    if (b->d_fitems) cudaFree(b->d_fitems);
    b->d_items = b->d_fitems = nullptr;
    if (cudaMalloc(&b->d_items, sizeof(int4) * std::max<size_t>(hv.size(), 1)) != cudaSuccess ||
        cudaMalloc(&b->d_fitems, sizeof(int4) * std::max<size_t>(fitems.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_batch: work-list allocation failed");
        return AKRA_ENOMEM;
    }
    AKRA_CUDA_TRY(cudaMemcpy(b->d_items, hv.data(), sizeof(int4) * hv.size(), cudaMemcpyHostToDevice));
    AKRA_CUDA_TRY(cudaMemcpy(b->d_fitems, fitems.data(), sizeof(int4) * fitems.size(), cudaMemcpyHostToDevice));
    b->nitems = (int)hv.size();
    b->nfitems = (int)fitems.size();
    b->items_shape = s;
    return AKRA_OK;
}

// (re)build the tensor-core synthesis items: (instance, m, 128-pair chunk, RHS group), heaviest first
static akra_status batch_titems(akra_batch b)
{
    if (b->tcg == 0 || (b->d_titems && b->titems_tcg == b->tcg)) return AKRA_OK;
    struct It { long long cost; int4 v; };
    std::vector<It> items;
    for (int i = 0; i < b->ninst; i++) {
        akra_plan p = b->plans[i];
        const int nu = p->n_active_units;
        const int nch = (nu + TC_NT - 1) / TC_NT, ng = (b->R[i] + b->tcg - 1) / b->tcg;
        for (int m = 0; m <= p->lmax; m++)
            for (int c = 0; c < nch; c++)
                for (int g = 0; g < ng; g++) {
                    const long long steps = p->lmax - std::max(m, 2) + 1;
                    items.push_back({steps * std::min(TC_NT, nu - c * TC_NT), make_int4(i, m, c, g)});
                }
    }
    std::stable_sort(items.begin(), items.end(), [](const It &a, const It &c) { return a.cost > c.cost; });
    std::vector<int4> hv(items.size());
    for (size_t k = 0; k < items.size(); k++) hv[k] = items[k].v;
    if (b->d_titems) cudaFree(b->d_titems);
    b->d_titems = nullptr;
    if (cudaMalloc(&b->d_titems, sizeof(int4) * std::max<size_t>(hv.size(), 1)) != cudaSuccess) {
        cudaGetLastError();
        set_error("akra_batch: work-list allocation failed");
        return AKRA_ENOMEM;
    }
    AKRA_CUDA_TRY(cudaMemcpy(b->d_titems, hv.data(), sizeof(int4) * hv.size(), cudaMemcpyHostToDevice));
    b->ntitems = (int)hv.size();
    b->titems_tcg = b->tcg;
    return AKRA_OK;
}

// FP32 workspaces of every instance for the batch shape, and FP64 ones for the outer residual
static akra_status batch_reserve(akra_batch b)
{
    AKRA_TRY(batch_items(b));
    AKRA_TRY(batch_titems(b));
    for (int i = 0; i < b->ninst; i++) {
        akra_plan p = b->plans[i];
        const int R = b->R[i];
        const LegShape s64 = leg_shape(p, AKRA_F64, R);
        const size_t nch64 = legendre_chunks(p->n_active_units, s64);
        const size_t part = std::max((size_t)b->nch[i] * R * p->ntri * 4 * sizeof(float),
                                     nch64 * R * p->ntri * 4 * sizeof(double));
        AKRA_TRY(ws_reserve(p, p->phi, (size_t)R * p->nring * (2 * (size_t)p->lmax + 1) * sizeof(double2)));
        AKRA_TRY(ws_reserve(p, p->partial, part));
        AKRA_TRY(tc_reserve(p, b->tcg, R));
        CgBufs cb;
        AKRA_TRY(cg_reserve(p, R, cb));
    }
    return AKRA_OK;
}

// upload the per-instance argument blocks for x[i] -> y[i] with the given skip flags
static akra_status batch_args(akra_batch b, void *const *x, void *const *y, const int *const *skips,
                              cudaStream_t st)
{
    std::vector<LegArgs<float>> syn(b->ninst), adj(b->ninst), syn_tc(b->ninst);
    std::vector<Fft32Args> fft(b->ninst);
    for (int i = 0; i < b->ninst; i++) {
        akra_plan p = b->plans[i];
        const int *sk = skips ? skips[i] : nullptr;
        syn[i] = leg_args<float>(p, b->shape, LegMode::KS, p->d_active_units, p->n_active_units, b->R[i]);
        syn[i].alm = (const float2 *)x[i];
        syn[i].phi = (float2 *)p->phi.ptr;
        syn[i].skip = sk;
        syn_tc[i] = leg_args<float>(p, LegShape{1, TC_NT, b->tcg > 0 ? b->tcg : 4}, LegMode::KS,
                                    p->d_active_units, p->n_active_units, b->R[i]);
        syn_tc[i].alm = syn[i].alm;
        syn_tc[i].phi = syn[i].phi;
        syn_tc[i].skip = sk;
        syn_tc[i].bpre = (const float *)p->bpre.ptr;
        syn_tc[i].tc_groups = b->tcg > 0 ? (b->R[i] + b->tcg - 1) / b->tcg : 0;
        adj[i] = syn[i];
        adj[i].phi_in = (const float2 *)p->phi.ptr;
        adj[i].partial = (float *)p->partial.ptr;
        fft[i] = fft32_args(p, true, p->d_active_rings);
        fft[i].phi = (float2 *)p->phi.ptr;
        fft[i].skip = sk;
    }
    (void)y;
    AKRA_CUDA_TRY(cudaMemcpyAsync(b->d_syn, syn.data(), sizeof(LegArgs<float>) * b->ninst, cudaMemcpyHostToDevice, st));
    AKRA_CUDA_TRY(cudaMemcpyAsync(b->d_adj, adj.data(), sizeof(LegArgs<float>) * b->ninst, cudaMemcpyHostToDevice, st));
    AKRA_CUDA_TRY(cudaMemcpyAsync(b->d_fft, fft.data(), sizeof(Fft32Args) * b->ninst, cudaMemcpyHostToDevice, st));
    AKRA_CUDA_TRY(cudaMemcpyAsync(b->d_syn_tc, syn_tc.data(), sizeof(LegArgs<float>) * b->ninst,
                                  cudaMemcpyHostToDevice, st));
    b->h_syn_tc = syn_tc;
    // the pageable sources must stay alive until the copies have been staged
    AKRA_CUDA_TRY(cudaStreamSynchronize(st));
    return AKRA_OK;
}

template <int P, int RG>
static akra_status launch_queue_pair(akra_batch b, int which, cudaStream_t st)
{
    constexpr int NT = 128;
    int per_sm = 0;
    const int nsm = num_sms();
    if (which == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leg_synth_queue<float, P, RG, NT>, NT, 0);
        const int grid = std::max(1, std::min(b->nitems, nsm * std::max(per_sm, 1)));
        k_leg_synth_queue<float, P, RG, NT><<<grid, NT, 0, st>>>(b->d_syn, b->d_items, b->nitems, b->d_counter);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_leg_adjoint_queue<float, P, RG, NT>, NT, 0);
        const int grid = std::max(1, std::min(b->nitems, nsm * std::max(per_sm, 1)));
        k_leg_adjoint_queue<float, P, RG, NT><<<grid, NT, 0, st>>>(b->d_adj, b->d_items, b->nitems,
                                                                   b->d_counter + 1);
    }
    AKRA_CUDA_TRY(cudaGetLastError());
    b->launches++;
    return AKRA_OK;
}

static akra_status launch_queue(akra_batch b, int which, cudaStream_t st)
{
    const LegShape s = b->shape;
#define AKRA_Q(PP, RR) if (s.P == PP && s.RG == RR) return launch_queue_pair<PP, RR>(b, which, st);
    AKRA_Q(1, 1) AKRA_Q(2, 1) AKRA_Q(4, 1) AKRA_Q(5, 1) AKRA_Q(6, 1) AKRA_Q(1, 2) AKRA_Q(2, 2) AKRA_Q(1, 4)
#undef AKRA_Q
    set_error("akra_batch: no kernel for P=%d RG=%d", s.P, s.RG);
    return AKRA_EINVAL;
}

// one batched FP32 H: y[i] = H_i x[i] for every instance (args already uploaded)
static akra_status batch_H32(akra_batch b, void *const *x, void *const *y, const int *const *skips,
                             cudaStream_t st)
{
    AKRA_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, 3 * sizeof(int), st));
    if (b->tcg > 0) {
        for (int i = 0; i < b->ninst; i++) {
            AKRA_TRY(legendre_tc_bstage(b->tcg, b->h_syn_tc[i], st));
            b->launches++;
        }
        if (b->ntitems > 0) {
            AKRA_TRY(legendre_synth_tc_queue(b->tcg, b->d_syn_tc, b->d_titems, b->ntitems, b->d_counter + 2, st));
            b->launches++;
        }
    } else {
        AKRA_TRY(launch_queue(b, 0, st));
    }
    const size_t smem = (size_t)(f32_slots(b->fft_mmax) + F32_NT) * sizeof(float2);
    if (smem > b->fft_smem_set) {
        // the attribute belongs to this translation unit's instance of the kernel
        AKRA_CUDA_TRY(cudaFuncSetAttribute(k_ring_fft32_batch<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        b->fft_smem_set = smem;
    }
    if (b->nfitems > 0) {
        k_ring_fft32_batch<2><<<b->nfitems, F32_NT, smem, st>>>(b->d_fft, b->d_fitems, b->fft_mmax);
        AKRA_CUDA_TRY(cudaGetLastError());
        b->launches++;
    }
    AKRA_TRY(launch_queue(b, 1, st));
    for (int i = 0; i < b->ninst; i++) {
        akra_plan p = b->plans[i];
        p->cur_skip = skips ? skips[i] : nullptr;
        const akra_status s = adjoint_epilogue<float>(p, LegMode::KS, p->partial.ptr, b->nch[i], x[i],
                                                      p->lambda_eff, y[i], b->R[i], st);
        p->cur_skip = nullptr;
        if (s != AKRA_OK) return s;
    }
    return AKRA_OK;
}

static bool graph_valid(akra_batch b)
{
    if (!b->graph) return false;
    const LegShape s = b->shape, g = b->graph_shape;
    if (s.P != g.P || s.RG != g.RG || s.NT != g.NT || b->tcg != b->graph_tcg) return false;
    for (int i = 0; i < b->ninst; i++)
        if (b->graph_gens[i] != b->plans[i]->ws_gen) return false;
    return true;
}

// capture one batched FP32 CG iteration (q = H p, then each instance's vector kernels)
static akra_status batch_graph(akra_batch b, std::vector<CgBufs> &cb)
{
    if (graph_valid(b)) return AKRA_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    std::vector<void *> xs(b->ninst), ys(b->ninst);
    std::vector<const int *> sk(b->ninst);
    for (int i = 0; i < b->ninst; i++) {
        xs[i] = cb[i].v32[3];
        ys[i] = cb[i].v32[4];
        sk[i] = &cb[i].ctl[1]->all_done;
    }
    AKRA_TRY(batch_args(b, xs.data(), ys.data(), sk.data(), b->stream));
    // capturing launches nothing: keep the launch counters as they are
    const long long b_launches = b->launches;
    std::vector<long long> p_launches(b->ninst);
    for (int i = 0; i < b->ninst; i++) p_launches[i] = b->plans[i]->launches;
    AKRA_CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    akra_status s = batch_H32(b, xs.data(), ys.data(), sk.data(), b->stream);
    for (int i = 0; i < b->ninst && s == AKRA_OK; i++) s = cg_launch_tail<float>(b->plans[i], cb[i], b->stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    b->launches = b_launches;
    for (int i = 0; i < b->ninst; i++) b->plans[i]->launches = p_launches[i];
    if (s != AKRA_OK) {
        if (graph) cudaGraphDestroy(graph);
        return s;
    }
    AKRA_CUDA_TRY(e);
    size_t nnodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nnodes);
    b->graph_kernels = (long long)nnodes;   // every captured node is a kernel launch
    const cudaError_t e2 = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    AKRA_CUDA_TRY(e2);
    b->graph_shape = b->shape;
    b->graph_tcg = b->tcg;
    b->graph_gens.resize(b->ninst);
    for (int i = 0; i < b->ninst; i++) b->graph_gens[i] = b->plans[i]->ws_gen;
    return AKRA_OK;
}

// run the batched FP32 CG on every instance whose slot-0 right-hand side is set; `active[i]`
// false leaves instance i untouched (its CG is marked done before the first iteration)
static akra_status batch_cg32(akra_batch b, std::vector<CgBufs> &cb, const std::vector<double> &tol,
                              const std::vector<char> &active, int maxiter,
                              std::vector<std::vector<CgState>> &hst,
                              std::chrono::steady_clock::time_point deadline)
{
    cudaStream_t st = b->stream;
    AKRA_TRY(batch_graph(b, cb));
    for (int i = 0; i < b->ninst; i++) {
        if (active[i]) {
            AKRA_TRY(cg_launch_init<float>(b->plans[i], b->R[i], cb[i], tol[i], maxiter, st));
        } else {
            // any nonzero value marks the instance's FP32 iteration as finished
            AKRA_CUDA_TRY(cudaMemsetAsync(&cb[i].ctl[1]->all_done, 1, sizeof(int), st));
        }
    }
    int launched = 0, chunk = 2;
    while (launched < maxiter) {
        const int k = std::min(chunk, maxiter - launched);
        for (int j = 0; j < k; j++) AKRA_CUDA_TRY(cudaGraphLaunch(b->graph, st));
        b->launches += (long long)k * b->graph_kernels;
        launched += k;
        for (int i = 0; i < b->ninst; i++)
            AKRA_CUDA_TRY(cudaMemcpyAsync(&b->h_flags[i], &cb[i].ctl[1]->all_done, sizeof(int),
                                          cudaMemcpyDeviceToHost, st));
        AKRA_CUDA_TRY(cudaEventRecord(b->ev, st));
        AKRA_TRY(bounded_wait(b->ev, deadline));
        bool all = true;
        for (int i = 0; i < b->ninst; i++) all &= b->h_flags[i] != 0;
        if (all) break;
        chunk = std::min(chunk * 2, 16);
    }
    hst.resize(b->ninst);
    for (int i = 0; i < b->ninst; i++) {
        hst[i].resize(b->R[i]);
        AKRA_CUDA_TRY(cudaMemcpyAsync(hst[i].data(), cb[i].st[1], sizeof(CgState) * b->R[i],
                                      cudaMemcpyDeviceToHost, st));
    }
    AKRA_CUDA_TRY(cudaEventRecord(b->ev, st));
    return bounded_wait(b->ev, deadline);
}

AKRA_DEBUG_COLLECTOR(batch)

}  // namespace akra

using namespace akra;

extern "C" akra_status akra_batch_create(int ninst, const akra_plan *plans, const int *R, akra_batch *out)
{
    if (!out || ninst < 1 || !plans || !R) {
        set_error("akra_batch_create: invalid argument");
        return AKRA_EINVAL;
    }
    *out = nullptr;
    for (int i = 0; i < ninst; i++) {
        if (!plans[i] || R[i] < 1 || R[i] > 64) {
            set_error("akra_batch_create: instance %d has no plan or R outside [1, 64]", i);
            return AKRA_EINVAL;
        }
        AKRA_TRY(reject_flat(plans[i], "akra_batch_create"));
        if (!plans[i]->has_weights) {
            set_error("akra_batch_create: plan %d has no weights (akra_plan_set_weights)", i);
            return AKRA_ENOWEIGHTS;
        }
        for (int j = 0; j < i; j++)
            if (plans[j] == plans[i]) {
                set_error("akra_batch_create: plan %d appears twice (use R for several RHS)", i);
                return AKRA_EINVAL;
            }
    }
    akra_batch b = new (std::nothrow) akra_batch_s();
    if (!b) {
        set_error("akra_batch_create: host allocation failed");
        return AKRA_ENOMEM;
    }
    b->ninst = ninst;
    b->plans.assign(plans, plans + ninst);
    b->R.assign(R, R + ninst);
    const int maxR = *std::max_element(b->R.begin(), b->R.end());
    b->shape = maxR >= 4 ? LegShape{1, 128, 4} : maxR >= 2 ? LegShape{2, 128, 2} : LegShape{4, 128, 1};
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) == cudaSuccess &&
              cudaMalloc(&b->d_syn, sizeof(LegArgs<float>) * ninst) == cudaSuccess &&
              cudaMalloc(&b->d_adj, sizeof(LegArgs<float>) * ninst) == cudaSuccess &&
              cudaMalloc(&b->d_fft, sizeof(Fft32Args) * ninst) == cudaSuccess &&
              cudaMalloc(&b->d_syn_tc, sizeof(LegArgs<float>) * ninst) == cudaSuccess &&
              cudaMalloc(&b->d_counter, 3 * sizeof(int)) == cudaSuccess &&
              cudaMallocHost(&b->h_flags, sizeof(int) * ninst) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        akra_batch_destroy(b);
        set_error("akra_batch_create: allocation failed");
        return AKRA_ENOMEM;
    }
    *out = b;
    return AKRA_OK;
}

extern "C" void akra_batch_destroy(akra_batch b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    void *ptrs[] = {b->d_syn, b->d_adj, b->d_fft, b->d_items, b->d_fitems, b->d_counter, b->d_syn_tc, b->d_titems};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (b->h_flags) cudaFreeHost(b->h_flags);
    if (b->ev) cudaEventDestroy(b->ev);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

static akra_status join(akra_batch b, cudaStream_t user)
{
    AKRA_CUDA_TRY(cudaEventRecord(b->ev, user));
    AKRA_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev, 0));
    return AKRA_OK;
}

static akra_status leave(akra_batch b, cudaStream_t user)
{
    AKRA_CUDA_TRY(cudaEventRecord(b->ev, b->stream));
    AKRA_CUDA_TRY(cudaStreamWaitEvent(user, b->ev, 0));
    return AKRA_OK;
}

extern "C" akra_status akra_batch_apply_H(akra_batch b, const void *const *d_x, void *const *d_y,
                                          void *stream)
{
    if (!b || !d_x || !d_y) {
        set_error("akra_batch_apply_H: invalid argument");
        return AKRA_EINVAL;
    }
    for (int i = 0; i < b->ninst; i++)
        if (!d_x[i] || !d_y[i] || d_x[i] == d_y[i]) {
            set_error("akra_batch_apply_H: instance %d has a NULL or aliased vector", i);
            return AKRA_EINVAL;
        }
    cudaStream_t user = (cudaStream_t)stream;
    AKRA_TRY(batch_reserve(b));
    AKRA_TRY(join(b, user));
    AKRA_TRY(batch_args(b, (void *const *)d_x, d_y, nullptr, b->stream));
    AKRA_TRY(batch_H32(b, (void *const *)d_x, d_y, nullptr, b->stream));
    return leave(b, user);
}

extern "C" akra_status akra_batch_autotune(akra_batch b, void *stream)
{
    if (!b) {
        set_error("akra_batch_autotune: invalid argument");
        return AKRA_EINVAL;
    }
    cudaStream_t user = (cudaStream_t)stream;
    std::vector<LegShape> cands = {{1, 128, 4}, {2, 128, 2}, {1, 128, 2}, {4, 128, 1}, {5, 128, 1}, {6, 128, 1},
                                   {2, 128, 1}};
    const int maxR = *std::max_element(b->R.begin(), b->R.end());
    std::vector<void *> xs(b->ninst), ys(b->ninst);
    for (int i = 0; i < b->ninst; i++) {
        akra_plan p = b->plans[i];
        const size_t bytes = (size_t)b->R[i] * 2 * p->ntri * sizeof(float2);
        if (cudaMalloc(&xs[i], bytes) != cudaSuccess || cudaMalloc(&ys[i], bytes) != cudaSuccess) {
            cudaGetLastError();
            for (void *q : xs) if (q) cudaFree(q);
            for (void *q : ys) if (q) cudaFree(q);
            set_error("akra_batch_autotune: scratch allocation failed");
            return AKRA_ENOMEM;
        }
        cudaMemsetAsync(xs[i], 0, bytes, user);
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    LegShape pick = b->shape;
    int pick_tcg = b->tcg;
    akra_status s = AKRA_OK;
    // every (tile shape, synthesis) pair: the CUDA-core synthesis (group 0) and, from R = 4 on,
    // the tensor-core one with groups up to twice the largest RHS count (the shape then serves
    // the adjoint alone)
    for (int g : {0, 4, 8, 16, 32}) {
        if (g > 0 && (maxR < 4 || g > 2 * maxR)) continue;
        for (auto &c : cands) {
            if (s != AKRA_OK) break;
            if (c.RG > maxR && c.RG > 1) continue;
            b->shape = c;
            b->tcg = g;
            s = batch_reserve(b);
            if (s == AKRA_OK) s = batch_args(b, xs.data(), ys.data(), nullptr, user);
            float tot = 0;
            for (int rep = 0; rep < 3 && s == AKRA_OK; rep++) {
                cudaEventRecord(e0, user);
                s = batch_H32(b, xs.data(), ys.data(), nullptr, user);
                cudaEventRecord(e1, user);
                cudaEventSynchronize(e1);
                float ms = 0;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;
            }
            if (s == AKRA_OK && tot < best) {
                best = tot;
                pick = c;
                pick_tcg = g;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(user);
    for (void *q : xs) cudaFree(q);
    for (void *q : ys) cudaFree(q);
    b->shape = pick;
    b->tcg = pick_tcg;
    if (s != AKRA_OK) return s;
    for (int i = 0; i < b->ninst; i++) AKRA_TRY(tc_error_check(b->plans[i]));
    return batch_reserve(b);
}

extern "C" akra_status akra_batch_set_tc_synthesis(akra_batch b, int group)
{
    if (!b || (group != 0 && group != 4 && group != 8 && group != 16 && group != 32)) {
        set_error("akra_batch_set_tc_synthesis: invalid argument (group 0, 4, 8, 16 or 32)");
        return AKRA_EINVAL;
    }
    b->tcg = group;
    return batch_reserve(b);
}

extern "C" akra_status akra_batch_get_tc_synthesis(akra_batch b, int *group)
{
    if (!b || !group) {
        set_error("akra_batch_get_tc_synthesis: invalid argument");
        return AKRA_EINVAL;
    }
    *group = b->tcg;
    return AKRA_OK;
}

extern "C" akra_status akra_batch_cg_solve(akra_batch b, akra_prec prec, const void *const *d_shear,
                                           void *const *d_x, double tol, int maxiter, akra_cg_info *info,
                                           void *stream)
{
    if (!b || !d_shear || !d_x || !(tol > 0) || maxiter < 1 || (prec != AKRA_MIXED && prec != AKRA_F32)) {
        set_error("akra_batch_cg_solve: invalid argument (precision must be AKRA_MIXED or AKRA_F32)");
        return AKRA_EINVAL;
    }
    const auto deadline = solve_deadline();
    cudaStream_t user = (cudaStream_t)stream;
    const int n = b->ninst;
    AKRA_TRY(batch_reserve(b));
    std::vector<CgBufs> cb(n);
    for (int i = 0; i < n; i++) AKRA_TRY(cg_reserve(b->plans[i], b->R[i], cb[i]));
    AKRA_TRY(join(b, user));
    StreamJoinGuard leave_guard{b->stream, user, b->ev};
    cudaStream_t st = b->stream;
    for (int i = 0; i < n; i++) {
        AKRA_CUDA_TRY(cudaMemsetAsync(cb[i].ctl[0], 0, sizeof(CgCtl), st));
        AKRA_CUDA_TRY(cudaMemsetAsync(cb[i].ctl[1], 0, sizeof(CgCtl), st));
    }
    std::vector<std::vector<double>> relres(n);
    std::vector<std::vector<int>> iters(n), status(n);
    std::vector<int> outer(n, 0), h64(n, 0), h32(n, 0), total(n, 0);
    std::vector<std::vector<CgState>> hst;
    std::vector<double> hres;
    for (int i = 0; i < n; i++) {
        relres[i].assign(b->R[i], 0.0);
        iters[i].assign(b->R[i], 0);
        status[i].assign(b->R[i], AKRA_OK);
    }
    if (prec == AKRA_F32) {
        for (int i = 0; i < n; i++)
            AKRA_TRY(op_adjoint<float>(b->plans[i], LegMode::KS, d_shear[i], cb[i].v32[0], true, b->R[i], st));
        std::vector<double> tl(n, tol);
        std::vector<char> act(n, 1);
        AKRA_TRY(batch_cg32(b, cb, tl, act, maxiter, hst, deadline));
        for (int i = 0; i < n; i++) {
            for (int r = 0; r < b->R[i]; r++) {
                iters[i][r] = hst[i][r].iters;
                status[i][r] = hst[i][r].status;
                relres[i][r] = hst[i][r].relres;
                total[i] = std::max(total[i], hst[i][r].iters);
            }
            h32[i] = total[i];
            AKRA_CUDA_TRY(cudaMemcpyAsync(d_x[i], cb[i].v32[1], (size_t)b->R[i] * 2 * b->plans[i]->ntri * sizeof(float2),
                                          cudaMemcpyDeviceToDevice, st));
        }
    } else {
        // b = A^T W y in FP64; x = 0; r = b
        for (int i = 0; i < n; i++) {
            akra_plan p = b->plans[i];
            const size_t V64 = (size_t)b->R[i] * 2 * p->ntri * sizeof(double2);
            AKRA_TRY(op_adjoint<double>(p, LegMode::KS, d_shear[i], cb[i].v64[0], true, b->R[i], st));
            h64[i] = 1;
            AKRA_CUDA_TRY(cudaMemsetAsync(cb[i].v64[1], 0, V64, st));
            AKRA_CUDA_TRY(cudaMemsetAsync(cb[i].v64[3], 0, V64, st));
            AKRA_TRY(launch_residual64(p, b->R[i], cb[i], cb[i].v64[0], cb[i].v64[3], cb[i].v64[2], st));
            hres.assign(2 * b->R[i], 0.0);
            AKRA_CUDA_TRY(cudaMemcpyAsync(hres.data(), cb[i].res, sizeof(double) * 2 * b->R[i],
                                          cudaMemcpyDeviceToHost, st));
            AKRA_CUDA_TRY(cudaEventRecord(b->ev, st));
            AKRA_TRY(bounded_wait(b->ev, deadline));
            for (int r = 0; r < b->R[i]; r++)
                relres[i][r] = hres[2 * r + 1] > 0 ? sqrt(hres[2 * r] / hres[2 * r + 1]) : 0.0;
        }
        int budget = maxiter;
        for (int round = 0; round < 30; round++) {
            const MixedPolicy mp = mixed_policy();
            std::vector<char> act(n, 0);
            std::vector<double> tl(n, tol);
            bool any = false;
            for (int i = 0; i < n; i++) {
                const double w = *std::max_element(relres[i].begin(), relres[i].end());
                bool bad = false;
                for (int r = 0; r < b->R[i]; r++) bad |= status[i][r] == AKRA_ENUMERIC;
                if (w >= tol && !bad) {
                    act[i] = 1;
                    any = true;
                    tl[i] = inner_tol(mp, b->plans[i]->lmax, tol, w);
                }
            }
            if (!any || budget <= 0) break;
            for (int i = 0; i < n; i++)
                if (act[i]) AKRA_TRY(launch_cast_scaled(b->plans[i], b->R[i], cb[i], st));
            AKRA_TRY(batch_cg32(b, cb, tl, act, budget, hst, deadline));
            int used = 0;
            for (int i = 0; i < n; i++) {
                if (!act[i]) continue;
                akra_plan p = b->plans[i];
                int it = 0;
                for (int r = 0; r < b->R[i]; r++) {
                    it = std::max(it, hst[i][r].iters);
                    iters[i][r] += hst[i][r].iters;
                    if (hst[i][r].status == AKRA_ENUMERIC) status[i][r] = AKRA_ENUMERIC;
                }
                used = std::max(used, it);
                total[i] += it;
                h32[i] += it;
                AKRA_TRY(launch_axpy_mixed(p, b->R[i], cb[i], st));
                AKRA_TRY(op_H<double>(p, cb[i].v64[1], cb[i].v64[3], b->R[i], st));
                AKRA_TRY(launch_residual64(p, b->R[i], cb[i], cb[i].v64[0], cb[i].v64[3], cb[i].v64[2], st));
                h64[i]++;
                outer[i]++;
                hres.assign(2 * b->R[i], 0.0);
                AKRA_CUDA_TRY(cudaMemcpyAsync(hres.data(), cb[i].res, sizeof(double) * 2 * b->R[i],
                                              cudaMemcpyDeviceToHost, st));
                AKRA_CUDA_TRY(cudaEventRecord(b->ev, st));
                AKRA_TRY(bounded_wait(b->ev, deadline));
                for (int r = 0; r < b->R[i]; r++) {
                    relres[i][r] = hres[2 * r + 1] > 0 ? sqrt(hres[2 * r] / hres[2 * r + 1]) : 0.0;
                    if (!std::isfinite(relres[i][r])) status[i][r] = AKRA_ENUMERIC;
                }
            }
            budget -= used;
        }
        for (int i = 0; i < n; i++) {
            for (int r = 0; r < b->R[i]; r++)
                if (status[i][r] == AKRA_OK && relres[i][r] >= tol) status[i][r] = AKRA_ENOCONV;
            AKRA_CUDA_TRY(cudaMemcpyAsync(d_x[i], cb[i].v64[1],
                                          (size_t)b->R[i] * 2 * b->plans[i]->ntri * sizeof(double2),
                                          cudaMemcpyDeviceToDevice, st));
        }
    }
    AKRA_TRY(leave(b, user));
    AKRA_CUDA_TRY(cudaEventRecord(b->ev, st));
    AKRA_TRY(bounded_wait(b->ev, deadline));
    for (int i = 0; i < n; i++) AKRA_TRY(tc_error_check(b->plans[i]));
    int worst = AKRA_OK;
    for (int i = 0; i < n; i++) {
        int w = AKRA_OK;
        double mx = 0;
        for (int r = 0; r < b->R[i]; r++) {
            mx = std::max(mx, relres[i][r]);
            if (status[i][r] != AKRA_OK && (w == AKRA_OK || status[i][r] > w)) w = status[i][r];
        }
        if (info) {
            info[i].iters = total[i];
            info[i].outer = outer[i];
            info[i].h_applies_f64 = h64[i];
            info[i].h_applies_f32 = h32[i];
            info[i].relres = mx;
            info[i].status = w;
            for (int r = 0; r < b->R[i]; r++) {
                if (info[i].relres_rhs) info[i].relres_rhs[r] = relres[i][r];
                if (info[i].iters_rhs) info[i].iters_rhs[r] = iters[i][r];
            }
        }
        if (w != AKRA_OK && (worst == AKRA_OK || w > worst)) worst = w;
    }
    if (worst != AKRA_OK) set_error("akra_batch_cg_solve: an instance did not converge cleanly");
    return (akra_status)worst;
}

extern "C" akra_status akra_batch_describe(akra_batch b, int *P, int *RG, long long *launches)
{
    if (!b) {
        set_error("akra_batch_describe: invalid argument");
        return AKRA_EINVAL;
    }
    if (P) *P = b->shape.P;
    if (RG) *RG = b->shape.RG;
    if (launches) *launches = b->launches;
    return AKRA_OK;
}
