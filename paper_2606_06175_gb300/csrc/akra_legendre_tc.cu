// akra_legendre_tc.cu -- FP32 spin-2 Legendre synthesis (Eq. 1 in the φ-separated form, one m and
// one ring pair per row) with the l-contraction on the 5th-generation tensor core.
//
// For one m, a chunk of 128 ring pairs and a group of RG right-hand sides, the synthesis is a
// product of a generated matrix with the staged coefficients:
//     D_{s,p}[u][n] = Σ_{l of parity p} ξ^s_l(u) · b_l[n],
// u = ring pair, s = spin (+2, -2), p = parity of l - l0, n = (RHS, component of c or d) where
// c = f_l σ_l s_l (E + iB), d = f_l σ_l s_l (E - iB) as in the FP32 CUDA-core item (s_l the state
// sign, σ_l the monic scale, f_l = -1 or the KS factor D_l).  The recurrences run on the CUDA cores
// (one pair per thread, both spins in one float2 with paired FMAs); every 16 l-steps the values
// are split into a TF32 head and an FP32 remainder and stored as the A tiles, and one thread
// issues the MMAs: 4 streams (s, p) x 3 products (head·head, head·rest, rest·head) of
// M = 128 rows, N = 4 RG columns, K = 8 l-values, accumulated in FP32 in tensor memory.
// Tiles are double-buffered: the recurrence of tile t+1 runs while the MMAs of tile t do.  After
// the last tile each thread reads its own row (TMEM lane = ring pair) and forms Φ(±m) of both
// rings as the CUDA-core item does.
#include <algorithm>

#include "akra_legendre_impl.cuh"
#include "akra_tc.cuh"

namespace akra {

namespace {

constexpr int TCT = 16;        // l-steps per tile: 8 of each parity (K = 8 TF32 per MMA)
constexpr int kWaitLimit = 1 << 20;

template <int RG>
struct TcSynth {
    static constexpr int N = 4 * RG;                         // MMA columns per stream
    static constexpr int A_TILE = 128 * 8 * 4;               // 4 KB
    static constexpr int A_BUF = 8 * A_TILE;                 // A[s][p][h] of one tile
    static constexpr int B_TILE = N * 8 * 4;
    static constexpr int B_SLOT = 4 * B_TILE;                // B[p][h] of one tile, pre-staged layout
    static constexpr int NSLOT = 4;                          // B / coefficient ring: 3 tiles ahead
    static constexpr int CF = TCT * 16;                      // 16 float4 coefficients of a tile
    static constexpr int OFF_B = 2 * A_BUF;
    static constexpr int OFF_CRAW = OFF_B + NSLOT * B_SLOT;  // raw coefficient ring
    static constexpr int OFF_CF = OFF_CRAW + NSLOT * CF;     // standard / difference-form, 2 tiles each
    static constexpr int USED = OFF_CF + 4 * CF;
    // TMEM columns: 4 streams x N (a power of two >= 32); shared memory sized so that the blocks
    // resident on an SM never ask for more than its 512 columns
    static constexpr uint32_t NCOL = 16 * RG < 32 ? 32 : 16 * RG;
    static constexpr int MAXB = 512 / (int)NCOL;
    static constexpr int SMEM = (MAXB >= 3 || USED * (MAXB + 1) > 227 * 1024) ? USED : (227 * 1024) / (MAXB + 1) + 1024;
};

__device__ __forceinline__ unsigned char *tc_a(unsigned char *abuf, int s, int p, int h)
{
    return abuf + ((s * 2 + p) * 2 + h) * (128 * 8 * 4);
}

template <int RG>
__device__ __forceinline__ unsigned char *tc_b(unsigned char *bslot, int p, int h)
{
    return bslot + (p * 2 + h) * TcSynth<RG>::B_TILE;
}

// issue the asynchronous copies of tile lj (l = lj .. lj+15, lj - l0 a multiple of 16) of RHS group
// g: its pre-staged B operand into a B slot and its 16 raw coefficient entries (zero past lmax)
template <int RG>
__device__ __forceinline__ void tc_prefetch(const LegArgs<float> &a, int m, long long mbase, int l0, int g, int lj,
                                            unsigned char *bslot, float4 *craw)
{
    using S = TcSynth<RG>;
    const int tid = threadIdx.x;
    constexpr int CH = S::B_SLOT / 16;                       // 16-byte chunks of a B slot
    const long long base = ((a.tc_tilebase[m] + (lj - l0) / TCT) * a.tc_groups + g) * CH;
    const long long bound = a.tc_tiles * a.tc_groups * CH;
    (void)bound;
    const float4 *src = reinterpret_cast<const float4 *>(a.bpre);
    for (int c = tid; c < CH; c += TC_NT)
        tc::cp_async16(bslot + 16 * c, src + AKRA_IX(base + c, bound, kDbgBpre), 16);
    if (tid < TCT) {
        const int l = lj + tid;
        const bool in = l <= a.L;
        tc::cp_async16(craw + tid, a.coef + AKRA_IX(mbase + (in ? l : l0), a.ntri, kDbgCoef), in ? 16u : 0u);
    }
}

// the per-step recurrence coefficients of a tile from its raw entries {A', c', σ, A' - 2}:
// sign-alternated {rA', rA', rc', -rc'} and, for blocks with polar pairs, the difference form's
// {A', A', (A' - 2) + c', (A' - 2) - c'} (threads 0..15)
__device__ __forceinline__ void tc_coefs(const float4 *craw, float4 *cf, float4 *cfd, bool diff)
{
    const int tid = threadIdx.x;
    if (tid < TCT) {
        const float4 c = craw[tid];
        cf[tid] = f2_coef_entry(c, tid);
        if (diff) cfd[tid] = make_float4(c.x, c.x, c.w + c.y, c.w - c.y);
    }
}

// the A rows of this thread (ring pair) for 8 consecutive steps: lam[j] = (ξ+, ξ-) at step
// 8 half + j, so parity p holds k = 4 half + q at j = p + 2q
__device__ __forceinline__ void tc_store_half(unsigned char *buf, int row, int half, const float2 (&lam)[8])
{
    const uint32_t o = tc::tile_off(row, 4 * half);
#pragma unroll
    for (int p = 0; p < 2; p++) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
            float4 hd, rs;
            float *ph = &hd.x, *pr = &rs.x;
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float x = s == 0 ? lam[p + 2 * q].x : lam[p + 2 * q].y;
                ph[q] = tc::tf32_head(x);
                pr[q] = x - ph[q];
            }
            *reinterpret_cast<float4 *>(tc_a(buf, s, p, 0) + o) = hd;
            *reinterpret_cast<float4 *>(tc_a(buf, s, p, 1) + o) = rs;
        }
    }
}

}  // namespace

// one work item (m, chunk of 128 ring pairs, RHS group from r0) into the block's TMEM columns
// (allocated once per block by the caller: a CTA allocates only until it gives up its permit).
// The two mbarriers are initialised at the start of the item and invalidated at its end, once
// every commit issued to them has been waited for, so a persistent block can run items back to back.
template <int RG>
__device__ __forceinline__ void tc_synth_item(const LegArgs<float> &a, const int m, const int chunk, const int r0,
                                              unsigned char *smem, uint64_t *s_mbar, const uint32_t tmem_base)
{
    using S = TcSynth<RG>;
    constexpr int N = S::N;
    const int L = a.L, nring = a.nring, nunits = a.nunits, nunit_all = a.nunit_all, R = a.R;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int l0 = m > 2 ? m : 2;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const long long tbound = (long long)(L + 1) * nunit_all;
    const size_t row = 2 * (size_t)L + 1;
    const long long pbound = (long long)R * nring * row;
    (void)pbound;

    // this thread's ring pair (row tid of every A tile)
    const int iu = chunk * TC_NT + tid;
    int uid1[1] = {iu < nunits ? (a.units ? a.units[AKRA_IX(iu, nunits, kDbgUnits)] : iu) : -1};
    int gs1[1] = {kNeverLive};
    float2 X2 = make_float2(0.f, 0.f);
    float2 V[1] = {make_float2(0.f, 0.f)}, VO[1] = {make_float2(0.f, 0.f)};
    int e1[1] = {0};
    bool polar = false;
    UnitInfo u0;
    if (uid1[0] >= 0) {
        u0 = a.uinfo[AKRA_IX(uid1[0], nunit_all, kDbgUnitInfo)];
        polar = u0.x >= kDiffX;
        gs1[0] = a.start[AKRA_IX((size_t)m * nunit_all + uid1[0], tbound, kDbgStart)].x;
    }
    // pairs near a pole run the difference form (warp-uniform; X2 then holds x - 1)
    const bool dkw = __any_sync(0xffffffffu, polar);
    if (uid1[0] >= 0) {
        const float x = dkw ? (float)(-exp2(2.0 * u0.ls + 1.0)) : (float)u0.x;
        X2 = make_float2(x, x);
    }
    const int warp_first = __reduce_min_sync(0xffffffffu, gs1[0]);
    const int l_first = block_min_start<TC_NT>(gs1[0]);
    const bool blk_diff = __syncthreads_or(dkw) != 0;

    float dv[2][2][4];   // D of this row: [spin][parity][c.re, c.im, d.re, d.im], per RHS below
    if (l_first <= L) {
        if (tid == 0) {
            tc::mbar_init(&s_mbar[0], 1);
            tc::mbar_init(&s_mbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
    }
    const bool active = l_first <= L;
    const uint32_t tmem = tmem_base;
    bool ok = true;
    const int T = active ? (L - l_first) / TCT + 1 : 0;
    unsigned char *bring = smem + S::OFF_B;                                    // B slots
    float4 *craw = reinterpret_cast<float4 *>(smem + S::OFF_CRAW);              // raw coefficient slots
    float4 *cf_all = reinterpret_cast<float4 *>(smem + S::OFF_CF);
    float4 *cfd_all = cf_all + 2 * TCT;
    const int g = r0 / RG;
    // copies of tile j go to slot j mod 4, three tiles ahead of the one being computed; one copy
    // group per tile (empty past the last), so that cp.async.wait_group 2 leaves only the two
    // newest in flight
    auto prefetch = [&](int j) {
        if (j < T) tc_prefetch<RG>(a, m, mbase, l0, g, l_first + j * TCT, bring + (j & 3) * S::B_SLOT, craw + (j & 3) * TCT);
        tc::cp_async_commit();
    };
    if (active) {
        prefetch(0);
        prefetch(1);
        prefetch(2);
        tc::cp_async_wait<2>();                                   // this thread's copies of tile 0
        tc_coefs(craw, cf_all, cfd_all, blk_diff);
        tc::fence_async_smem();
        __syncthreads();
    }
    const uint32_t idesc = tc::idesc_tf32(128, N);
    for (int t = 0; t < T; t++) {
        const int lt = l_first + t * TCT, b = t & 1;
        unsigned char *buf = smem + b * S::A_BUF;
        unsigned char *bslot = bring + (t & 3) * S::B_SLOT;
        const float4 *cf = cf_all + b * TCT;
        const float4 *cfd = cfd_all + b * TCT;
        f2_start_pairs<1>(a.seeds, a.start, (size_t)m * nunit_all, tbound, lt, uid1, gs1, V, VO, e1);
        if (dkw && gs1[0] == lt)   // difference form: second register holds μ_g - μ_{g-1}
            VO[0] = a.dseeds[AKRA_IX((size_t)m * nunit_all + uid1[0], tbound, kDbgSeeds)];
        if (warp_first > lt + TCT - 1) {
            // none of this warp's pairs has started: zero rows
            const float2 z[8] = {};
            tc_store_half(buf, tid, 0, z);
            tc_store_half(buf, tid, 1, z);
        } else {
            const bool all_live = __all_sync(0xffffffffu, e1[0] == 0);
#pragma unroll
            for (int half = 0; half < 2; half++) {
                float2 lam[8];
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    const int i = half * 8 + j;
                    const float2 cur = (i & 1) == 0 ? V[0] : VO[0];
                    // difference form: the state is μ, the A tiles take ξ = s_l μ
                    const float2 cx = (dkw && (i & 2)) ? make_float2(-cur.x, -cur.y) : cur;
                    lam[j] = (!all_live && e1[0] != 0) ? make_float2(0.f, 0.f) : cx;
                    if (dkw) {
                        const float4 cd = cfd[i];
                        const float2 uu = f2fma(make_float2(cd.x, cd.y), X2, make_float2(cd.z, cd.w));
                        if ((i & 1) == 0) {
                            const float2 dn = f2fma(uu, V[0], VO[0]);
                            VO[0] = __fadd2_rn(V[0], dn);
                            V[0] = dn;
                            if (!all_live) f2_rescale<1>(0, V, VO, e1, VO[0]);
                        } else {
                            const float2 dn = f2fma(uu, VO[0], V[0]);
                            V[0] = __fadd2_rn(VO[0], dn);
                            VO[0] = dn;
                            if (!all_live) f2_rescale<1>(0, V, VO, e1, V[0]);
                        }
                    } else {
                        const float4 c4 = cf[i];
                        const float2 tt = f2fma(make_float2(c4.x, c4.y), X2, make_float2(c4.z, c4.w));
                        if ((i & 1) == 0) {
                            VO[0] = f2fma(tt, V[0], VO[0]);
                            if (!all_live) f2_rescale<1>(0, V, VO, e1, VO[0]);
                        } else {
                            V[0] = f2fma(tt, VO[0], V[0]);
                            if (!all_live) f2_rescale<1>(0, V, VO, e1, V[0]);
                        }
                    }
                }
                tc_store_half(buf, tid, half, lam);
            }
        }
        if (t + 1 < T) {
            // the other A buffer and B slot (t + 3) mod 4 are free once the MMAs of tile t-1 have
            // completed; then tile t+3's copies go out and tile t+1's (issued at t-2) are waited for
            if (t >= 1) ok &= tc::mbar_wait(&s_mbar[(t + 1) & 1], ((t - 1) >> 1) & 1, kWaitLimit, a.err);
            prefetch(t + 3);
            tc::cp_async_wait<2>();
            tc_coefs(craw + ((t + 1) & 3) * TCT, cf_all + ((t + 1) & 1) * TCT, cfd_all + ((t + 1) & 1) * TCT,
                     blk_diff);
        }
        tc::fence_async_smem();
        tc::fence_before();
        __syncthreads();
        tc::fence_after();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    const uint32_t d = tmem + (uint32_t)((s * 2 + p) * N);
                    const uint64_t ah = tc::sdesc(tc::smem_u32(tc_a(buf, s, p, 0)));
                    const uint64_t al = tc::sdesc(tc::smem_u32(tc_a(buf, s, p, 1)));
                    const uint64_t bh = tc::sdesc(tc::smem_u32(tc_b<RG>(bslot, p, 0)));
                    const uint64_t bl = tc::sdesc(tc::smem_u32(tc_b<RG>(bslot, p, 1)));
                    tc::mma_tf32(d, ah, bh, idesc, t > 0 ? 1u : 0u);
                    tc::mma_tf32(d, ah, bl, idesc, 1u);
                    tc::mma_tf32(d, al, bh, idesc, 1u);
                }
            tc::commit(&s_mbar[b]);
        }
    }
    if (active) {
        // the last two commits (tiles T-2 and T-1, one per barrier; earlier ones were waited for in
        // the loop), so that no arrival is pending when the barriers are invalidated
        if (T >= 2) ok &= tc::mbar_wait(&s_mbar[(T - 2) & 1], ((T - 2) >> 1) & 1, kWaitLimit, a.err);
        ok &= tc::mbar_wait(&s_mbar[(T - 1) & 1], ((T - 1) >> 1) & 1, kWaitLimit, a.err);
        tc::fence_after();
        if (!ok && a.err) atomicExch(a.err, 1);
        tc::cp_async_wait<0>();   // only empty groups can remain; none may outlive the item
    }

    // Φ(±m) of both rings of this row's pair, per RHS
    const bool swap = ((l0 + m) & 1) != 0;
    UnitInfo ui;
    ui.ring_n = ui.ring_s = -1;
    if (uid1[0] >= 0) ui = a.uinfo[AKRA_IX(uid1[0], nunit_all, kDbgUnitInfo)];
    for (int rr = 0; rr < RG; rr++) {
        const int r = r0 + rr;
        if (active) {
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int p = 0; p < 2; p++)
                    tc::tmem_ld4(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((s * 2 + p) * N + 4 * rr), dv[s][p]);
        } else {
#pragma unroll
            for (int s = 0; s < 2; s++)
#pragma unroll
                for (int p = 0; p < 2; p++)
#pragma unroll
                    for (int c = 0; c < 4; c++) dv[s][p][c] = 0.f;
        }
        if (uid1[0] < 0 || r >= R) continue;
        // per parity: [0] Σcλ+ re, [1] Σcλ+ im, [2] Σdλ- re, [3] Σdλ- im,
        //             [4] Σcλ- re, [5] Σcλ- im, [6] Σdλ+ re, [7] Σdλ+ im
        float se[8], so[8];
#pragma unroll
        for (int p = 0; p < 2; p++) {
            float *dst = ((p == 0) != swap) ? se : so;
            dst[0] = dv[0][p][0];
            dst[1] = dv[0][p][1];
            dst[2] = dv[1][p][2];
            dst[3] = dv[1][p][3];
            dst[4] = dv[1][p][0];
            dst[5] = dv[1][p][1];
            dst[6] = dv[0][p][2];
            dst[7] = dv[0][p][3];
        }
#pragma unroll
        for (int side = 0; side < 2; side++) {
            const int ring = side == 0 ? ui.ring_n : ui.ring_s;
            if (ring < 0) continue;
            if (a.ring_active && !a.ring_active[AKRA_IX(ring, nring, kDbgRingActive)]) continue;
            const int o = side == 0 ? 0 : 4;
            const float sg = side == 0 ? 1.f : -1.f;
            const float fr = se[o + 0] + sg * so[o + 0], fi = se[o + 1] + sg * so[o + 1];
            const float gr = se[o + 2] + sg * so[o + 2], gi = se[o + 3] + sg * so[o + 3];
            const size_t pb = ((size_t)r * nring + ring) * row + L;   // Φ(ring, m = 0)
            a.phi[AKRA_IX(pb + m, pbound, kDbgPhiWrite)] = make_float2(fr, fi);
            if (m > 0) a.phi[AKRA_IX(pb - m, pbound, kDbgPhiWrite)] = make_float2(gr, -gi);
        }
    }
    // every thread's TMEM loads (and, for the next item, its shared-memory reads) come before
    // the next item's set-up
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (active && tid == 0) {
        tc::mbar_inval(&s_mbar[0]);
        tc::mbar_inval(&s_mbar[1]);
    }
    __syncthreads();
}

// TMEM columns of the block, allocated by warp 0 (which then gives up the block's permit)
template <int RG>
__device__ __forceinline__ uint32_t tc_block_alloc(uint32_t *s_tmem)
{
    if (threadIdx.x < 32) tc::tmem_alloc(s_tmem, TcSynth<RG>::NCOL);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    return *s_tmem;
}

template <int RG>
__device__ __forceinline__ void tc_block_free(uint32_t tmem)
{
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (threadIdx.x < 32) tc::tmem_dealloc(tmem, TcSynth<RG>::NCOL);
}

template <int RG>
__global__ void __launch_bounds__(TC_NT) k_leg_synth_tc(LegArgs<float> a)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    if (a.skip && *a.skip) return;
    const uint32_t tmem = tc_block_alloc<RG>(&s_tmem);
    const int m = blockIdx.x / a.nchunks;
    tc_synth_item<RG>(a, m, blockIdx.x - m * a.nchunks, blockIdx.y * RG, smem, s_mbar, tmem);
    tc_block_free<RG>(tmem);
}

// persistent form over several plans: blocks take (instance, m, chunk, RHS group) items from a
// queue ordered by cost
template <int RG>
__global__ void __launch_bounds__(TC_NT)
k_leg_synth_tc_queue(const LegArgs<float> *__restrict__ insts, const int4 *__restrict__ items, int nitems,
                     int *counter)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_it;
    const uint32_t tmem = tc_block_alloc<RG>(&s_tmem);
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_it;
        __syncthreads();
        if (it >= nitems) break;
        const int4 w = items[it];
        const LegArgs<float> &a = insts[w.x];
        if (a.skip && *a.skip) continue;
        tc_synth_item<RG>(a, w.y, w.z, w.w * RG, smem, s_mbar, tmem);
    }
    tc_block_free<RG>(tmem);
}

// B operand tiles of one plan's alm for RHS groups of RG, in the shared-memory layout of a tile:
// [tile][group][parity][head, rest][N rows x 8 K] (K-major canonical core matrices, tile_off),
// tiles of 16 l-steps from l0 = max(m, 2), values f_l σ_l s_l (E ± iB) with s_l the state sign
// relative to the tile start.  One block row per m; consecutive threads write consecutive words.
template <int RG>
__global__ void __launch_bounds__(256) k_tc_bstage(LegArgs<float> a, float *out)
{
    using S = TcSynth<RG>;
    constexpr int N = S::N;
    const int m = blockIdx.x, L = a.L, R = a.R;
    const int l0 = m > 2 ? m : 2;
    const long long ntri = a.ntri, mbase = (long long)m * (2 * L + 1 - m) / 2;
    const int ntile = (L - l0) / TCT + 1;
    const long long per_tile = (long long)a.tc_groups * 16 * N;
    const long long tb = a.tc_tilebase[AKRA_IX(m, L + 1, kDbgBpre)];
    const long long obound = a.tc_tiles * a.tc_groups * (S::B_SLOT / 4);
    const long long abound = (long long)R * 2 * ntri;
    (void)obound;
    (void)abound;
    for (long long idx = threadIdx.x + (long long)blockIdx.y * blockDim.x; idx < ntile * per_tile;
         idx += (long long)blockDim.x * gridDim.y) {
        const int q = (int)(idx / per_tile);
        const long long rem = idx - q * per_tile;
        const int g = (int)(rem / (16 * N)), e = (int)(rem - (long long)g * 16 * N);
        // e bits 0-1: k mod 4, 2-4: row mod 8, 5: k / 4, 6: parity, 7+: row / 8
        const int kq = e & 3, r8 = (e >> 2) & 7, kh = (e >> 5) & 1, p = (e >> 6) & 1, rb = e >> 7;
        const int row = rb * 8 + r8, k = kh * 4 + kq, i = p + 2 * k;
        const int rr = row >> 2, c = row & 3;
        const int l = l0 + q * TCT + i, r = g * RG + rr;
        float v = 0.f;
        if (l <= L && r < R) {
            float2 E = a.alm[AKRA_IX(((size_t)r * 2 + 0) * ntri + mbase + l, abound, kDbgAlm)];
            float2 B = a.alm[AKRA_IX(((size_t)r * 2 + 1) * ntri + mbase + l, abound, kDbgAlm)];
            const float f = (a.fl ? a.fl[AKRA_IX(l, L + 1, kDbgKsFactor)] : -1.f) *
                            a.coef[AKRA_IX(mbase + l, ntri, kDbgCoef)].z * f2_sign(i);
            if (m == 0) E.y = B.y = 0.f;
            // rows c = 0..3 of an RHS: c = f (E + iB) re, im; d = f (E - iB) re, im
            v = c == 0 ? f * (E.x - B.y) : c == 1 ? f * (E.y + B.x) : c == 2 ? f * (E.x + B.y) : f * (E.y - B.x);
        }
        const float hd = tc::tf32_head(v);
        const long long o = ((tb + q) * a.tc_groups + g) * (S::B_SLOT / 4) + p * (S::B_TILE / 2) +
                            tc::tile_off(row, k) / 4;
        out[AKRA_IX(o, obound, kDbgBpre)] = hd;
        out[AKRA_IX(o + S::B_TILE / 4, obound, kDbgBpre)] = v - hd;
    }
}

template <int RG>
static akra_status launch_bstage(const LegArgs<float> &a, cudaStream_t st)
{
    k_tc_bstage<RG><<<dim3((unsigned)a.L + 1, 4), 256, 0, st>>>(a, const_cast<float *>(a.bpre));
    AKRA_CUDA_TRY(cudaGetLastError());
    return AKRA_OK;
}

template <int RG>
static akra_status launch_synth_tc(akra_plan p, LegMode mode, const void *alm, void *phi, int R,
                                   const int *units, int nunits, cudaStream_t st)
{
    AKRA_TRY(tc_reserve(p, RG, R));
    LegArgs<float> a = leg_args<float>(p, LegShape{1, TC_NT, RG}, mode, units, nunits, R);
    a.alm = (const float2 *)alm;
    a.phi = (float2 *)phi;
    a.bpre = (const float *)p->bpre.ptr;
    a.tc_groups = (R + RG - 1) / RG;
    AKRA_TRY(launch_bstage<RG>(a, st));
    p->launches++;
    dim3 grid((unsigned)(p->lmax + 1) * a.nchunks, (R + RG - 1) / RG);
    k_leg_synth_tc<RG><<<grid, TC_NT, TcSynth<RG>::SMEM, st>>>(a);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

// the shared-memory opt-in of the tensor-core kernels (at plan creation, never inside a capture)
akra_status legendre_tc_prepare()
{
#define AKRA_TC_ATTR(G)                                                                                  \
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_leg_synth_tc<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                       TcSynth<G>::SMEM));                                               \
    AKRA_CUDA_TRY(cudaFuncSetAttribute(k_leg_synth_tc_queue<G>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                       TcSynth<G>::SMEM));
    AKRA_TC_ATTR(4) AKRA_TC_ATTR(8) AKRA_TC_ATTR(16) AKRA_TC_ATTR(32)
#undef AKRA_TC_ATTR
    return AKRA_OK;
}

// persistent tensor-core synthesis over a batch's item list (akra_batch.cu)
template <int RG>
static akra_status launch_tc_queue(const LegArgs<float> *insts, const int4 *items, int nitems, int *counter,
                                   cudaStream_t st)
{
    // resident blocks per SM from shared memory (dynamic + static + the per-block reservation)
    // and TMEM columns; blocks beyond what fits simply start later (no block waits on another)
    int dev = 0, nsm = 1, smem_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_leg_synth_tc_queue<RG>);
    const int per_blk = TcSynth<RG>::SMEM + (int)fa.sharedSizeBytes + reserved;
    const int per_sm = std::max(1, std::min(smem_sm / std::max(per_blk, 1), 512 / (int)TcSynth<RG>::NCOL));
    const int grid = std::max(1, std::min(nitems, nsm * per_sm));
    k_leg_synth_tc_queue<RG><<<grid, TC_NT, TcSynth<RG>::SMEM, st>>>(insts, items, nitems, counter);
    AKRA_CUDA_TRY(cudaGetLastError());
    return AKRA_OK;
}

akra_status legendre_synth_tc_queue(int tcg, const LegArgs<float> *insts, const int4 *items, int nitems,
                                    int *counter, cudaStream_t st)
{
    switch (tcg) {
    case 4: return launch_tc_queue<4>(insts, items, nitems, counter, st);
    case 8: return launch_tc_queue<8>(insts, items, nitems, counter, st);
    case 16: return launch_tc_queue<16>(insts, items, nitems, counter, st);
    case 32: return launch_tc_queue<32>(insts, items, nitems, counter, st);
    default:
        set_error("no tensor-core synthesis for an RHS group of %d", tcg);
        return AKRA_EINVAL;
    }
}

size_t tc_bpre_bytes(akra_plan p, int tcg, int R)
{
    if (tcg <= 0) return 0;
    return (size_t)p->tc_tiles * (size_t)((R + tcg - 1) / tcg) * (size_t)(128 * 4 * tcg);
}

akra_status tc_reserve(akra_plan p, int tcg, int R)
{
    if (tcg <= 0) return AKRA_OK;
    return ws_reserve(p, p->bpre, tc_bpre_bytes(p, tcg, R));
}

akra_status legendre_tc_bstage(int tcg, const LegArgs<float> &a, cudaStream_t st)
{
    switch (tcg) {
    case 4: return launch_bstage<4>(a, st);
    case 8: return launch_bstage<8>(a, st);
    case 16: return launch_bstage<16>(a, st);
    case 32: return launch_bstage<32>(a, st);
    default:
        set_error("no tensor-core synthesis for an RHS group of %d", tcg);
        return AKRA_EINVAL;
    }
}

// FP32 synthesis with the tensor-core contraction, RHS in groups of tcg (4, 8, 16 or 32)
akra_status legendre_synth_tc(akra_plan p, int tcg, LegMode mode, const void *alm, void *phi, int R,
                              const int *units, int nunits, cudaStream_t st)
{
    if (nunits <= 0) return AKRA_OK;
    switch (tcg) {
    case 4: return launch_synth_tc<4>(p, mode, alm, phi, R, units, nunits, st);
    case 8: return launch_synth_tc<8>(p, mode, alm, phi, R, units, nunits, st);
    case 16: return launch_synth_tc<16>(p, mode, alm, phi, R, units, nunits, st);
    case 32: return launch_synth_tc<32>(p, mode, alm, phi, R, units, nunits, st);
    default:
        set_error("no tensor-core synthesis for an RHS group of %d", tcg);
        return AKRA_EINVAL;
    }
}

AKRA_DEBUG_COLLECTOR(legendre_tc)

}  // namespace akra
