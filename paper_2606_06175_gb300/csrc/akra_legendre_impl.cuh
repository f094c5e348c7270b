// akra_legendre_impl.cuh -- bodies of the Legendre kernels (one work item: one m, one chunk
// of ring pairs, one group of RHS) shared by the per-plan launches (akra_legendre.cu) and the
// persistent multi-instance launches (akra_batch.cu).  See akra_legendre.cu for the method.
#pragma once
#include <type_traits>

#include "akra_internal.cuh"

namespace akra {

constexpr int TL = 64;  // l-steps staged in shared memory per tile (even)

// seeds 2λ_{l0 m} (vp) and (-2)λ_{l0 m} (vm) with their shared exponent index e, from the
// plan's table (computed in FP64 at plan creation)
// smallest start grid point over the block (kNeverLive if no pair of the block ever starts)
template <int NT>
__device__ __forceinline__ int block_min_start(int v)
{
    __shared__ int s_first;
    if (threadIdx.x == 0) s_first = kNeverLive;
    __syncthreads();
    v = __reduce_min_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) atomicMin(&s_first, v);
    __syncthreads();
    return s_first;
}

// at an l-tile that begins at lt (a grid point, even offset from l0, so that vp / vm hold the
// current values): load the state of every pair whose recurrence starts here
template <typename V4, typename T, int P>
__device__ __forceinline__ void start_pairs(const V4 *__restrict__ seeds, const int2 *__restrict__ start,
                                            size_t base, long long tbound, int lt, const int (&uid)[P],
                                            const int (&gs)[P], T (&vp)[P], T (&vm)[P],
                                            T (&vpo)[P], T (&vmo)[P], int (&e)[P])
{
    (void)tbound;
#pragma unroll
    for (int k = 0; k < P; k++) {
        if (gs[k] == lt) {
            const V4 s = seeds[AKRA_IX(base + uid[k], tbound, kDbgSeeds)];
            vp[k] = s.x;
            vm[k] = s.y;
            vpo[k] = s.z;
            vmo[k] = s.w;
            e[k] = start[AKRA_IX(base + uid[k], tbound, kDbgStart)].y;
        }
    }
}

// FP32 difference-form pairs: at their start the second state register holds d_g = μ_g - μ_{g-1}
template <typename T, int P>
__device__ __forceinline__ void start_diff(const float2 *__restrict__ dseeds, size_t base, long long tbound,
                                           int lt, const int (&uid)[P], const int (&gs)[P], const bool (&dk)[P],
                                           T (&vpo)[P], T (&vmo)[P])
{
    (void)tbound;
#pragma unroll
    for (int k = 0; k < P; k++) {
        if (dk[k] && gs[k] == lt) {
            const float2 d = dseeds[AKRA_IX(base + uid[k], tbound, kDbgSeeds)];
            vpo[k] = d.x;
            vmo[k] = d.y;
        }
    }
}

// which rings of a unit the operator needs (weighted operators list only the active rings):
// 0 both (or every ring), 1 the north ring alone (or the equator ring), 2 the south ring alone,
// 3 no unit.  The warp takes the one-ring contraction when all its units are of one such kind.
__device__ __forceinline__ int unit_side(const UnitInfo &ui, const unsigned char *ring_active, int nring)
{
    (void)nring;
    if (!ring_active) return 0;
    const bool an = ring_active[AKRA_IX(ui.ring_n, nring, kDbgRingActive)] != 0;
    const bool as = ui.ring_s >= 0 && ring_active[AKRA_IX(ui.ring_s, nring, kDbgRingActive)] != 0;
    return an && as ? 0 : an ? 1 : as ? 2 : 0;
}

__device__ __forceinline__ int warp_side(int mine)
{
    // mine: this lane's common side over its slots (3: no unit); 0 unless the warp agrees
    const bool all1 = __all_sync(0xffffffffu, mine == 1 || mine == 3);
    const bool all2 = __all_sync(0xffffffffu, mine == 2 || mine == 3);
    return all1 ? 1 : all2 ? 2 : 0;
}

// fold one slot's side into the lane's common side (3: none yet, 0: mixed)
__device__ __forceinline__ int side_join(int acc, int s) { return acc == 3 ? s : (acc == s ? acc : 0); }

}  // namespace akra

#include "akra_legendre_f32x2.cuh"   // FP32 items with paired FMAs (use TL, block_min_start)

namespace akra {

// ---------------------------------------------------------------------------
// synthesis: Φ(ring, ±m) for every ring of the listed units.  Where only one ring of a pair is
// needed (a footprint in one hemisphere), a warp whose pairs all need the same single ring
// accumulates that ring's two sums directly -- the north ring takes even + odd terms, the south
// ring even - odd (sign folded per slot) -- 4 FMA per step and RHS instead of 8.
// ---------------------------------------------------------------------------
template <typename T, int P, int RG, int NT>
__device__ __forceinline__ void leg_synth_item(const LegArgs<T> &a, const int m, const int chunk,
                                               const int r0, v4_t<T> *s_coef, v4_t<T> (*s_alm)[RG])
{
    using C2 = cx_t<T>;
    using V4 = v4_t<T>;
    const int L = a.L, nring = a.nring, nunits = a.nunits, nunit_all = a.nunit_all, R = a.R;
    const long long ntri = a.ntri;
    const int *__restrict__ units = a.units;
    const UnitInfo *__restrict__ uinfo = a.uinfo;
    const v4_t<T> *__restrict__ coef = a.coef;
    const v4_t<T> *__restrict__ seeds = a.seeds;
    const int2 *__restrict__ start = a.start;
    const unsigned char *__restrict__ ring_active = a.ring_active;
    const T *__restrict__ fl = a.fl;
    const cx_t<T> *__restrict__ alm = a.alm;
    cx_t<T> *__restrict__ phi = a.phi;
    const int l0 = m > 2 ? m : 2;
    const int tid = threadIdx.x;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const long long tbound = (long long)(L + 1) * nunit_all;   // extent of the start tables

    // every pair's recurrence starts at its grid point gs (state loaded there); until then
    // its state is zero, which the recurrence keeps and the contraction ignores
    T x[P], y[P], vp[P], vm[P], vpo[P], vmo[P];
    int e[P], uid[P], gs[P];
    bool dk[P];   // FP32: this warp's pairs of slot k run the difference form (warp-uniform)
    T acc[P][RG][16];
    int my_first = kNeverLive;
    bool any_diff = false;
    int my_side = 3;
#pragma unroll
    for (int k = 0; k < P; k++) {
        const int iu = (chunk * P + k) * NT + tid;
        uid[k] = iu < nunits ? (units ? units[AKRA_IX(iu, nunits, kDbgUnits)] : iu) : -1;
        x[k] = y[k] = 0;
        vp[k] = vm[k] = vpo[k] = vmo[k] = 0;
        e[k] = 0;
        gs[k] = kNeverLive;
        bool polar = false;
        if (uid[k] >= 0) {
            const UnitInfo ui = uinfo[AKRA_IX(uid[k], nunit_all, kDbgUnitInfo)];
            my_side = side_join(my_side, unit_side(ui, ring_active, nring));
            x[k] = (T)ui.x;
            y[k] = (T)(-exp2(2.0 * ui.ls + 1.0));   // x - 1 = -2 sin^2(θ/2), accurate near the pole
            polar = std::is_same<T, float>::value && ui.x >= kDiffX;
            gs[k] = start[AKRA_IX((size_t)m * nunit_all + uid[k], tbound, kDbgStart)].x;
        }
        dk[k] = __any_sync(0xffffffffu, polar);
        any_diff |= dk[k];
        my_first = min(my_first, gs[k]);
#pragma unroll
        for (int r = 0; r < RG; r++)
#pragma unroll
            for (int j = 0; j < 16; j++) acc[k][r][j] = 0;
    }
    const int warp_first = __reduce_min_sync(0xffffffffu, my_first);
    const int side = warp_side(my_side);
    const int l_first = block_min_start<NT>(my_first);
    const bool blk_diff = __syncthreads_or(any_diff) != 0;   // block-uniform
    __shared__ float2 s_cb[TL];   // difference form: {(A'-2) + c', (A'-2) - c'} per step

    for (int lt = l_first; lt <= L; lt += TL) {
        __syncthreads();
        // recurrence coefficients of two consecutive steps per entry: {A'_l, c'_l, A'_l+1, c'_l+1}
        for (int i = tid; i < TL / 2; i += NT) {
            const int l = lt + 2 * i;
            const V4 c0 = (l <= L) ? coef[AKRA_IX(mbase + l, ntri, kDbgCoef)] : V4{0, 0, 0, 0};
            const V4 c1 = (l + 1 <= L) ? coef[AKRA_IX(mbase + l + 1, ntri, kDbgCoef)] : V4{0, 0, 0, 0};
            s_coef[i] = V4{c0.x, c0.y, c1.x, c1.y};
            if (blk_diff) {
                s_cb[2 * i] = make_float2((float)(c0.w + c0.y), (float)(c0.w - c0.y));
                s_cb[2 * i + 1] = make_float2((float)(c1.w + c1.y), (float)(c1.w - c1.y));
            }
        }
        for (int i = tid; i < TL * RG; i += NT) {
            const int li = i / RG, rr = i - li * RG;
            const int l = lt + li, r = r0 + rr;
            V4 v{0, 0, 0, 0};
            if (l <= L && r < R) {
                const long long abound = (long long)R * 2 * ntri;
                C2 E = alm[AKRA_IX(((size_t)r * 2 + 0) * ntri + mbase + l, abound, kDbgAlm)];
                C2 B = alm[AKRA_IX(((size_t)r * 2 + 1) * ntri + mbase + l, abound, kDbgAlm)];
                // KS (or -1) factor times the monic scale σ_l: λ_l = σ_l μ_l
                const T f = (fl ? fl[AKRA_IX(l, L + 1, kDbgKsFactor)] : T(-1)) *
                            coef[AKRA_IX(mbase + l, ntri, kDbgCoef)].z;
                if (m == 0) E.y = B.y = 0;
                // c = f (E + iB), d = f (E - iB)
                v = V4{f * (E.x - B.y), f * (E.y + B.x), f * (E.x + B.y), f * (E.y - B.x)};
            }
            s_alm[li][rr] = v;
        }
        __syncthreads();
        const int nl = min(TL, L - lt + 1);
        start_pairs(seeds, start, (size_t)m * nunit_all, tbound, lt, uid, gs, vp, vm, vpo, vmo, e);
        if (blk_diff) start_diff<T, P>(a.dseeds, (size_t)m * nunit_all, tbound, lt, uid, gs, dk, vpo, vmo);
        if (warp_first > lt + TL - 1) continue;   // none of this warp's pairs has started yet
        bool live = true;
#pragma unroll
        for (int k = 0; k < P; k++) live &= (e[k] == 0);
        const bool all_live = __all_sync(0xffffffffu, live);

        // one l-step: contract at l (slot S = parity of l - l0), then recur to l+1.
        // vp = 2λ, vm = (-2)λ; accumulators per slot: P1 = Σ c 2λ, P2 = Σ d (-2)λ,
        // P3 = Σ c (-2)λ, P4 = Σ d 2λ (complex)
#define AKRA_SYNTH_STEP(I, S, GATED, CA, CC, DIFF, SIDE)                                            \
    {                                                                                       \
        bool any = true;                                                                    \
        if (GATED) {                                                                        \
            bool a_ = false;                                                                \
            _Pragma("unroll") for (int k = 0; k < P; k++) a_ |= (e[k] == 0);                \
            any = __any_sync(0xffffffffu, a_);                                              \
        }                                                                                   \
        if (any) {                                                                          \
            _Pragma("unroll") for (int k = 0; k < P; k++) {                                 \
                const T lp = (GATED && e[k] != 0) ? T(0) : ((S) == 0 ? vp[k] : vpo[k]);     \
                const T lm = (GATED && e[k] != 0) ? T(0) : ((S) == 0 ? vm[k] : vmo[k]);     \
                _Pragma("unroll") for (int r = 0; r < RG; r++) {                            \
                    const V4 a = s_alm[I][r];                                               \
                    if ((SIDE) == 0) {                                                      \
                        T *ac = &acc[k][r][(S) * 8];                                        \
                        ac[0] = fma(a.x, lp, ac[0]);                                        \
                        ac[1] = fma(a.y, lp, ac[1]);                                        \
                        ac[2] = fma(a.z, lm, ac[2]);                                        \
                        ac[3] = fma(a.w, lm, ac[3]);                                        \
                        ac[4] = fma(a.x, lm, ac[4]);                                        \
                        ac[5] = fma(a.y, lm, ac[5]);                                        \
                        ac[6] = fma(a.z, lp, ac[6]);                                        \
                        ac[7] = fma(a.w, lp, ac[7]);                                        \
                    } else {                                                                \
                        /* one ring: north P1 = Σ c 2λ, P2 = Σ d (-2)λ over both parities;  */ \
                        /* south P3 = Σ ± c (-2)λ, P4 = Σ ± d 2λ, + for slot A, - for slot B */ \
                        const T u = (SIDE) == 1 ? lp : ((S) == 0 ? lm : -lm);               \
                        const T v = (SIDE) == 1 ? lm : ((S) == 0 ? lp : -lp);               \
                        T *ac = &acc[k][r][0];                                              \
                        ac[0] = fma(a.x, u, ac[0]);                                         \
                        ac[1] = fma(a.y, u, ac[1]);                                         \
                        ac[2] = fma(a.z, v, ac[2]);                                         \
                        ac[3] = fma(a.w, v, ac[3]);                                         \
                    }                                                                       \
                }                                                                           \
            }                                                                               \
        }                                                                                   \
        _Pragma("unroll") for (int k = 0; k < P; k++) {                                     \
            /* the new value overwrites the older register; the roles swap every step */    \
            T &cp_ = (S) == 0 ? vp[k] : vpo[k], &op_ = (S) == 0 ? vpo[k] : vp[k];           \
            T &cm_ = (S) == 0 ? vm[k] : vmo[k], &om_ = (S) == 0 ? vmo[k] : vm[k];           \
            if (DIFF && dk[k]) {                                                            \
                /* difference form: op_ held d_l, receives μ_{l+1}; cp_ receives d_{l+1} */ \
                const float2 cb = s_cb[I];                                                  \
                const T u1 = fma((CA), y[k], (T)cb.x), u2 = fma((CA), y[k], (T)cb.y);       \
                const T d1 = fma(u1, cp_, op_), d2 = fma(u2, cm_, om_);                     \
                op_ = cp_ + d1;                                                             \
                om_ = cm_ + d2;                                                             \
                cp_ = d1;                                                                   \
                cm_ = d2;                                                                   \
            } else {                                                                        \
                const T t1 = fma((CA), x[k], (CC));                                         \
                const T t2 = fma((CA), x[k], -(CC));                                        \
                op_ = fma(t1, cp_, -op_);                                                   \
                om_ = fma(t2, cm_, -om_);                                                   \
            }                                                                               \
            if (GATED && e[k] < 0 && (fabs(op_) > Scale<T>::hi() || fabs(om_) > Scale<T>::hi())) { \
                vp[k] *= Scale<T>::inv();                                                   \
                vm[k] *= Scale<T>::inv();                                                   \
                vpo[k] *= Scale<T>::inv();                                                  \
                vmo[k] *= Scale<T>::inv();                                                  \
                e[k]++;                                                                     \
            }                                                                               \
        }                                                                                   \
    }

#define AKRA_SYNTH_LOOP(GATED, DIFF, SIDE)                                                  \
    for (int i = 0; i < nl; i += 2) {                                                       \
        const V4 cc = s_coef[i >> 1];                                                       \
        AKRA_SYNTH_STEP(i, 0, GATED, cc.x, cc.y, DIFF, SIDE)                                \
        AKRA_SYNTH_STEP(i + 1, 1, GATED, cc.z, cc.w, DIFF, SIDE)                            \
    }
#define AKRA_SYNTH_SIDES(GATED, DIFF)                                                       \
    if (side == 2) { AKRA_SYNTH_LOOP(GATED, DIFF, 2) }                                      \
    else if (side == 1) { AKRA_SYNTH_LOOP(GATED, DIFF, 1) }                                 \
    else { AKRA_SYNTH_LOOP(GATED, DIFF, 0) }
        if (!(std::is_same<T, float>::value && blk_diff)) {
            if (all_live) {
                AKRA_SYNTH_SIDES(false, false)
            } else {
                AKRA_SYNTH_SIDES(true, false)
            }
        } else if constexpr (std::is_same<T, float>::value) {
            // a block with pairs near a pole (rare): some warps run the difference form
            AKRA_SYNTH_SIDES(true, true)
        }
#undef AKRA_SYNTH_SIDES
#undef AKRA_SYNTH_LOOP
#undef AKRA_SYNTH_STEP
    }

    // combine parities into the north and south rings and write Φ(±m)
    const bool swap = ((l0 + m) & 1) != 0;   // slot A holds odd (l+m) when l0+m is odd
    const size_t row = 2 * (size_t)L + 1;
    const long long pbound = (long long)R * nring * row;   // extent of Φ
    (void)pbound;
#pragma unroll
    for (int k = 0; k < P; k++) {
        if (uid[k] < 0) continue;
        const UnitInfo ui = uinfo[AKRA_IX(uid[k], nunit_all, kDbgUnitInfo)];
#pragma unroll
        for (int rr = 0; rr < RG; rr++) {
            const int r = r0 + rr;
            if (r >= R) continue;
            if (side != 0) {
                // one ring: its Φ(m) and conj Φ(-m) directly (south: even - odd, i.e. the sign of
                // slot A, which holds odd l + m when l0 + m is odd)
                const int ring = side == 1 ? ui.ring_n : ui.ring_s;
                if (ring < 0) continue;
                if (ring_active && !ring_active[AKRA_IX(ring, nring, kDbgRingActive)]) continue;
                const T sg = (side == 2 && swap) ? T(-1) : T(1);
                const T *ac = acc[k][rr];
                const size_t pb = ((size_t)r * nring + ring) * row + L;   // Φ(ring, m = 0)
                phi[AKRA_IX(pb + m, pbound, kDbgPhiWrite)] = C2{sg * ac[0], sg * ac[1]};
                if (m > 0) phi[AKRA_IX(pb - m, pbound, kDbgPhiWrite)] = C2{sg * ac[2], -(sg * ac[3])};
                continue;
            }
            T se[8], so[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                se[j] = swap ? acc[k][rr][8 + j] : acc[k][rr][j];
                so[j] = swap ? acc[k][rr][j] : acc[k][rr][8 + j];
            }
            // north: Φ(m) = P1,  conj Φ(-m) = P2        (even + odd)
            // south: Φ(m) = P3,  conj Φ(-m) = P4        (even - odd)
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int ring = sd == 0 ? ui.ring_n : ui.ring_s;
                if (ring < 0) continue;
                if (ring_active && !ring_active[AKRA_IX(ring, nring, kDbgRingActive)]) continue;
                const int o = sd == 0 ? 0 : 4;
                const T sg = sd == 0 ? T(1) : T(-1);
                const T fr = se[o + 0] + sg * so[o + 0], fi = se[o + 1] + sg * so[o + 1];
                const T gr = se[o + 2] + sg * so[o + 2], gi = se[o + 3] + sg * so[o + 3];
                const size_t pb = ((size_t)r * nring + ring) * row + L;   // Φ(ring, m = 0)
                phi[AKRA_IX(pb + m, pbound, kDbgPhiWrite)] = C2{fr, fi};
                if (m > 0) phi[AKRA_IX(pb - m, pbound, kDbgPhiWrite)] = C2{gr, -gi};
            }
        }
    }
}

// ---------------------------------------------------------------------------
// adjoint: partial[chunk][r][idx(l,m)] = Σ_{units in chunk} (E-part, B-part) at each l
//   E-part = Σ_rings [2λ P + (-2)λ Q],  B-part = Σ_rings [2λ P - (-2)λ Q]
//   with P = G(m), Q = conj(G(-m)) of the ring's Φ' row.  With the mirror relation and
//   U1 = P_N + Q_S, U2 = Q_N + P_S, U3 = P_N - Q_S, U4 = P_S - Q_N:
//     (l+m) even: E += 2λ U1 + (-2)λ U2,  B += 2λ U3 + (-2)λ U4
//     (l+m) odd : E += 2λ U3 - (-2)λ U4,  B += 2λ U1 - (-2)λ U2
// ---------------------------------------------------------------------------
// one synthesis work item (FP32 and FP64 share the scalar item: for the synthesis, whose
// contraction reads one staged coefficient per step for all of a thread's pairs, the paired-FMA
// form measured slower -- 10.25 against 9.50 ms at Nside 2048 / lmax 4096 -- as the FMA pipe,
// not instruction issue, bounds it)
template <typename T, int P, int RG, int NT>
__device__ __forceinline__ void synth_item(const LegArgs<T> &a, int m, int chunk, int r0)
{
    __shared__ v4_t<T> s_coef[TL];
    __shared__ v4_t<T> s_alm[TL][RG];
    leg_synth_item<T, P, RG, NT>(a, m, chunk, r0, s_coef, s_alm);
}

template <typename T, int P, int RG, int NT>
__global__ void __launch_bounds__(NT) k_leg_synth(LegArgs<T> a)
{
    if (a.skip && *a.skip) return;
    const int m = blockIdx.x / a.nchunks;
    synth_item<T, P, RG, NT>(a, m, blockIdx.x - m * a.nchunks, blockIdx.y * RG);
}

// persistent form: blocks take (instance, m, chunk, RHS group) items from a queue ordered by cost
template <typename T, int P, int RG, int NT>
__global__ void __launch_bounds__(NT)
k_leg_synth_queue(const LegArgs<T> *__restrict__ insts, const int4 *__restrict__ items, int nitems,
                  int *counter)
{
    __shared__ int s_it;
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_it;
        __syncthreads();
        if (it >= nitems) break;
        const int4 w = items[it];
        const LegArgs<T> a = insts[w.x];
        if (a.skip && *a.skip) continue;
        synth_item<T, P, RG, NT>(a, w.y, w.z, w.w * RG);
    }
}

// row stride (in elements) of the per-warp transpose buffer, conflict-free for both uses: the
// FP64 item stores one scalar per lane into a column and loads 16-byte rows (34 doubles); the
// FP32 paired item stores 16-byte rows and loads 8-byte columns (36 floats)
template <typename T> struct TrStride;
template <> struct TrStride<float> { static constexpr int v = 36; };
template <> struct TrStride<double> { static constexpr int v = 34; };

// adjoint l-tile: 64 steps, shorter for FP64 with several RHS (48 KB of static smem)
template <typename T, int RG> struct AdjTile { static constexpr int v = sizeof(T) == 8 ? 64 / RG : TL; };

template <typename T, int P, int RG, int NT, int ONE = 0>
__device__ __forceinline__ void leg_adjoint_item(
    const LegArgs<T> &a, const int m, const int chunk, const int r0, v4_t<T> *s_coef,
    T (*s_red)[AdjTile<T, RG>::v][RG][4], T (*s_tr)[32][TrStride<T>::v])
{
    using C2 = cx_t<T>;
    using V4 = v4_t<T>;
    constexpr int NW = NT / 32;
    constexpr int K = 8 / RG;   // l-steps per reduction block: K * 4 * RG = 32 values per lane
    constexpr int S = TrStride<T>::v;
    static_assert(K >= 2 && K * 4 * RG == 32, "RG must be 1, 2 or 4");
    constexpr int TLA = AdjTile<T, RG>::v;
    const int L = a.L, nring = a.nring, nunits = a.nunits, nunit_all = a.nunit_all, R = a.R;
    const long long ntri = a.ntri;
    const int *__restrict__ units = a.units;
    const UnitInfo *__restrict__ uinfo = a.uinfo;
    const v4_t<T> *__restrict__ coef = a.coef;
    const v4_t<T> *__restrict__ seeds = a.seeds;
    const int2 *__restrict__ start = a.start;
    const unsigned char *__restrict__ ring_active = a.ring_active;
    const cx_t<T> *__restrict__ phi = a.phi_in;
    T *__restrict__ partial = a.partial;
    const int l0 = m > 2 ? m : 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    (void)NW;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const size_t row = 2 * (size_t)L + 1;
    const bool swap = ((l0 + m) & 1) != 0;
    const long long tbound = (long long)(L + 1) * nunit_all;        // extent of the start tables
    const long long pbound = (long long)R * nring * row;            // extent of Φ'
    const long long qbound = (long long)a.nchunks * R * ntri * 4;   // extent of the partial sums
    (void)pbound;
    (void)qbound;

    T x[P], vp[P], vm[P], vpo[P], vmo[P];
    int e[P], uid[P], gs[P];
    int my_first = kNeverLive;
    // per unit and RHS, the partners of 2λ and (-2)λ in slot A (l - l0 even):
    //   E += 2λ X1 + (-2)λ X2,  B += 2λ X3 + (-2)λ X4;   slot B: E += 2λ X3 - (-2)λ X4,
    //   B += 2λ X1 - (-2)λ X2   (X = U1..U4, or U3, -U4, U1, -U2 when l0+m is odd)
    // ONE = 1 or 2: every pair needs only its north / south ring (only the one-ring form is
    // compiled, and X3, X4 are dead)
    C2 X1[P][RG], X2[P][RG], X3[P][RG], X4[P][RG];
    int rn[P], rs[P];
    int my_side = 3;
#pragma unroll
    for (int k = 0; k < P; k++) {
        // each warp holds 32 P consecutive pairs (close in latitude, so close in start point)
        const int iu = chunk * P * NT + warp * 32 * P + k * 32 + lane;
        const int u = iu < nunits ? (units ? units[AKRA_IX(iu, nunits, kDbgUnits)] : iu) : -1;
        uid[k] = u;
        x[k] = 0;
        vp[k] = vm[k] = vpo[k] = vmo[k] = 0;
        e[k] = 0;
        gs[k] = kNeverLive;
        rn[k] = rs[k] = -1;
        if (u >= 0) {
            const UnitInfo ui = uinfo[AKRA_IX(u, nunit_all, kDbgUnitInfo)];
            x[k] = (T)ui.x;
            gs[k] = start[AKRA_IX((size_t)m * nunit_all + u, tbound, kDbgStart)].x;
            rn[k] = ui.ring_n;
            rs[k] = ui.ring_s;
            my_side = side_join(my_side, unit_side(ui, ring_active, nring));
        }
        my_first = min(my_first, gs[k]);
    }
    // one ring per pair over the whole warp: X1 holds Xa (partner of 2λ), X2 Xb (of (-2)λ), and the
    // contraction keeps a = Σ 2λ Xa, b = Σ (-2)λ Xb, from which E and B follow
    const int side = ONE ? ONE : warp_side(my_side);
    (void)my_side;
#pragma unroll
    for (int k = 0; k < P; k++) {
#pragma unroll
        for (int rr = 0; rr < RG; rr++) {
            const int r = r0 + rr;
            C2 Pv[2], Qv[2];
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int ring = sd == 0 ? rn[k] : rs[k];
                Pv[sd] = C2{0, 0};
                Qv[sd] = C2{0, 0};
                if (ring < 0 || r >= R) continue;
                if (ring_active && !ring_active[AKRA_IX(ring, nring, kDbgRingActive)]) continue;
                const size_t pb = ((size_t)r * nring + ring) * row + L;   // Φ'(ring, m = 0)
                const C2 g = phi[AKRA_IX(pb + m, pbound, kDbgPhiRead)];
                const C2 gm = phi[AKRA_IX(pb - m, pbound, kDbgPhiRead)];
                Pv[sd] = g;
                Qv[sd] = C2{gm.x, -gm.y};
            }
            if (side == 1) {          // north: Xa = P_N, Xb = Q_N
                X1[k][rr] = Pv[0];
                X2[k][rr] = Qv[0];
                X3[k][rr] = X4[k][rr] = C2{0, 0};
            } else if (side == 2) {   // south: Xa = Q_S, Xb = P_S
                X1[k][rr] = Qv[1];
                X2[k][rr] = Pv[1];
                X3[k][rr] = X4[k][rr] = C2{0, 0};
            } else {
                const C2 u1{Pv[0].x + Qv[1].x, Pv[0].y + Qv[1].y};
                const C2 u2{Qv[0].x + Pv[1].x, Qv[0].y + Pv[1].y};
                const C2 u3{Pv[0].x - Qv[1].x, Pv[0].y - Qv[1].y};
                const C2 u4{Pv[1].x - Qv[0].x, Pv[1].y - Qv[0].y};
                X1[k][rr] = swap ? u3 : u1;
                X2[k][rr] = swap ? C2{-u4.x, -u4.y} : u2;
                X3[k][rr] = swap ? u1 : u3;
                X4[k][rr] = swap ? C2{-u2.x, -u2.y} : u4;
            }
        }
    }

    T (*tr)[S] = s_tr[warp];
    const int warp_first = __reduce_min_sync(0xffffffffu, my_first);
    const int l_first = block_min_start<NT>(my_first);
    // the l below the first start get zero partial sums
    for (int i = tid; i < (min(l_first, L + 1) - l0) * RG * 4; i += NT) {
        const int step = i / (RG * 4), rem = i - step * RG * 4, rr = rem >> 2, q = rem & 3;
        const int r = r0 + rr;
        if (r < R)
            partial[AKRA_IX((((size_t)chunk * R + r) * ntri + mbase + l0 + step) * 4 + q, qbound,
                            kDbgPartialWrite)] = T(0);
    }
    for (int lt = l_first; lt <= L; lt += TLA) {
        __syncthreads();
        for (int i = tid; i < TLA; i += NT) {
            const int l = lt + i;
            s_coef[i] = (l <= L) ? coef[AKRA_IX(mbase + l, ntri, kDbgCoef)] : V4{0, 0, 0, 0};
        }
        __syncthreads();
        const int nl = min(TLA, L - lt + 1);
        start_pairs(seeds, start, (size_t)m * nunit_all, tbound, lt, uid, gs, vp, vm, vpo, vmo, e);
        if (warp_first > lt + TLA - 1) {
            // none of this warp's pairs has started yet: its rows of the tile sum are zero
            T *zr = &s_red[warp][0][0][0];
            for (int i = lane; i < TLA * RG * 4; i += 32) zr[i] = T(0);
        } else {
        bool live = true;
#pragma unroll
        for (int k = 0; k < P; k++) live &= (e[k] == 0);
        const bool all_live = __all_sync(0xffffffffu, live);
        const int nkb = (nl + K - 1) / K;

        // K l-steps into ta[K][RG][4] (slot of step kk = parity of kk), then recur
#define AKRA_ADJ_KBLOCK(GATED, SIDE)                                                            \
    for (int kb = 0; kb < nkb; kb++) {                                                          \
        T ta[K][RG][4];                                                                         \
        _Pragma("unroll") for (int kk = 0; kk < K; kk++)                                        \
            _Pragma("unroll") for (int rr = 0; rr < RG; rr++)                                   \
                _Pragma("unroll") for (int q = 0; q < 4; q++) ta[kk][rr][q] = 0;                \
        _Pragma("unroll") for (int kk = 0; kk < K; kk++) {                                      \
            const V4 c = s_coef[kb * K + kk];                                                   \
            const bool slotA = (kk & 1) == 0;                                                   \
            bool any = true;                                                                    \
            if (GATED) {                                                                        \
                bool a_ = false;                                                                \
                _Pragma("unroll") for (int k = 0; k < P; k++) a_ |= (e[k] == 0);                \
                any = __any_sync(0xffffffffu, a_);                                              \
            }                                                                                   \
            if (any) {                                                                          \
                _Pragma("unroll") for (int k = 0; k < P; k++) {                                 \
                    const T lp = (GATED && e[k] != 0) ? T(0) : (slotA ? vp[k] : vpo[k]);        \
                    const T lm0 = (GATED && e[k] != 0) ? T(0) : (slotA ? vm[k] : vmo[k]);       \
                    const T lm = slotA ? lm0 : -lm0;                                            \
                    _Pragma("unroll") for (int rr = 0; rr < RG; rr++) {                         \
                        T *t = ta[kk][rr];                                                      \
                        if ((SIDE) == 0) {                                                      \
                            const C2 eP = slotA ? X1[k][rr] : X3[k][rr];                        \
                            const C2 eM = slotA ? X2[k][rr] : X4[k][rr];                        \
                            const C2 bP = slotA ? X3[k][rr] : X1[k][rr];                        \
                            const C2 bM = slotA ? X4[k][rr] : X2[k][rr];                        \
                            t[0] = fma(lp, eP.x, fma(lm, eM.x, t[0]));                          \
                            t[1] = fma(lp, eP.y, fma(lm, eM.y, t[1]));                          \
                            t[2] = fma(lp, bP.x, fma(lm, bM.x, t[2]));                          \
                            t[3] = fma(lp, bP.y, fma(lm, bM.y, t[3]));                          \
                        } else {                                                                \
                            /* one ring: a = Σ 2λ Xa, b = Σ (-2)λ Xb */                         \
                            t[0] = fma(lp, X1[k][rr].x, t[0]);                                  \
                            t[1] = fma(lp, X1[k][rr].y, t[1]);                                  \
                            t[2] = fma(lm0, X2[k][rr].x, t[2]);                                 \
                            t[3] = fma(lm0, X2[k][rr].y, t[3]);                                 \
                        }                                                                       \
                    }                                                                           \
                }                                                                               \
            }                                                                                   \
            _Pragma("unroll") for (int k = 0; k < P; k++) {                                     \
                const T t1 = fma(c.x, x[k], c.y);                                               \
                const T t2 = fma(c.x, x[k], -c.y);                                              \
                /* the new value overwrites the older register (K is even) */               \
                T &cp_ = slotA ? vp[k] : vpo[k], &op_ = slotA ? vpo[k] : vp[k];                 \
                T &cm_ = slotA ? vm[k] : vmo[k], &om_ = slotA ? vmo[k] : vm[k];                 \
                op_ = fma(t1, cp_, -op_);                                                       \
                om_ = fma(t2, cm_, -om_);                                                       \
                if (GATED && e[k] < 0 &&                                                        \
                    (fabs(op_) > Scale<T>::hi() || fabs(om_) > Scale<T>::hi())) {               \
                    vp[k] *= Scale<T>::inv();                                                   \
                    vm[k] *= Scale<T>::inv();                                                   \
                    vpo[k] *= Scale<T>::inv();                                                  \
                    vmo[k] *= Scale<T>::inv();                                                  \
                    e[k]++;                                                                     \
                }                                                                               \
            }                                                                                   \
        }                                                                                       \
        /* warp transpose through shared memory: lane L's value i goes to tr[i][L]; lane j */  \
        /* then sums row j, i.e. value j over all lanes */                                       \
        _Pragma("unroll") for (int kk = 0; kk < K; kk++)                                        \
            _Pragma("unroll") for (int rr = 0; rr < RG; rr++)                                   \
                _Pragma("unroll") for (int q = 0; q < 4; q++)                                   \
                    tr[(kk * RG + rr) * 4 + q][lane] = ta[kk][rr][q];                           \
        __syncwarp();                                                                           \
        T sum = 0;                                                                              \
        _Pragma("unroll") for (int i = 0; i < 32; i++) sum += tr[lane][i];                      \
        __syncwarp();                                                                           \
        {                                                                                       \
            const int kk = lane / (4 * RG), rr = (lane / 4) % RG, q = lane & 3;                 \
            T val = sum;                                                                        \
            if ((SIDE) != 0) {                                                                  \
                /* one ring: the lanes hold the totals of (a.re, a.im, b.re, b.im); with the */  \
                /* partner's (lane ^ 2): north E = a + b, B = a - b; south E = s (a + b), */     \
                /* B = s (b - a), s = +1 in slot A unless swapped */                            \
                const T other = __shfl_xor_sync(0xffffffffu, sum, 2);                           \
                if ((SIDE) == 1) {                                                              \
                    val = q < 2 ? sum + other : other - sum;                                    \
                } else {                                                                        \
                    const T sg = (((kk & 1) == 0) != swap) ? T(1) : T(-1);                      \
                    val = sg * (q < 2 ? sum + other : sum - other);                             \
                }                                                                               \
            }                                                                                   \
            s_red[warp][kb * K + kk][rr][q] = val;                                              \
        }                                                                                       \
    }

#define AKRA_ADJ_SIDES(GATED)                                                                   \
    if constexpr (ONE == 1) { AKRA_ADJ_KBLOCK(GATED, 1) }                                       \
    else if constexpr (ONE == 2) { AKRA_ADJ_KBLOCK(GATED, 2) }                                  \
    else {                                                                                      \
        if (side == 2) { AKRA_ADJ_KBLOCK(GATED, 2) }                                            \
        else if (side == 1) { AKRA_ADJ_KBLOCK(GATED, 1) }                                       \
        else { AKRA_ADJ_KBLOCK(GATED, 0) }                                                      \
    }
        if (all_live) {
            AKRA_ADJ_SIDES(false)
        } else {
            AKRA_ADJ_SIDES(true)
        }
#undef AKRA_ADJ_SIDES
#undef AKRA_ADJ_KBLOCK
        }
        __syncthreads();
        // sum the warps and write this chunk's partial sums for the tile
        for (int i = tid; i < nl * RG * 4; i += NT) {
            const int step = i / (RG * 4), rem = i - step * RG * 4, rr = rem >> 2, q = rem & 3;
            const int r = r0 + rr;
            if (r >= R) continue;
            T sv = 0;
#pragma unroll
            for (int w = 0; w < NW; w++) sv += s_red[w][step][rr][q];
            // the recurrence ran on μ_l = λ_l / σ_l
            partial[AKRA_IX((((size_t)chunk * R + r) * ntri + mbase + lt + step) * 4 + q, qbound,
                            kDbgPartialWrite)] = sv * s_coef[step].z;
        }
    }
}

// one adjoint work item: FP32 with paired FMAs (ONE: see leg_adjoint_item_f2), FP64 scalar
template <typename T, int P, int RG, int NT, int ONE = 0>
__device__ __forceinline__ void adjoint_item(const LegArgs<T> &a, int m, int chunk, int r0)
{
    if constexpr (std::is_same<T, float>::value) {
        __shared__ float4 s_cf[TL];
        __shared__ float s_sig[TL];
        __shared__ float s_red[NT / 32][TL][RG][4];
        __shared__ __align__(16) float s_tr[NT / 32][32][36];
        __shared__ float4 s_cfd[TL];
        leg_adjoint_item_f2<P, RG, NT, ONE>(a, m, chunk, r0, s_cf, s_sig, s_red, s_tr, s_cfd);
    } else {
        __shared__ v4_t<T> s_coef[AdjTile<T, RG>::v];
        __shared__ T s_red[NT / 32][AdjTile<T, RG>::v][RG][4];
        __shared__ __align__(16) T s_tr[NT / 32][32][TrStride<T>::v];
        leg_adjoint_item<T, P, RG, NT, ONE>(a, m, chunk, r0, s_coef, s_red, s_tr);
    }
}

template <typename T, int P, int RG, int NT, int ONE = 0>
__global__ void __launch_bounds__(NT) k_leg_adjoint(LegArgs<T> a)
{
    if (a.skip && *a.skip) return;
    const int m = blockIdx.x / a.nchunks;
    adjoint_item<T, P, RG, NT, ONE>(a, m, blockIdx.x - m * a.nchunks, blockIdx.y * RG);
}

template <typename T, int P, int RG, int NT>
__global__ void __launch_bounds__(NT)
k_leg_adjoint_queue(const LegArgs<T> *__restrict__ insts, const int4 *__restrict__ items, int nitems,
                    int *counter)
{
    __shared__ int s_it;
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_it;
        __syncthreads();
        if (it >= nitems) break;
        const int4 w = items[it];
        const LegArgs<T> a = insts[w.x];
        if (a.skip && *a.skip) continue;
        adjoint_item<T, P, RG, NT>(a, w.y, w.z, w.w * RG);
    }
}


}  // namespace akra
