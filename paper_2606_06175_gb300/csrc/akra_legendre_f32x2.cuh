// akra_legendre_f32x2.cuh -- the FP32 Legendre adjoint with paired FP32 FMAs (sm_100 family:
// one fma.rn.f32x2 instruction performs two independent, correctly rounded FP32 FMAs; it
// occupies the FMA pipe for two cycles but takes one issue slot).
//
// The two spin recurrences of a ring pair advance together as one float2 (λ+, λ-):
//   * recurrence: T = (A'x + c', A'x - c') is one paired FMA, the update another (2 issues per
//     pair-step instead of 4);
//   * contraction: the ring-pair data are paired across the spins, (X+, X-), and
//     (Σ λ+ X+, Σ λ- X-) += (λ+, λ-)·(X+, X-), the two halves added once per value after the
//     warp's sum over its lanes: 4 paired FMAs per pair-step and RHS instead of 8.
// The adjoint, which also spends issue slots on its warp reduction, gains from the freed
// slots (12.77 -> 12.08 ms at Nside 2048 / lmax 4096); the synthesis, bound by the FMA pipe
// itself, does not and keeps the scalar form.  The recurrences round every product and sum as
// the scalar form does; the contraction sums the two spins' terms in separate partial sums,
// added once per step (another summation order, the same FP32 accuracy).
//
// Sign-alternated state: with s_l = (-1)^floor((l - l0)/2) the monic recurrence
// μ_{l+1} = t_l μ_l - μ_{l-1} becomes, for ξ_l = s_l μ_l,
//     ξ_{l+1} = r_l t_l ξ_l + ξ_{l-1},   r_l = s_{l+1}/s_l = +1 (l - l0 even), -1 (odd),
// an update with no negated operand.  r_l is folded into the staged coefficients, s_l into
// the staged coefficients of the synthesis and into the per-l scale of the partial sums of the
// adjoint; the
// start state (μ_g, μ_{g-1}) at a grid point g (g - l0 a multiple of 64) is (ξ_g, -ξ_{g-1}).
// The tensor-core synthesis (akra_legendre_tc.cu) runs the same sign-alternated recurrence.
// Sign flips are exact, so the arithmetic is the scalar form's.
#pragma once
#include "akra_internal.cuh"

namespace akra {

__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// recurrence coefficients of step i of a tile (l = lt + i), sign r folded in: {rA', rA', rc', -rc'}
__device__ __forceinline__ float4 f2_coef_entry(const float4 c, int i)
{
    const float r = (i & 1) ? -1.f : 1.f;
    return make_float4(r * c.x, r * c.x, r * c.y, -r * c.y);
}

// s_l relative to a tile start lt (lt - l0 a multiple of 64): s = (-1)^floor(i/2)
__device__ __forceinline__ float f2_sign(int i) { return (i & 2) ? -1.f : 1.f; }

template <int P>
__device__ __forceinline__ void f2_start_pairs(const float4 *__restrict__ seeds, const int2 *__restrict__ start,
                                               size_t base, long long tbound, int lt, const int (&uid)[P],
                                               const int (&gs)[P], float2 (&V)[P], float2 (&VO)[P], int (&e)[P])
{
    (void)tbound;
#pragma unroll
    for (int k = 0; k < P; k++) {
        if (gs[k] == lt) {
            const float4 s = seeds[AKRA_IX(base + uid[k], tbound, kDbgSeeds)];
            V[k] = make_float2(s.x, s.y);
            VO[k] = make_float2(-s.z, -s.w);   // ξ_{g-1} = -μ_{g-1}
            e[k] = start[AKRA_IX(base + uid[k], tbound, kDbgStart)].y;
        }
    }
}

// exponent-index rescale of a pair whose state is still below the float range
template <int P>
__device__ __forceinline__ void f2_rescale(int k, float2 (&V)[P], float2 (&VO)[P], int (&e)[P], const float2 nw)
{
    if (e[k] < 0 && (fabsf(nw.x) > Scale<float>::hi() || fabsf(nw.y) > Scale<float>::hi())) {
        const float2 s = make_float2(Scale<float>::inv(), Scale<float>::inv());
        V[k] = __fmul2_rn(V[k], s);
        VO[k] = __fmul2_rn(VO[k], s);
        e[k]++;
    }
}

// ---------------------------------------------------------------------------
// adjoint: partial[chunk][r][idx(l,m)] = Σ_{units in chunk} (E-part, B-part) at each l (FP32,
// paired FMAs).  Per unit and RHS the spin-paired data are Q0 = (X1.re, X2.re),
// Q1 = (X1.im, X2.im), Q2 = (X3.re, X4.re), Q3 = (X3.im, X4.im) (X1..X4 as in the scalar item),
// and per step Fj = Σ_units (λ+, λ-)·Qj.  Then, for l - l0 even, E = (F0.x + F0.y) + i (F1.x + F1.y)
// and B = (F2.x + F2.y) + i (F3.x + F3.y); for l - l0 odd, E = (F2.x - F2.y) + i (F3.x - F3.y) and
// B = (F0.x - F0.y) + i (F1.x - F1.y).
// ---------------------------------------------------------------------------
// ONE = 1 or 2: every ring pair of the launch needs only its north (1) or south (2) ring, so only
// that form is compiled (half the Φ' registers); ONE = 0 decides per warp.
template <int P, int RG, int NT, int ONE = 0>
__device__ __forceinline__ void leg_adjoint_item_f2(const LegArgs<float> &a, const int m, const int chunk,
                                                    const int r0, float4 *s_cf, float *s_sig,
                                                    float (*s_red)[TL][RG][4], float (*s_tr)[32][36],
                                                    float4 *s_cfd)
{
    // s_cfd: difference-form coefficients {A', A', (A'-2) + c', (A'-2) - c'} per step, staged only in
    // blocks that hold ring pairs near a pole
    constexpr int NW = NT / 32;
    constexpr int K = 8 / RG;   // l-steps per block of the step loop (one or two reduction groups)
    static_assert(K >= 2 && K * 4 * RG == 32, "RG must be 1, 2 or 4");
    const int L = a.L, nring = a.nring, nunits = a.nunits, nunit_all = a.nunit_all, R = a.R;
    const long long ntri = a.ntri;
    const int *__restrict__ units = a.units;
    const UnitInfo *__restrict__ uinfo = a.uinfo;
    const float4 *__restrict__ coef = a.coef;
    const float4 *__restrict__ seeds = a.seeds;
    const int2 *__restrict__ start = a.start;
    const unsigned char *__restrict__ ring_active = a.ring_active;
    const float2 *__restrict__ phi = a.phi_in;
    float *__restrict__ partial = a.partial;
    const int l0 = m > 2 ? m : 2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const size_t row = 2 * (size_t)L + 1;
    const bool swap = ((l0 + m) & 1) != 0;
    const long long tbound = (long long)(L + 1) * nunit_all;    // extent of the start tables
    const long long pbound = (long long)R * nring * row;        // extent of Φ'
    const long long qbound = (long long)a.nchunks * R * ntri * 4;   // extent of the partial sums
    (void)pbound;
    (void)qbound;

    float2 X2[P], V[P], VO[P];   // X2 = (x, x), or (x - 1, x - 1) for the difference form
    int e[P], uid[P], gs[P];
    bool dk[P];                  // this warp's pairs of slot k run the difference form (warp-uniform)
    int my_first = kNeverLive;
    bool any_diff = false;
    int my_side = 3;
    int rn[P], rs[P];            // the pair's north and south rings
    // Q: the spin-paired Φ' data; with one ring per pair (side 1: north, 2: south) only Q[.][.][0..1]
    // = ((Xa.re, Xb.re), (Xa.im, Xb.im)), Xa / Xb the partners of 2λ / (-2)λ
    float2 Q[P][RG][ONE ? 2 : 4];
#pragma unroll
    for (int k = 0; k < P; k++) {
        // each warp holds 32 P consecutive pairs (close in latitude, so close in start point)
        const int iu = chunk * P * NT + warp * 32 * P + k * 32 + lane;
        const int u = iu < nunits ? (units ? units[AKRA_IX(iu, nunits, kDbgUnits)] : iu) : -1;
        uid[k] = u;
        X2[k] = make_float2(0.f, 0.f);
        V[k] = VO[k] = make_float2(0.f, 0.f);
        e[k] = 0;
        gs[k] = kNeverLive;
        UnitInfo ui;
        ui.ring_n = ui.ring_s = -1;
        bool polar = false;
        if (u >= 0) {
            ui = uinfo[AKRA_IX(u, nunit_all, kDbgUnitInfo)];
            polar = ui.x >= kDiffX;
            gs[k] = start[AKRA_IX((size_t)m * nunit_all + u, tbound, kDbgStart)].x;
            my_side = side_join(my_side, unit_side(ui, ring_active, nring));
        }
        dk[k] = __any_sync(0xffffffffu, polar);
        any_diff |= dk[k];
        if (u >= 0) {
            // x - 1 = -2 sin^2(θ/2), accurate near the pole
            const float x = dk[k] ? (float)(-exp2(2.0 * ui.ls + 1.0)) : (float)ui.x;
            X2[k] = make_float2(x, x);
        }
        my_first = min(my_first, gs[k]);
        rn[k] = ui.ring_n;
        rs[k] = ui.ring_s;
    }
    // one ring per pair over the whole warp (a footprint in one hemisphere): the contraction keeps
    // a = Σ 2λ Xa and b = Σ (-2)λ Xb and forms E and B from them after the sum over the pairs
    const int side = ONE ? ONE : warp_side(my_side);
    (void)my_side;
#pragma unroll
    for (int k = 0; k < P; k++) {
#pragma unroll
        for (int rr = 0; rr < RG; rr++) {
            const int r = r0 + rr;
            float2 Pv[2], Qv[2];
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int ring = sd == 0 ? rn[k] : rs[k];
                Pv[sd] = make_float2(0.f, 0.f);
                Qv[sd] = make_float2(0.f, 0.f);
                if (ring < 0 || r >= R) continue;
                if (ring_active && !ring_active[AKRA_IX(ring, nring, kDbgRingActive)]) continue;
                const size_t pb = ((size_t)r * nring + ring) * row + L;   // Φ'(ring, m = 0)
                const float2 g = phi[AKRA_IX(pb + m, pbound, kDbgPhiRead)];
                const float2 gm = phi[AKRA_IX(pb - m, pbound, kDbgPhiRead)];
                Pv[sd] = g;
                Qv[sd] = make_float2(gm.x, -gm.y);
            }
            if (side == 1) {          // north: Xa = P_N, Xb = Q_N
                Q[k][rr][0] = make_float2(Pv[0].x, Qv[0].x);
                Q[k][rr][1] = make_float2(Pv[0].y, Qv[0].y);
            } else if (side == 2) {   // south: Xa = Q_S, Xb = P_S
                Q[k][rr][0] = make_float2(Qv[1].x, Pv[1].x);
                Q[k][rr][1] = make_float2(Qv[1].y, Pv[1].y);
            } else if constexpr (ONE == 0) {
                const float2 u1 = make_float2(Pv[0].x + Qv[1].x, Pv[0].y + Qv[1].y);
                const float2 u2 = make_float2(Qv[0].x + Pv[1].x, Qv[0].y + Pv[1].y);
                const float2 u3 = make_float2(Pv[0].x - Qv[1].x, Pv[0].y - Qv[1].y);
                const float2 u4 = make_float2(Pv[1].x - Qv[0].x, Pv[1].y - Qv[0].y);
                const float2 x1 = swap ? u3 : u1;
                const float2 x2 = swap ? make_float2(-u4.x, -u4.y) : u2;
                const float2 x3 = swap ? u1 : u3;
                const float2 x4 = swap ? make_float2(-u2.x, -u2.y) : u4;
                Q[k][rr][0] = make_float2(x1.x, x2.x);
                Q[k][rr][1] = make_float2(x1.y, x2.y);
                Q[k][rr][2] = make_float2(x3.x, x4.x);
                Q[k][rr][3] = make_float2(x3.y, x4.y);
            }
        }
    }

    float (*tr)[36] = s_tr[warp];
    const int warp_first = __reduce_min_sync(0xffffffffu, my_first);
    const int l_first = block_min_start<NT>(my_first);
    const bool blk_diff = __syncthreads_or(any_diff) != 0;   // block-uniform
    // the l below the first start get zero partial sums
    for (int i = tid; i < (min(l_first, L + 1) - l0) * RG * 4; i += NT) {
        const int step = i / (RG * 4), rem = i - step * RG * 4, rr = rem >> 2, q = rem & 3;
        const int r = r0 + rr;
        if (r < R)
            partial[AKRA_IX((((size_t)chunk * R + r) * ntri + mbase + l0 + step) * 4 + q, qbound,
                            kDbgPartialWrite)] = 0.f;
    }
    for (int lt = l_first; lt <= L; lt += TL) {
        __syncthreads();
        for (int i = tid; i < TL; i += NT) {
            const int l = lt + i;
            const float4 c = (l <= L) ? coef[AKRA_IX(mbase + l, ntri, kDbgCoef)] : make_float4(0.f, 0.f, 0.f, 0.f);
            s_cf[i] = f2_coef_entry(c, i);
            s_sig[i] = c.z * f2_sign(i);   // the recurrence ran on ξ_l = s_l λ_l / σ_l
            if (blk_diff) s_cfd[i] = make_float4(c.x, c.x, c.w + c.y, c.w - c.y);
        }
        __syncthreads();
        const int nl = min(TL, L - lt + 1);
        f2_start_pairs<P>(seeds, start, (size_t)m * nunit_all, tbound, lt, uid, gs, V, VO, e);
        if (blk_diff) {
#pragma unroll
            for (int k = 0; k < P; k++)
                if (dk[k] && gs[k] == lt)   // difference form: second register holds μ_g - μ_{g-1}
                    VO[k] = a.dseeds[AKRA_IX((size_t)m * nunit_all + uid[k], tbound, kDbgSeeds)];
        }
        if (warp_first > lt + TL - 1) {
            // none of this warp's pairs has started yet: its rows of the tile sum are zero
            float *zr = &s_red[warp][0][0][0];
            for (int i = lane; i < TL * RG * 4; i += 32) zr[i] = 0.f;
        } else {
        bool live = true;
#pragma unroll
        for (int k = 0; k < P; k++) live &= (e[k] == 0);
        const bool all_live = __all_sync(0xffffffffu, live);
        const int nkb = (nl + K - 1) / K;

        // K l-steps (slot of step kk = parity of kk); every KR_ steps the warp sums its lanes' raw
        // (λ+, λ-)-paired sums through the transpose buffer and forms E and B from the totals
#define AKRA_F2_ADJ_KBLOCK(GATED, DIFF, SIDE)                                                   \
    for (int kb = 0; kb < nkb; kb++) {                                                          \
        /* NV_ float2 sums per step and RHS; KR_ steps fill a reduction group of 16 float2 */     \
        constexpr int NV_ = (SIDE) == 0 ? 4 : 2, KR_ = 16 / (NV_ * RG);                         \
        _Pragma("unroll") for (int kk = 0; kk < K; kk++) {                                      \
            const bool slotA = (kk & 1) == 0;                                                   \
            float2 F[RG][4];                                                                    \
            _Pragma("unroll") for (int rr = 0; rr < RG; rr++)                                   \
                _Pragma("unroll") for (int j = 0; j < 4; j++) F[rr][j] = make_float2(0.f, 0.f); \
            bool any = true;                                                                    \
            if (GATED) {                                                                        \
                bool a_ = false;                                                                \
                _Pragma("unroll") for (int k = 0; k < P; k++) a_ |= (e[k] == 0);                \
                any = __any_sync(0xffffffffu, a_);                                              \
            }                                                                                   \
            if (any) {                                                                          \
                _Pragma("unroll") for (int k = 0; k < P; k++) {                                 \
                    const float2 cur = slotA ? V[k] : VO[k];                                    \
                    /* difference form: the state is μ; the contraction takes ξ = s_l μ, with */ \
                    /* s_l from the step's index in the tile (K = 2 at RG = 4: kk alone misses it) */ \
                    const float2 cx = (DIFF && dk[k] && ((kb * K + kk) & 2)) ? make_float2(-cur.x, -cur.y) : cur; \
                    const float2 lam = (GATED && e[k] != 0) ? make_float2(0.f, 0.f) : cx;       \
                    _Pragma("unroll") for (int rr = 0; rr < RG; rr++)                           \
                        _Pragma("unroll") for (int j = 0; j < ((SIDE) == 0 ? 4 : 2); j++)       \
                            F[rr][j] = f2fma(lam, Q[k][rr][j], F[rr][j]);                       \
                }                                                                               \
            }                                                                                   \
            /* this lane's raw sums of the step go to its row of the warp's buffer (row-major, */ \
            /* 16-byte stores); E and B are formed after the sum over the lanes */                \
            _Pragma("unroll") for (int rr = 0; rr < RG; rr++) {                                 \
                float4 *dst = reinterpret_cast<float4 *>(                                       \
                    &tr[lane][((kk % KR_) * RG + rr) * NV_ * 2]);                               \
                dst[0] = make_float4(F[rr][0].x, F[rr][0].y, F[rr][1].x, F[rr][1].y);           \
                if ((SIDE) == 0) dst[1] = make_float4(F[rr][2].x, F[rr][2].y, F[rr][3].x, F[rr][3].y); \
            }                                                                                   \
            const float4 cf = s_cf[kb * K + kk];                                                \
            _Pragma("unroll") for (int k = 0; k < P; k++) {                                     \
                if (DIFF && dk[k]) {                                                            \
                    /* d_{l+1} = u μ_l + d_l, μ_{l+1} = μ_l + d_{l+1}: the register that held d_l */ \
                    /* receives μ_{l+1}, the one that held μ_l receives d_{l+1} */             \
                    const float4 cd = s_cfd[kb * K + kk];                                       \
                    const float2 uu = f2fma(make_float2(cd.x, cd.y), X2[k], make_float2(cd.z, cd.w)); \
                    if (slotA) {                                                                \
                        const float2 dn = f2fma(uu, V[k], VO[k]);                               \
                        VO[k] = __fadd2_rn(V[k], dn);                                           \
                        V[k] = dn;                                                              \
                        if (GATED) f2_rescale<P>(k, V, VO, e, VO[k]);                           \
                    } else {                                                                    \
                        const float2 dn = f2fma(uu, VO[k], V[k]);                               \
                        V[k] = __fadd2_rn(VO[k], dn);                                           \
                        VO[k] = dn;                                                             \
                        if (GATED) f2_rescale<P>(k, V, VO, e, V[k]);                            \
                    }                                                                           \
                } else {                                                                        \
                    const float2 t = f2fma(make_float2(cf.x, cf.y), X2[k], make_float2(cf.z, cf.w)); \
                    if (slotA) {                                                                \
                        VO[k] = f2fma(t, V[k], VO[k]);                                          \
                        if (GATED) f2_rescale<P>(k, V, VO, e, VO[k]);                           \
                    } else {                                                                    \
                        V[k] = f2fma(t, VO[k], V[k]);                                           \
                        if (GATED) f2_rescale<P>(k, V, VO, e, V[k]);                            \
                    }                                                                           \
                }                                                                               \
            }                                                                                   \
            if ((kk + 1) % KR_ == 0) {                                                          \
                /* a group of KR_ steps: 16 float2 per lane.  Lane (h, v) sums value v over the */ \
                /* rows (lanes) 16h .. 16h+15, the two halves are added, and half h forms the */  \
                /* E part (h = 0) or the B part (h = 1) of that value */                          \
                __syncwarp();                                                                   \
                const int h_ = lane >> 4, v_ = lane & 15;                                       \
                const float2 *c2 = reinterpret_cast<const float2 *>(&tr[16 * h_][0]) + v_;      \
                float2 sm = make_float2(0.f, 0.f);                                              \
                _Pragma("unroll") for (int t = 0; t < 16; t++) sm = __fadd2_rn(sm, c2[t * 18]); \
                sm.x += __shfl_xor_sync(0xffffffffu, sm.x, 16);                                 \
                sm.y += __shfl_xor_sync(0xffffffffu, sm.y, 16);                                 \
                __syncwarp();                                                                   \
                const int pp = v_ / (NV_ * RG), rr = (v_ / NV_) % RG, j = v_ % NV_;             \
                const int st = kb * K + kk + 1 - KR_ + pp;                                      \
                const bool sa = (st & 1) == 0;                                                  \
                if ((SIDE) == 1) {                                                              \
                    /* north: E = a + b, B = a - b */                                           \
                    s_red[warp][st][rr][j + 2 * h_] = h_ == 0 ? sm.x + sm.y : sm.x - sm.y;      \
                } else if ((SIDE) == 2) {                                                       \
                    /* south: E = s (a + b), B = s (b - a), s = +1 in slot A unless swapped */  \
                    const float sg = (sa != swap) ? 1.f : -1.f;                                 \
                    s_red[warp][st][rr][j + 2 * h_] = sg * (h_ == 0 ? sm.x + sm.y : sm.y - sm.x); \
                } else if (h_ == 0) {                                                           \
                    /* slot A: (E, B) = F0..F3 summed; slot B: E = F2, F3 and B = F0, F1 differenced */ \
                    s_red[warp][st][rr][sa ? j : (j ^ 2)] = sa ? sm.x + sm.y : sm.x - sm.y;     \
                }                                                                               \
            }                                                                                   \
        }                                                                                       \
    }

#define AKRA_F2_ADJ_SIDES(GATED, DIFF)                                                          \
    if constexpr (ONE == 1) { AKRA_F2_ADJ_KBLOCK(GATED, DIFF, 1) }                              \
    else if constexpr (ONE == 2) { AKRA_F2_ADJ_KBLOCK(GATED, DIFF, 2) }                         \
    else {                                                                                      \
        if (side == 2) { AKRA_F2_ADJ_KBLOCK(GATED, DIFF, 2) }                                   \
        else if (side == 1) { AKRA_F2_ADJ_KBLOCK(GATED, DIFF, 1) }                              \
        else { AKRA_F2_ADJ_KBLOCK(GATED, DIFF, 0) }                                             \
    }
        if (blk_diff) {
            AKRA_F2_ADJ_SIDES(true, true)   // a block with pairs near a pole (rare)
        } else if (all_live) {
            AKRA_F2_ADJ_SIDES(false, false)
        } else {
            AKRA_F2_ADJ_SIDES(true, false)
        }
#undef AKRA_F2_ADJ_SIDES
#undef AKRA_F2_ADJ_KBLOCK
        }
        __syncthreads();
        // sum the warps and write this chunk's partial sums for the tile
        for (int i = tid; i < nl * RG * 4; i += NT) {
            const int step = i / (RG * 4), rem = i - step * RG * 4, rr = rem >> 2, q = rem & 3;
            const int r = r0 + rr;
            if (r >= R) continue;
            float sv = 0.f;
#pragma unroll
            for (int w = 0; w < NW; w++) sv += s_red[w][step][rr][q];
            partial[AKRA_IX((((size_t)chunk * R + r) * ntri + mbase + lt + step) * 4 + q, qbound,
                            kDbgPartialWrite)] = sv * s_sig[step];
        }
    }
}

}  // namespace akra
