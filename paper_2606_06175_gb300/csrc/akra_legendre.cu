// akra_legendre.cu -- spin-2 Legendre stages of the synthesis (Eq. 1) and of its exact
// transpose, fused with the KS factor (Eq. 3) and the E/B <-> spin ±2 recombination (Eq. 2).
//
// Work unit: one m and one ring pair (north ring θ, south ring π-θ; the equator ring alone).
// Two recurrences run in ℓ, one per spin s = ±2 (x = cos θ, A_l, B_l the normalised
// Wigner-d coefficients):
//     sλ_{l+1} = (A_l x + s A_l m/(l(l+1))) sλ_l - A_l B_l sλ_{l-1},
// carried in monic form μ_l = sλ_l / σ_l (σ from the plan's table, between 0.17 and 1), so a
// step is μ_{l+1} = (A'_l x ± c'_l) μ_l - μ_{l-1}: 2 FMA per spin; σ_l is folded into the staged
// alm (synthesis) and into the per-l partial sums (adjoint).
// (kept separate: near the poles one spin is O(1) and the other tiny, and any mixed
// combination would leak the large one's rounding into the small one).  The mirror ring
// follows from  sλ_lm(π-θ) = (-1)^{l+m} (-s)λ_lm(θ), so one pair of recurrences feeds both
// rings through even/odd (l+m) accumulators.  Seeds at l0 = max(m,2) are formed in FP64 in
// log2 form; the recurrence carries a per-unit exponent index e (value = v 2^(Q e)) and
// contributes only once e == 0.
#include <type_traits>

#include "akra_legendre_impl.cuh"

namespace akra {

// ---------------------------------------------------------------------------
// epilogue: sum chunk partials, apply f_l/2 and the spin ±2 -> E/B recombination
//   E = (f/2) E-part,  B = (-i f/2) B-part,  optional + λ x
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_adj_epilogue(int L, long long ntri, int nchunks, int R,
                               const T *__restrict__ partial, const T *__restrict__ fl,
                               const cx_t<T> *__restrict__ xreg, T lam, cx_t<T> *__restrict__ out,
                               const int *__restrict__ skip, int fields)
{
    if (skip && *skip) return;
    using C2 = cx_t<T>;
    const int m = blockIdx.x, r = blockIdx.y;
    const long long mbase = (long long)m * (2 * L + 1 - m) / 2;
    const long long qbound = (long long)nchunks * R * ntri * 4;   // extent of the partial sums
    const long long abound = (long long)R * 2 * ntri;             // extent of x and out
    (void)qbound;
    (void)abound;
    for (int l = m + threadIdx.x; l <= L; l += blockDim.x) {
        const long long idx = mbase + l;
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        if (l >= 2) {
            for (int c = 0; c < nchunks; c++) {
                const long long pq = (((size_t)c * R + r) * ntri + idx) * 4;
                a0 += partial[AKRA_IX(pq + 0, qbound, kDbgPartialRead)];
                a1 += partial[AKRA_IX(pq + 1, qbound, kDbgPartialRead)];
                a2 += partial[AKRA_IX(pq + 2, qbound, kDbgPartialRead)];
                a3 += partial[AKRA_IX(pq + 3, qbound, kDbgPartialRead)];
            }
        }
        const T h = (fl ? fl[AKRA_IX(l, L + 1, kDbgKsFactor)] : T(-1)) * T(0.5);
        C2 E{h * a0, h * a1};
        C2 B{h * a3, -h * a2};
        if (xreg) {
            C2 xe = xreg[AKRA_IX(((size_t)r * 2 + 0) * ntri + idx, abound, kDbgAlm)];
            C2 xb = xreg[AKRA_IX(((size_t)r * 2 + 1) * ntri + idx, abound, kDbgAlm)];
            E.x += lam * xe.x;
            E.y += lam * xe.y;
            B.x += lam * xb.x;
            B.y += lam * xb.y;
        }
        if (m == 0) E.y = B.y = 0;
        // a field outside the solve's field set is held at zero (its block row is dropped)
        if (!(fields & 1)) E = C2{0, 0};
        if (!(fields & 2)) B = C2{0, 0};
        out[AKRA_IX(((size_t)r * 2 + 0) * ntri + idx, abound, kDbgAlmOut)] = E;
        out[AKRA_IX(((size_t)r * 2 + 1) * ntri + idx, abound, kDbgAlmOut)] = B;
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T> const v4_t<T> *coef_ptr(akra_plan p);
template <> const float4 *coef_ptr<float>(akra_plan p) { return p->d_coef32; }
template <> const double4_32a *coef_ptr<double>(akra_plan p) { return p->d_coef64; }
template <typename T> const v4_t<T> *seed_ptr(akra_plan p);
template <> const float4 *seed_ptr<float>(akra_plan p) { return p->d_seed32; }
template <> const double4_32a *seed_ptr<double>(akra_plan p) { return p->d_seed64; }
template <typename T> static const int2 *start_ptr(akra_plan p);
template <> const int2 *start_ptr<float>(akra_plan p) { return p->d_start32; }
template <> const int2 *start_ptr<double>(akra_plan p) { return p->d_start64; }
template <typename T> const T *D_ptr(akra_plan p);
template <> const float *D_ptr<float>(akra_plan p) { return p->d_D32; }
template <> const double *D_ptr<double>(akra_plan p) { return p->d_D64; }

template <typename T>
LegArgs<T> leg_args(akra_plan p, const LegShape &s, LegMode mode, const int *units, int nunits, int R)
{
    LegArgs<T> a{};
    a.L = p->lmax;
    a.nring = p->nring;
    a.nchunks = (nunits + s.NT * s.P - 1) / (s.NT * s.P);
    a.nunits = nunits;
    a.nunit_all = p->nunit;
    a.R = R;
    a.ntri = p->ntri;
    a.units = units;
    a.uinfo = p->d_units;
    a.coef = coef_ptr<T>(p);
    a.seeds = seed_ptr<T>(p);
    a.dseeds = p->d_dseed32;
    a.start = start_ptr<T>(p);
    a.fl = mode == LegMode::KS ? D_ptr<T>(p) : nullptr;
    a.ring_active = units == p->d_all_units ? nullptr : p->d_ring_active;
    a.skip = p->cur_skip;
    a.err = p->d_tc_err;
    a.bpre = (const float *)p->bpre.ptr;
    a.tc_tilebase = p->d_tc_tilebase;
    a.tc_groups = s.TC > 0 ? (R + s.TC - 1) / s.TC : 0;
    a.tc_tiles = p->tc_tiles;
    return a;
}

template <typename T, int P, int RG, int NT>
static void launch_synth(akra_plan p, LegMode mode, const void *alm, void *phi, int R,
                         const int *units, int nunits, cudaStream_t st)
{
    LegArgs<T> a = leg_args<T>(p, LegShape{P, NT, RG}, mode, units, nunits, R);
    a.alm = (const cx_t<T> *)alm;
    a.phi = (cx_t<T> *)phi;
    dim3 grid((unsigned)(p->lmax + 1) * a.nchunks, (R + RG - 1) / RG);
    k_leg_synth<T, P, RG, NT><<<grid, NT, 0, st>>>(a);
}

template <typename T, int P, int RG, int NT, int ONE = 0>
static int launch_adjoint(akra_plan p, const void *phi, void *partial, int R, const int *units,
                          int nunits, cudaStream_t st)
{
    LegArgs<T> a = leg_args<T>(p, LegShape{P, NT, RG}, LegMode::Synth, units, nunits, R);
    a.phi_in = (const cx_t<T> *)phi;
    a.partial = (T *)partial;
    dim3 grid((unsigned)(p->lmax + 1) * a.nchunks, (R + RG - 1) / RG);
    k_leg_adjoint<T, P, RG, NT, ONE><<<grid, NT, 0, st>>>(a);
    return a.nchunks;
}

// shape dispatch: (P, RG) combinations compiled for each precision, NT = 128
template <typename T>
akra_status legendre_synth(akra_plan p, const LegShape &s, LegMode mode, const void *alm,
                           void *phi, int R, const int *units, int nunits, cudaStream_t st)
{
    if (nunits <= 0) return AKRA_OK;
    if constexpr (std::is_same<T, float>::value)
        if (s.TC > 0) return legendre_synth_tc(p, s.TC, mode, alm, phi, R, units, nunits, st);
#define AKRA_S(PP, RR)                                                                      \
    if (s.P == PP && s.RG == RR) {                                                          \
        launch_synth<T, PP, RR, 128>(p, mode, alm, phi, R, units, nunits, st);              \
        AKRA_CUDA_TRY(cudaGetLastError());                                                  \
        p->launches++;                                                                      \
        return AKRA_OK;                                                                     \
    }
    AKRA_S(1, 1) AKRA_S(2, 1) AKRA_S(4, 1) AKRA_S(1, 2) AKRA_S(2, 2) AKRA_S(1, 4)
    if constexpr (std::is_same<T, float>::value) { AKRA_S(3, 1) AKRA_S(5, 1) AKRA_S(6, 1) AKRA_S(8, 1) }
#undef AKRA_S
    set_error("no synthesis kernel for P=%d RG=%d", s.P, s.RG);
    return AKRA_EINVAL;
}

template <typename T>
akra_status legendre_adjoint(akra_plan p, const LegShape &s, const void *phi, void *partial,
                             int R, const int *units, int nunits, int *nchunks_out,
                             cudaStream_t st)
{
    *nchunks_out = 0;
    if (nunits <= 0) return AKRA_OK;
    const int pa = s.adjP();
    {
        // the active ring pairs of a one-hemisphere footprint all need the same single ring: the
        // kernel compiled for that form alone (fewer registers); FP32 at 3-8 ring pairs per
        // thread, FP64 at 1, 2 and 4, one RHS per block
        const int one = (units != p->d_all_units && s.adjRG() == 1) ? p->one_side : 0;
#define AKRA_A1(PP)                                                                          \
        if (one && pa == PP) {                                                               \
            *nchunks_out = one == 1 ? launch_adjoint<T, PP, 1, 128, 1>(p, phi, partial, R, units, nunits, st) \
                                    : launch_adjoint<T, PP, 1, 128, 2>(p, phi, partial, R, units, nunits, st); \
            AKRA_CUDA_TRY(cudaGetLastError());                                               \
            p->launches++;                                                                   \
            return AKRA_OK;                                                                  \
        }
        if constexpr (std::is_same<T, float>::value) { AKRA_A1(3) AKRA_A1(4) AKRA_A1(5) AKRA_A1(6) AKRA_A1(8) }
        else { AKRA_A1(1) AKRA_A1(2) AKRA_A1(4) }
#undef AKRA_A1
    }
#define AKRA_A(PP, RR)                                                                      \
    if (pa == PP && s.adjRG() == RR) {                                                      \
        *nchunks_out = launch_adjoint<T, PP, RR, 128>(p, phi, partial, R, units, nunits, st); \
        AKRA_CUDA_TRY(cudaGetLastError());                                                  \
        p->launches++;                                                                      \
        return AKRA_OK;                                                                     \
    }
    AKRA_A(1, 1) AKRA_A(2, 1) AKRA_A(4, 1) AKRA_A(1, 2) AKRA_A(2, 2) AKRA_A(1, 4)
    if constexpr (std::is_same<T, float>::value) { AKRA_A(3, 1) AKRA_A(5, 1) AKRA_A(6, 1) AKRA_A(8, 1) }
#undef AKRA_A
    set_error("no adjoint kernel for P=%d RG=%d", pa, s.adjRG());
    return AKRA_EINVAL;
}

template <typename T>
akra_status adjoint_epilogue(akra_plan p, LegMode mode, const void *partial, int nchunks,
                             const void *x_reg, double lam, void *alm_out, int R, cudaStream_t st,
                             int fields)
{
    dim3 grid(p->lmax + 1, R);
    k_adj_epilogue<T><<<grid, 128, 0, st>>>(p->lmax, p->ntri, nchunks, R, (const T *)partial,
                                            mode == LegMode::KS ? D_ptr<T>(p) : nullptr,
                                            (const cx_t<T> *)x_reg, (T)lam, (cx_t<T> *)alm_out,
                                            p->cur_skip, fields);
    AKRA_CUDA_TRY(cudaGetLastError());
    p->launches++;
    return AKRA_OK;
}

// chunks of the adjoint (its partial sums are laid out per chunk)
int legendre_chunks(int nunits, const LegShape &s)
{
    const int per = s.NT * s.adjP();
    return (nunits + per - 1) / per;
}

template LegArgs<float> leg_args<float>(akra_plan, const LegShape &, LegMode, const int *, int, int);
template LegArgs<double> leg_args<double>(akra_plan, const LegShape &, LegMode, const int *, int, int);
template akra_status legendre_synth<float>(akra_plan, const LegShape &, LegMode, const void *, void *,
                                           int, const int *, int, cudaStream_t);
template akra_status legendre_synth<double>(akra_plan, const LegShape &, LegMode, const void *,
                                            void *, int, const int *, int, cudaStream_t);
template akra_status legendre_adjoint<float>(akra_plan, const LegShape &, const void *, void *, int,
                                             const int *, int, int *, cudaStream_t);
template akra_status legendre_adjoint<double>(akra_plan, const LegShape &, const void *, void *, int,
                                              const int *, int, int *, cudaStream_t);
template akra_status adjoint_epilogue<float>(akra_plan, LegMode, const void *, int, const void *,
                                             double, void *, int, cudaStream_t, int);
template akra_status adjoint_epilogue<double>(akra_plan, LegMode, const void *, int, const void *,
                                              double, void *, int, cudaStream_t, int);

AKRA_DEBUG_COLLECTOR(legendre)

}  // namespace akra
