// akra_internal.cuh -- internal declarations of the sm_103a AKRA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "../../include/akra.h"

namespace akra {

// ---------------------------------------------------------------------------
// error handling: every failure becomes an akra_status plus a thread-local message
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);

#define AKRA_CUDA_TRY(expr)                                                              \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) {                                                         \
            akra::set_error("%s:%d: %s failed: %s", __FILE__, __LINE__, #expr,           \
                            cudaGetErrorString(_e));                                     \
            return AKRA_ECUDA;                                                           \
        }                                                                                \
    } while (0)

#define AKRA_TRY(expr)                                                                   \
    do {                                                                                 \
        akra_status _s = (expr);                                                         \
        if (_s != AKRA_OK) return _s;                                                    \
    } while (0)

// ---------------------------------------------------------------------------
// bounds-checked build (-DAKRA_DEBUG, built as libakra_debug.so): the index of every
// global-memory access of the operator kernels (Legendre items, epilogue, ring FFTs) is checked
// against its array's extent.  An index outside [0, bound) is replaced by 0, so no access
// leaves its array, and the first violation (call site, index, bound) is recorded in a device
// record of the translation unit; akra_debug_violations() collects and clears the records.
// No kernel traps: the call's results are wrong and the host is told.  The release build
// compiles the plain index.
// ---------------------------------------------------------------------------
struct DebugRecord {
    unsigned long long count;   // out-of-bounds accesses seen
    long long index, bound;     // the first one
    int site;                   // its call site (DebugSite)
    int pad;
};
enum DebugSite {
    kDbgUnits = 1, kDbgUnitInfo, kDbgStart, kDbgSeeds, kDbgCoef, kDbgAlm, kDbgKsFactor,
    kDbgPhiWrite, kDbgPhiRead, kDbgPartialWrite, kDbgPartialRead, kDbgAlmOut, kDbgRingActive,
    kDbgFftPhi, kDbgFftMapIn, kDbgFftMapOut, kDbgFftWeight, kDbgFftRing, kDbgBpre
};
#ifdef AKRA_DEBUG
static __device__ DebugRecord g_akra_dbg;   // one per translation unit
__device__ __forceinline__ long long dbg_index(long long i, long long bound, int site)
{
    if (i >= 0 && i < bound) return i;
    if (atomicAdd(&g_akra_dbg.count, 1ull) == 0ull) {
        g_akra_dbg.index = i;
        g_akra_dbg.bound = bound;
        g_akra_dbg.site = site;
    }
    return 0;
}
#define AKRA_IX(i, bound, site) ::akra::dbg_index((long long)(i), (long long)(bound), (site))
#define AKRA_DEBUG_COLLECTOR(tu)                                                           \
    akra_status debug_collect_##tu(DebugRecord *acc)                                       \
    {                                                                                      \
        DebugRecord r{}, zero{};                                                           \
        AKRA_CUDA_TRY(cudaMemcpyFromSymbol(&r, g_akra_dbg, sizeof(r)));                    \
        AKRA_CUDA_TRY(cudaMemcpyToSymbol(g_akra_dbg, &zero, sizeof(zero)));                \
        if (r.count && !acc->count) {                                                      \
            acc->index = r.index;                                                          \
            acc->bound = r.bound;                                                          \
            acc->site = r.site;                                                            \
        }                                                                                  \
        acc->count += r.count;                                                             \
        return AKRA_OK;                                                                    \
    }
#else
#define AKRA_IX(i, bound, site) (i)
#define AKRA_DEBUG_COLLECTOR(tu) \
    akra_status debug_collect_##tu(DebugRecord *) { return AKRA_OK; }
#endif
akra_status debug_collect_legendre(DebugRecord *acc);
akra_status debug_collect_legendre_tc(DebugRecord *acc);
akra_status debug_collect_batch(DebugRecord *acc);
akra_status debug_collect_ringfft(DebugRecord *acc);
akra_status debug_collect_ringfft32(DebugRecord *acc);

// ---------------------------------------------------------------------------
// small vector types
// ---------------------------------------------------------------------------
template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };
template <typename T> using cx_t = typename Cx<T>::type;

template <typename T> struct V4t;
template <> struct V4t<float> { using type = float4; };
template <> struct V4t<double> { using type = double4_32a; };
template <typename T> using v4_t = typename V4t<T>::type;

// scaled-recurrence parameters: a value v with exponent index e < 0 stands for
// v * 2^(Q e); a rescale by 2^-Q happens when |v| > 2^(Q/2); contributions start when e == 0
// recurrences start at grid points l0 + kStartGrid j (a multiple of every l-tile width)
constexpr int kStartGrid = 64;
// FP32 ring pairs within 0.1 rad of a pole (x = cos θ >= kDiffX) run the recurrence in difference
// form: with d_l = μ_l - μ_{l-1} and u_l = t_l - 2 = A'_l (x - 1) + (A'_l - 2) ± c'_l (all three
// pieces small and each accurate to FP32 rounding),
//     d_{l+1} = u_l μ_l + d_l,   μ_{l+1} = μ_l + d_{l+1}.
// Near x = 1 the standard step rounds t_l ~ 2 to an absolute 2^-23 while the recurrence turns
// by an angle ~θ per step, so each step's phase error is ~2^-23/θ and grows over the l-range (up
// to ~1e-1 relative at θ ~ 1e-3, l ~ 4000); the difference form carries the small quantities
// themselves (measured in FP32 emulation: ~1e-6 at every θ < 0.1).  Away from the poles it has
// no advantage and costs one more operation per step, so the other pairs keep the standard form.
constexpr double kDiffX = 0.99500416527802582;   // cos(0.1)
constexpr int kNeverLive = 0x7fffffff;   // start index of a pair whose harmonics stay negligible

template <typename T> struct Scale;
template <> struct Scale<float> {
    static constexpr int Q = 64;
    __host__ __device__ static constexpr float hi() { return 4294967296.0f; }                  // 2^32
    __host__ __device__ static constexpr float inv() { return 5.421010862427522e-20f; }        // 2^-64
};
template <> struct Scale<double> {
    static constexpr int Q = 600;
    __host__ __device__ static constexpr double hi() { return 0x1p300; }
    __host__ __device__ static constexpr double inv() { return 0x1p-600; }
};

// ---------------------------------------------------------------------------
// plan tables
// ---------------------------------------------------------------------------
struct RingInfo {          // one HEALPix ring (row r = ring index - 1)
    double z, st;          // cos θ, sin θ
    long long first;       // first pixel (RING order)
    long long tw_off;      // offset of this ring length's table of e^{iπ t/n}, t in [0, 2n)
    int nphi;              // pixels on the ring, n
    int sigma;             // pixel phases φ_j = π(2j + σ)/n
    int ilen;              // n = 4 * ilen (index into the FFT factor table)
    int pad;
};

struct UnitInfo {          // one north/south ring pair (or the equator ring alone)
    double x;              // cos θ of the north ring (>= 0)
    double ls, lc;         // log2 sin(θ/2), log2 cos(θ/2) of the north ring
    int ring_n, ring_s;    // rows of the two rings; ring_s = -1 for the equator
};

constexpr int kMaxFactors = 16;
// FP64 ring FFT: a prime factor >= kBluePrime is transformed by Bluestein's chirp-z form (a
// convolution of power-of-two length, O(p log p)) instead of a direct O(p^2) pass
constexpr int kBluePrime = 67;
struct FftFactors {
    int nf;
    int f[kMaxFactors];    // mixed-radix passes: odd primes below kBluePrime, then 4s and a 2
    int blue_p;            // a prime factor >= kBluePrime, transformed last by Bluestein (0: none)
    int blue_M;            // its convolution length (a power of two >= 2 blue_p - 1)
    long long blue_off;    // its tables in d_blue64: chirp h[p], then G+[M], G-[M]
};

constexpr int kMaxNside = 2048;

// Legendre tile shape (chosen per precision and RHS count; see autotune)
struct LegShape {
    int P;                 // ring pairs per thread (synthesis)
    int NT;                // threads per block
    int RG;                // RHS handled together by one block
    int PA = 0;            // ring pairs per thread of the adjoint (0: same as P)
    int TC = 0;            // FP32 synthesis on the tensor core with RHS groups of TC (4, 8, 16,
                           // 32); 0: CUDA-core synthesis of shape (P, RG)
    int RGA = 0;           // RHS per block of the adjoint (0: same as RG)
    int adjP() const { return PA > 0 ? PA : P; }
    int adjRG() const { return RGA > 0 ? RGA : RG; }
};

// arguments of one Legendre kernel instance (one plan; the batched launches hold an array)
template <typename T>
struct LegArgs {
    int L, nring, nchunks, nunits, nunit_all, R;
    long long ntri;
    const int *units;                 // ring pairs to process
    const UnitInfo *uinfo;
    const v4_t<T> *coef;              // recurrence coefficients
    const v4_t<T> *seeds;             // start states per (m, ring pair)
    const float2 *dseeds;             // FP32: start differences (μ_g - μ_{g-1}) per (m, ring pair)
    const int2 *start;                // their grid points and exponent indices
    const T *fl;                      // synthesis: per-l factor (nullptr = -1)
    const cx_t<T> *alm;               // synthesis input  [R][2][ntri]
    cx_t<T> *phi;                     // synthesis output [R][nring][2L+1]
    const cx_t<T> *phi_in;            // adjoint input    [R][nring][2L+1]
    T *partial;                       // adjoint output   [nchunks][R][ntri][4]
    const unsigned char *ring_active; // nullptr = all rings
    const int *skip;                  // device flag: return at once if set
    int *err;                         // device flag set when a bounded in-kernel wait runs out
    // tensor-core synthesis: the B operand pre-staged per (m, 16-step tile, RHS group) in the
    // tile layout of shared memory (legendre_tc_bstage), the first tile index of each m, and the
    // number of RHS groups
    const float *bpre;
    const long long *tc_tilebase;
    int tc_groups;
    long long tc_tiles;
};

// arguments of one FP32 ring-FFT instance
struct Fft32Args {
    int L, nring, mmax;
    long long npix;
    const int *rings;                 // ring list (nullptr = all rings by block index)
    const RingInfo *rinfo;
    const int *fftM;
    const long long *bhat_off;
    const float2 *bhat_all;
    const float2 *tw2;
    const float2 *tw_all;
    const float *W;          // FP32 W in the FFT's pixel order (bit-reversed in power-of-two rings)
    int weighted;
    float2 *phi;
    const float *map_in;
    float *map_out;
    const int *skip;
};

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

struct CgGraph;            // CUDA-graph state of one CG configuration (akra_cg.cu)

}  // namespace akra

struct akra_plan_s {
    // 0: HEALPix sphere (spin-2 SHTs); 1: flat-sky n x n periodic patch (2D FFTs), where
    // nside holds n, lmax is -1 (no m = 0 entries in the CG metric), npix = n^2, ntri = n^2/2
    int kind = 0;
    int nside = 0, lmax = 0, nring = 0, nunit = 0;
    long long npix = 0, ntri = 0;
    int device = 0;

    // geometry and recurrence tables (device)
    akra::RingInfo *d_rings = nullptr;
    akra::UnitInfo *d_units = nullptr;
    akra::FftFactors *d_factors = nullptr;   // [nside + 1] by ring length index
    double2 *d_blue64 = nullptr;             // FP64 Bluestein tables of the primes >= kBluePrime
    double4_32a *d_coef64 = nullptr;            // [ntri] {A, A B, A 2m/(l(l+1)), 0}
    float4 *d_coef32 = nullptr;
    double *d_seedC = nullptr;               // [lmax + 1] log2 seed prefactor per m
    // start states of the recurrences per (m, ring pair), computed in FP64 at plan time:
    // {μ+_g, μ-_g, μ+_{g-1}, μ-_{g-1}} at the grid point g (l0 + 64 j) where the pair's
    // harmonics first exceed the precision's threshold, scaled by 2^(-Q e)
    float4 *d_seed32 = nullptr;              // [(lmax+1) nunit]
    float2 *d_dseed32 = nullptr;             // [(lmax+1) nunit] {μ+_g - μ+_{g-1}, μ-_g - μ-_{g-1}}, scaled as
                                             // d_seed32 (start of the FP32 difference form)
    double4_32a *d_seed64 = nullptr;         // [(lmax+1) nunit]
    int2 *d_start32 = nullptr;               // [(lmax+1) nunit] {g (kNeverLive: none), e}
    int2 *d_start64 = nullptr;
    unsigned long long *d_steps = nullptr;   // [2 nunit] Σ_m (lmax + 1 - g) per ring pair, FP32 / FP64
    std::vector<unsigned long long> steps32, steps64;   // host copies
    std::vector<int> h_active_units;         // host copy of the active pairs
    std::vector<unsigned char> h_unit_one_ring;   // per active unit: needs one ring only
    double *d_D64 = nullptr;                 // [lmax + 1] KS kernel D_l
    float *d_D32 = nullptr;
    double2 *d_tw64 = nullptr;               // ring twiddles e^{iπ t/n}
    float2 *d_tw32 = nullptr;
    int fft32_mmax = 0;                      // FP32 ring FFT: largest convolution length
    int *d_fft32_M = nullptr;                // [nside + 1] per ring length index: M (== n if 2^k)
    long long *d_fft32_off = nullptr;        // [nside + 1] offset of the chirp spectrum
    float2 *d_fft32_tw2 = nullptr;           // e^{-2πi t/MMAX}
    float2 *d_fft32_bhat = nullptr;          // chirp spectra (DIF output order)
    std::vector<int> fft32_M_host;           // [nside + 1] host copy of d_fft32_M
    int fft32_msmall = 0;                    // largest M below fft32_mmax (0: a single class)
    int *d_fft32_rings_all = nullptr;        // [nring] all rings, those with M <= msmall first
    int fft32_nsmall_all = 0;
    int *d_fft32_rings_act = nullptr;        // [nring] active rings in the same order
    int fft32_nsmall_act = 0;
    int *d_all_rings = nullptr;              // [nring] 0..nring-1
    int *d_all_units = nullptr;              // [nunit] 0..nunit-1

    // flat-sky plan: twiddles e^{-2πi t/n}, weights W = M N^-1 transposed and scaled by 1/n^2
    int flat_logn = 0;
    double2 *d_ftw64 = nullptr;
    float2 *d_ftw32 = nullptr;
    double *d_fWt64 = nullptr;
    float *d_fWt32 = nullptr;

    // fields H acts on inside a field-restricted solve (bit 0 E, bit 1 B); 3 everywhere else
    int fields = 3;

    // preconditioner: 0 = the scalar P of Eq. 15, 1 = the per-l diagonal
    // (mean_all(M N^-1) D_l^2 + λ_eff)^-1, as weights per packed index in d_pw64 / d_pw32
    int precond_kind = 0;
    double *d_pw64 = nullptr;
    float *d_pw32 = nullptr;

    // weights
    bool has_weights = false;
    double lambda = 0, lambda_eff = 0, precond = 1, omega = 0;
    double *d_W64 = nullptr;                 // [npix] ω M N^-1
    float *d_W32 = nullptr;
    float *d_W32r = nullptr;                 // [npix] W in the FP32 ring FFT's pixel order
                                             // (bit-reversed within power-of-two rings)
    int *d_active_rings = nullptr;           // rings with any W != 0
    int n_active_rings = 0;
    int *d_active_units = nullptr;           // units with an active ring
    int n_active_units = 0;
    int one_side = 0;                        // every active unit needs only its north (1) / south (2) ring
    unsigned char *d_ring_active = nullptr;  // [nring] flag

    // workspaces (grown on demand)
    akra::Workspace phi, partial, cg, red;
    akra::Workspace xsave;                   // κ_E kept aside by the conditional B-mode solve
    akra::Workspace red_cl;                  // per-l spectra before binning into band powers
    akra::Workspace bpre;                    // tensor-core synthesis: pre-staged B operand tiles
    long long tc_tiles = 0;                  // 16-step l-tiles over all m (from l0(m) to lmax)
    long long *d_tc_tilebase = nullptr;      // [lmax+1] first tile index of each m
    cudaStream_t stream = nullptr;           // internal stream for captured CG graphs
    cudaEvent_t ev_a = nullptr, ev_b = nullptr;
    std::map<long long, akra::LegShape> shapes;   // key: prec*1000 + R
    std::map<long long, akra::CgGraph *> graphs;
    unsigned ws_gen = 0;                     // bumped whenever a workspace is reallocated
    const int *cur_skip = nullptr;           // device flag: operator kernels return early if set
    int *d_tc_err = nullptr;                 // device flag: a bounded wait inside a Legendre kernel ran out
    void *h_pinned = nullptr;                // pinned host mirror for status polling
    size_t bytes_tables = 0;
    long long launches = 0;                  // kernels launched (host-side count)
};

namespace akra {

// workspace growth (device); returns ENOMEM on failure
akra_status ws_reserve(akra_plan p, Workspace &w, size_t bytes);
size_t plan_device_bytes(akra_plan p);

// the operator pieces (all asynchronous on `st`)
enum class LegMode { Synth, KS };   // per-l factor f_l = -1 (pure spin-2 SHT) or D_l (KS)

// FP32 synthesis with the tensor-core contraction (akra_legendre_tc.cu), RHS in groups of tcg
akra_status legendre_synth_tc(akra_plan p, int tcg, LegMode mode, const void *alm, void *phi, int R,
                              const int *units, int nunits, cudaStream_t st);
constexpr int TC_NT = 128;   // tensor-core synthesis: threads = ring pairs per block = MMA rows
akra_status legendre_tc_prepare();
// bytes of the pre-staged B operand for R RHS in groups of tcg, and its reservation (a no-op when
// large enough; call before any stream capture that may run the tensor-core synthesis)
size_t tc_bpre_bytes(akra_plan p, int tcg, int R);
akra_status tc_reserve(akra_plan p, int tcg, int R);
// write the B operand tiles of x (one plan's [R][2][ntri] alm) for RHS groups of tcg
akra_status legendre_tc_bstage(int tcg, const LegArgs<float> &a, cudaStream_t st);
// persistent tensor-core synthesis over a work list of (instance, m, 128-pair chunk, RHS group)
akra_status legendre_synth_tc_queue(int tcg, const LegArgs<float> *insts, const int4 *items, int nitems,
                                    int *counter, cudaStream_t st);
// reads and clears the plan's kernel-wait error flag (blocking): ECUDA if a bounded wait ran out
akra_status tc_error_check(akra_plan p);


LegShape leg_shape(akra_plan p, akra_prec prec, int R);
int legendre_chunks(int nunits, const LegShape &s);
void cg_release_graphs(akra_plan p);   // akra_cg.cu
akra_status metric_inverse(akra_plan p, bool dbl, const void *in, void *out, int R, cudaStream_t st);

// the LegArgs of plan p for precision T (pointers for data are filled by the caller)
template <typename T>
LegArgs<T> leg_args(akra_plan p, const LegShape &s, LegMode mode, const int *units, int nunits, int R);

// alm [R][2][ntri] -> Φ [R][nring][2L+1] on the listed units
template <typename T>
akra_status legendre_synth(akra_plan p, const LegShape &s, LegMode mode, const void *alm, void *phi,
                           int R, const int *units, int nunits, cudaStream_t st);
// Φ' [R][nring][2L+1] -> partial sums [chunks][R][ntri] (vec4) on the listed units
template <typename T>
akra_status legendre_adjoint(akra_plan p, const LegShape &s, const void *phi, void *partial,
                             int R, const int *units, int nunits, int *nchunks_out,
                             cudaStream_t st);
// partial sums -> alm (with f_l/2, E/B recombination and optional + λ x); fields: bit 0 E,
// bit 1 B -- a field outside the set is written as zero
template <typename T>
akra_status adjoint_epilogue(akra_plan p, LegMode mode, const void *partial, int nchunks,
                             const void *x_reg, double lam, void *alm_out, int R, cudaStream_t st,
                             int fields = 3);

enum class FftMode { Synth = 0, Adjoint = 1, Happly = 2 };
template <typename T>
akra_status ring_fft(akra_plan p, FftMode mode, void *phi, const void *map_in, void *map_out,
                     bool weighted, int R, const int *rings, int nrings, cudaStream_t st);
// FP32 ring FFT with Bluestein for non-power-of-two rings (akra_ringfft32.cu)
akra_status ring_fft32_build(akra_plan p);
// flat-sky operators (akra_flat.cu); the op_* entry points dispatch to them for kind == 1
template <typename T>
akra_status flat_op_A(akra_plan p, const void *x, void *map, bool weighted, int R, cudaStream_t st);
template <typename T>
akra_status flat_op_At(akra_plan p, const void *map, void *x, bool weighted, int R, cudaStream_t st);
template <typename T>
akra_status flat_op_H(akra_plan p, const void *x, void *y, int R, cudaStream_t st);
akra_status flat_set_weights(akra_plan p, const double *d_ninv, double lambda, cudaStream_t st);
inline bool is_flat(akra_plan p) { return p && p->kind == 1; }
// entry points that need the sphere's spin-2 SHT machinery reject flat-sky plans
inline akra_status reject_flat(akra_plan p, const char *who)
{
    if (!is_flat(p)) return AKRA_OK;
    set_error("%s: not defined for a flat-sky plan", who);
    return AKRA_EINVAL;
}
akra_status ring_fft32_order(akra_plan p, const std::vector<int> &rings, int *d_out, int *nsmall);
Fft32Args fft32_args(akra_plan p, bool weighted, const int *rings);
akra_status ring_fft32(akra_plan p, FftMode mode, void *phi, const void *map_in, void *map_out,
                       bool weighted, int R, const int *rings, int nrings, cudaStream_t st);

// whole operators
template <typename T>
akra_status op_synth(akra_plan p, LegMode mode, const void *alm, void *map, bool weighted, int R,
                     cudaStream_t st);
template <typename T>
akra_status op_adjoint(akra_plan p, LegMode mode, const void *map, void *alm, bool weighted, int R,
                       cudaStream_t st);
template <typename T>
akra_status op_H(akra_plan p, const void *x, void *y, int R, cudaStream_t st);

}  // namespace akra
