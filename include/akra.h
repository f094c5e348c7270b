/*
 * akra.h -- C ABI of the GB300 (sm_103a) implementation of the AKRA 3.0 hot path:
 * the matrix-free normal-equation operator  H = A^T N^{-1} A  (+ λ_eff I) and the
 * (preconditioned) conjugate-gradient solve built on it.
 *
 *   A  : E/B convergence harmonics --KS kernel D_l (Eq. 3)--> spin-2 harmonics
 *        (Eq. 2) --spin-2 synthesis (Eq. 1)--> shear (γ1, γ2) on HEALPix pixels
 *   N^-1: per-pixel inverse noise variance, zero off the mask (Eq. 4, Eqs. 17-19)
 *   A^T: the exact transpose of A (Sec. II B, "the adjoint reverses this sequence")
 *   CG : Sec. II B "The inversion problem"; regulariser λ_eff I (Eq. 14);
 *        scalar preconditioner P = (<M^2 N^-1> + λ_eff)^{-1} I (Eq. 15).
 *
 * Conventions (shared by every entry point)
 *   - nside: HEALPix resolution (1 <= nside <= 2048); npix = 12 nside^2; pixels in
 *     RING order.  lmax: band limit, 2 <= lmax <= 4 nside.
 *   - harmonic vectors ("alm"): [R][2][ntri] complex, ntri = (lmax+1)(lmax+2)/2,
 *     index [r][field][m(2 lmax + 1 - m)/2 + l] for 0 <= m <= l <= lmax, field 0 = E,
 *     1 = B; complex = interleaved (re, im).  The fields are real on the sphere
 *     (x_{l,-m} = (-1)^m conj x_lm), so only m >= 0 is stored; Im(x_{l0}) is ignored on
 *     input and written as 0 on output.  Harmonic inner products count every real
 *     degree of freedom: <x,y> = Σ_l [x_l0 y_l0 + 2 Re Σ_{m>0} x_lm conj(y_lm)].
 *   - maps: [R][2][npix] real, component 0 = γ1, 1 = γ2.
 *   - precision: AKRA_F64 -> double / complex double; AKRA_F32 -> float /
 *     complex float; AKRA_MIXED (cg_solve only) -> FP64 inputs and outputs, FP32 inner
 *     iterations, FP64 outer residual.
 *   - all array arguments named d_* are DEVICE pointers owned by the caller, 256-byte
 *     aligned as returned by cudaMalloc (or a torch CUDA tensor), contiguous.
 *   - stream: a cudaStream_t passed as void* (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream unless stated otherwise.
 *   - errors are returned as akra_status, never by exception or abort;
 *     akra_last_error() returns a thread-local message for the last failure.
 *   - a plan is not thread-safe: calls on one plan must be serialised by the caller.
 */
#ifndef AKRA_H
#define AKRA_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct akra_plan_s *akra_plan;

typedef enum {
    AKRA_OK = 0,
    AKRA_EINVAL = 1,     /* bad argument (sizes, null pointer, precision) */
    AKRA_ENOMEM = 2,     /* device or host allocation failed */
    AKRA_ECUDA = 3,      /* a CUDA runtime call failed */
    AKRA_ENOCONV = 4,    /* CG reached maxiter before the tolerance */
    AKRA_ENUMERIC = 5,   /* NaN/Inf or a non-positive curvature <p,Hp> in CG */
    AKRA_ETIMEOUT = 6,   /* the host-side wall-clock budget of a blocking call ran out */
    AKRA_ENOWEIGHTS = 7  /* an operator needing N^-1 was called before set_weights */
} akra_status;

typedef enum { AKRA_F64 = 0, AKRA_F32 = 1, AKRA_MIXED = 2 } akra_prec;

/* Result of a CG solve (host struct, filled by akra_cg_solve / akra_cg_solve_b). */
typedef struct {
    int iters;            /* CG iterations (AKRA_MIXED: all inner FP32 iterations) */
    int outer;            /* AKRA_MIXED: outer refinement steps; 0 otherwise */
    int h_applies_f64;    /* FP64 operator applications (H, and the A^T of b) */
    int h_applies_f32;    /* FP32 operator applications */
    double relres;        /* max over RHS of the final relative residual ||b - H x|| / ||b||:
                             F64/MIXED: recomputed in FP64 at exit; F32: recursive */
    int status;           /* worst akra_status over the RHS */
    double *relres_rhs;   /* optional caller-owned host array [R] (may be NULL) */
    int *iters_rhs;       /* optional caller-owned host array [R] (may be NULL) */
} akra_cg_info;

/* Read-only description of a plan. */
typedef struct {
    int nside, lmax, nring, nunit;    /* nunit = 2 nside ring pairs (north/south + equator) */
    long long npix, ntri;
    int has_weights;
    int n_active_rings;               /* rings with any N^-1 > 0 */
    int n_active_units;               /* ring pairs with an active ring (the units H transforms) */
    double lambda, lambda_eff;        /* λ and λ_eff = λ <N^-1>_M  (Eq. 14) */
    double precond;                   /* scalar P of Eq. 15 */
    double omega;                     /* pixel area 4π/npix folded into W = ω M N^-1 */
    size_t device_bytes;              /* device memory currently held by the plan */
    long long kernel_launches;        /* kernels this plan has launched so far (host count;
                                         a captured CG iteration counts its 7-8 kernels) */
    long long legendre_steps_f32;     /* (l, m, ring pair) steps of one FP32 Legendre pass over
                                         the pairs H transforms, per RHS: each pair's recurrence
                                         starts where its harmonics exceed 2^-40 (Sec. II B
                                         recurrences; the terms below are negligible) */
    long long legendre_steps_f64;     /* the same for FP64 (threshold 2^-90) */
    long long legendre_steps_f32_one_ring;  /* the part of legendre_steps_f32 over pairs that need
                                               one ring only (one-ring contraction, half the FMAs) */
    long long legendre_steps_f64_one_ring;  /* the same for FP64 */
} akra_plan_desc;

/* Create a plan for (nside, lmax): HEALPix ring tables, spin-2 recurrence tables, ring
 * FFT twiddles (all on the current device).  *out receives an opaque handle owned by
 * the library; free it with akra_plan_destroy.  Blocking.
 * Errors: EINVAL for nside outside [1,2048], lmax outside [2, 4 nside] or out == NULL;
 * ENOMEM; ECUDA. */
akra_status akra_plan_create(int nside, int lmax, akra_plan *out);

/* Flat-sky variant (Sec. II B: each SHT replaced by a 2D FFT, the operator's four steps and
 * the CG solver unchanged).  Creates a plan for an n x n periodic pixel grid, n a power of two
 * in [16, 8192].  On such a plan the unknown x [R][n][n] complex is the unitary 2D Fourier
 * transform of κ_E + i κ_B (rows k2, columns k1, FFT frequency order); maps are [R][2][n*n]
 * (γ1, γ2; pixel (row y, column x) at y*n + x).  A x = F^-1(D x) with the flat-sky
 * Kaiser-Squires kernel D(k) = (k1² - k2² + 2i k1 k2)/|k|² (D(0) = 0), A^T its exact adjoint,
 * W = M N^-1 (no pixel-area factor; the unitary transforms carry the normalisation), λ_eff and
 * the scalar P as for the sphere (Eqs. 14-15).  akra_plan_set_weights (d_ninv [n*n]),
 * akra_apply_A / At / H, akra_cg_solve(_b) in F64, F32 and MIXED, akra_shuffle_shear,
 * akra_plan_describe and akra_plan_destroy accept the plan; the other entry points (the
 * sphere's spin-2 SHTs, tile shapes, batches, field-restricted solves, spectra and the
 * autograd pair) return EINVAL for it.  Errors: EINVAL (n), ENOMEM, ECUDA. */
akra_status akra_flat_plan_create(int n, akra_plan *out);

/* Release every device and host resource of the plan (NULL is ignored).  Blocking. */
void akra_plan_destroy(akra_plan plan);

/* Thread-local description of the last error on this thread ("" if none). */
const char *akra_last_error(void);

/* Library version string. */
const char *akra_version(void);

/* Fill *out with the plan's sizes and weight statistics.  Blocking. */
akra_status akra_plan_describe(akra_plan plan, akra_plan_desc *out);

/* Bounds-check record of the debug build (libakra_debug.so, compiled with -DAKRA_DEBUG; the
 * paper has no counterpart).  In that build the index of every global-memory access of the
 * operator kernels (Legendre synthesis and adjoint, epilogue, ring FFTs) is checked against its
 * array's extent; an index outside it is replaced by 0 (no access leaves its array, no kernel
 * traps) and counted.  This call synchronises the device, returns the number of violations
 * since the last call in *count, with the call site, index and extent of the first one, and
 * clears the record.  In the release build *count = -1 (no checks compiled in).  site, index
 * and bound may be NULL.  Errors: EINVAL (count NULL), ECUDA. */
akra_status akra_debug_violations(long long *count, int *site, long long *index, long long *bound);

/* Testing aid (a substitute for a memory checker; the paper has no counterpart): set every
 * byte of every device workspace the plan currently holds -- phase array, adjoint partial
 * sums, CG vectors and reduction scratch, field and spectra scratch -- to `byte`.  With 0xFF
 * each FP32 and FP64 entry becomes a NaN, so an operator or solve that reads a workspace entry
 * it did not write first returns non-finite results.  Workspaces keep their addresses, so
 * captured CG graphs stay valid.  Asynchronous on `stream`.  Errors: EINVAL (NULL plan, byte
 * outside [0, 255]), ECUDA. */
akra_status akra_plan_fill_workspaces(akra_plan plan, int byte, void *stream);

/* Set the pixel weights from d_ninv [npix] (double, N^-1_p >= 0, 0 off the mask; the mask
 * is M_p = [N^-1_p > 0]).  Stores W_p = ω M_p N^-1_p (ω = 4π/npix) in FP64 and FP32,
 * λ_eff = lambda · mean_{M}(N^-1) (Eq. 14) and P = 1/(mean_all(M N^-1) + λ_eff) (Eq. 15),
 * and the list of rings with any nonzero weight (the only rings H needs).  An all-zero d_ninv
 * (empty footprint) is accepted: no ring is active, λ_eff = 0, H = 0 and solves return x = 0.
 * Blocking (reads the statistics back).  Errors: EINVAL (NULL, lambda < 0, negative or
 * non-finite N^-1), ECUDA. */
akra_status akra_plan_set_weights(akra_plan plan, const double *d_ninv, double lambda,
                                  void *stream);

/* Spin-2 synthesis (Eqs. 1-2): γ1 + iγ2 = Σ_{l>=2} Σ_m γ_{2,lm} 2Y_lm with
 * γ_{2,lm} = -(a_E,lm + i a_B,lm).  d_alm [R][2][ntri] (E, B) -> d_map [R][2][npix].
 * prec: F64 or F32.  Errors: EINVAL, ENOMEM (workspace), ECUDA. */
akra_status akra_synth_spin2(akra_plan plan, akra_prec prec, const void *d_alm, void *d_map,
                             int R, void *stream);

/* akra_synth_spin2 without any device allocation.  The paper has no counterpart: this is
 * for callers that cannot allocate device memory at the point of the call -- code running
 * under a device-memory budget or inside a memory pool that must not grow, a process where
 * another component has already reserved the device memory, or a latency-critical loop where
 * cudaMalloc's implicit device synchronisation is not acceptable.  Same arguments, layouts and
 * result as akra_synth_spin2 (the same kernels run); the phase-array scratch is a fixed
 * 32 MiB device array inside the library (held by every GPU that loads the library until the
 * process exits) instead of a plan workspace.  The plan must already exist, and its device
 * must be the current device (EINVAL otherwise).
 * Limit: R * (4 nside - 1) * (2 lmax + 1) * sizeof(complex) <= 32 MiB (for R = 1: FP64 up to
 * about nside 256 / lmax 512, FP32 up to nside 512 / lmax 1024); larger sizes return
 * EINVAL with a message.  The first call on each device looks up the scratch address
 * (cudaGetSymbolAddress): make that first call before any stream capture.  All calls share
 * the one scratch array, so calls whose kernels overlap on the GPU (different streams, or
 * several threads) race and corrupt each other's results; serialise them.  Nothing in the
 * scratch needs clearing: each call writes every entry before reading it. */
akra_status akra_synth_spin2_static(akra_plan plan, akra_prec prec, const void *d_alm,
                                    void *d_map, int R, void *stream);

/* Exact transpose of akra_synth_spin2 in the real-dof inner product:
 * (a_E, a_B) = (-(g+h)/2, (i/2)(g-h)) with g_lm = Σ_p (u1+iu2)_p 2Y*_lm(p) and
 * h_lm = Σ_p (u1-iu2)_p (-2)Y*_lm(p).  d_map [R][2][npix] -> d_alm [R][2][ntri].
 * No quadrature weights (this is A^T's SHT half, not an inverse transform). */
akra_status akra_adjoint_synth_spin2(akra_plan plan, akra_prec prec, const void *d_map,
                                     void *d_alm, int R, void *stream);

/* Forward operator A (Eq. 7 with Eqs. 2-3): (κ_E, κ_B) -> shear maps,
 * a_E = -D_l κ_E, a_B = -D_l κ_B, then synthesis.  weighted != 0 multiplies the maps by
 * W = ω M N^-1 (needs set_weights, else ENOWEIGHTS). */
akra_status akra_apply_A(akra_plan plan, akra_prec prec, const void *d_x, void *d_map,
                         int weighted, int R, void *stream);

/* Transpose A^T: maps -> (κ_E, κ_B); weighted != 0 multiplies the maps by W first
 * (so weighted A^T y = A^T W y = b of Eq. 8 up to the ω folded into W). */
akra_status akra_apply_At(akra_plan plan, akra_prec prec, const void *d_map, void *d_x,
                          int weighted, int R, void *stream);

/* y = H x = A^T W A x + λ_eff x  (Sec. II B; Eq. 14 operator).  d_x, d_y [R][2][ntri].
 * Only rings with nonzero W are transformed (the others contribute exactly zero).
 * d_x and d_y must not overlap.  Errors: EINVAL, ENOWEIGHTS, ENOMEM, ECUDA. */
akra_status akra_apply_H(akra_plan plan, akra_prec prec, const void *d_x, void *d_y, int R,
                         void *stream);

/* Solve (A^T W A + λ_eff I) x = A^T W y by PCG with x_0 = 0 (Eq. 14 estimator), stopping
 * when ||r||/||b|| < tol for every RHS (or maxiter).  d_shear [R][2][npix] (the pixel
 * shear y), d_x [R][2][ntri] output.  prec F64: everything FP64.  F32: everything FP32
 * (dot products accumulated in FP64).  MIXED: FP64 in/out, b and the outer residual in
 * FP64, inner CG in FP32 (iterative refinement).  The loop runs on the device (one CUDA
 * graph per iteration block); the host only polls a device status.  Blocking; info may be
 * NULL.  Returns the worst per-RHS status: OK, ENOCONV, ENUMERIC, ETIMEOUT (wall-clock
 * budget from akra_set_timeout), or an argument/CUDA error.  On every return, including
 * ETIMEOUT and errors after work was queued, `stream` is ordered after all work the call
 * queued, so d_shear and d_x may be freed or reused in stream order.  After ETIMEOUT the
 * contents of d_x are unspecified and that work can still be running on the device (up to
 * 16 launched CG iterations, and kernels or copies still reading d_shear): synchronise
 * `stream` before the host reads or frees those buffers outside stream order. */
akra_status akra_cg_solve(akra_plan plan, akra_prec prec, const void *d_shear, void *d_x,
                          int R, double tol, int maxiter, akra_cg_info *info, void *stream);

/* As akra_cg_solve but for a given harmonic right-hand side d_b [R][2][ntri]
 * (used for the implicit-adjoint solve of a gradient).  Same precisions and errors. */
akra_status akra_cg_solve_b(akra_plan plan, akra_prec prec, const void *d_b, void *d_x,
                            int R, double tol, int maxiter, akra_cg_info *info, void *stream);

/* Implicit adjoint solve for gradients through akra_cg_solve: given d_g [R][2][ntri], the
 * gradient of a loss w.r.t. the stored (re, im) components of the solution x̂, solve
 * H u = G^{-1} g (G: the real-dof metric, 1 at m = 0 real parts, 2 at m > 0; the ignored
 * imaginary parts at m = 0 get 0) into d_u.  Then dL/dy = W A u (akra_apply_A with
 * weighted = 1) and dL/dN^-1 follows from akra_weight_grad.  Same precisions, tolerances,
 * blocking behaviour and errors as akra_cg_solve_b (the differentiation form of the north
 * star; Eq. 14's estimator differentiated with λ_eff held fixed). */
akra_status akra_cg_solve_adjoint(akra_plan plan, akra_prec prec, const void *d_g, void *d_u,
                                  int R, double tol, int maxiter, akra_cg_info *info,
                                  void *stream);

/* d_grad[p] = ω M_p Σ_r Σ_c Au[r][c][p] (y[r][c][p] - Ax[r][c][p])  for p < npix:
 * the gradient of the loss w.r.t. N^-1_p when Au = A u (u from akra_cg_solve_adjoint) and
 * Ax = A x̂ (both unweighted maps [R][2][npix]), y the shear.  Maps and d_grad in the
 * precision's real type (F64: double, F32: float).  Errors: EINVAL, ENOWEIGHTS, ECUDA. */
akra_status akra_weight_grad(akra_plan plan, akra_prec prec, const void *d_Au, const void *d_y,
                             const void *d_Ax, void *d_grad, int R, void *stream);

/* ---- several instances (uneven nside / lmax, several RHS each) solved together ----------
 * Motivated by the paper's noise realisations and tomographic bins (Sec. III); the batched
 * form is not in the paper.  Each FP32 H application of the inner CG runs as one persistent
 * Legendre-synthesis launch over the work items of all instances (a queue of
 * (instance, m, ring-pair chunk, RHS group) items, heaviest first), one ring-FFT launch over
 * all instances' rings and one persistent Legendre-adjoint launch. */
typedef struct akra_batch_s *akra_batch;

/* Group ninst plans (each with weights set; no plan twice) with R[i] RHS each (1..64).
 * The plans must outlive the batch.  Blocking.  Errors: EINVAL, ENOWEIGHTS, ENOMEM. */
akra_status akra_batch_create(int ninst, const akra_plan *plans, const int *R, akra_batch *out);
void akra_batch_destroy(akra_batch batch);

/* Choose the batch's Legendre tile shape by timing the batched FP32 H (blocking). */
akra_status akra_batch_autotune(akra_batch batch, void *stream);

/* d_y[i] = H_i d_x[i] in FP32 for every instance (complex float [R_i][2][ntri_i]) in one
 * batched pass.  Asynchronous on stream after a blocking upload of the launch arguments. */
akra_status akra_batch_apply_H(akra_batch batch, const void *const *d_x, void *const *d_y,
                               void *stream);

/* Solve every instance: d_shear[i] [R_i][2][npix_i] -> d_x[i] [R_i][2][ntri_i].
 * AKRA_MIXED: FP64 in/out, FP64 b and outer residuals per instance, batched FP32 inner CG;
 * AKRA_F32: FP32 in/out.  info: host array [ninst] (may be NULL).  Blocking; returns the worst
 * status over all instances and RHS. */
akra_status akra_batch_cg_solve(akra_batch batch, akra_prec prec, const void *const *d_shear,
                                void *const *d_x, double tol, int maxiter, akra_cg_info *info,
                                void *stream);

/* Current tile shape (ring pairs per thread, RHS per block) and batched launches so far. */
akra_status akra_batch_describe(akra_batch batch, int *P, int *RG, long long *launches);

/* Run the batch's FP32 Legendre synthesis on the tensor cores (as akra_plan_set_tc_synthesis
 * does for one plan): group = 4, 8, 16 or 32 RHS per work item, 0 for the CUDA-core synthesis.
 * The tensor-core items are (instance, m, 128-ring-pair chunk, RHS group), heaviest first; the
 * adjoint keeps the CUDA-core items.  akra_batch_autotune considers every group up to twice the
 * largest R (from R = 4 on).  A tensor-core completion wait that exceeds its bound is reported as
 * ECUDA by the next akra_batch_cg_solve or akra_batch_autotune.  Blocking (rebuilds the work
 * list).  Errors: EINVAL, ENOMEM. */
akra_status akra_batch_set_tc_synthesis(akra_batch batch, int group);
/* The batch's tensor-core synthesis group (0: CUDA-core synthesis).  Errors: EINVAL. */
akra_status akra_batch_get_tc_synthesis(akra_batch batch, int *group);

/* Preconditioner of the plan's CG solves.  AKRA_PRECOND_SCALAR (default): the paper's scalar
 * P = (mean_all(M N^-1) + λ_eff)^-1 of Eq. 15 (for a scalar P the PCG iterates equal the CG
 * ones).  AKRA_PRECOND_PER_L: the per-l diagonal (mean_all(M N^-1) D_l^2 + λ_eff)^-1, the
 * uniform-sky diagonal of H with the Eq. 3 kernel (beyond the paper; it equals 1/λ_eff on the
 * l < 2 modes, which only the regulariser constrains).  Takes effect at the next solve that
 * involves this plan (single-plan and batched); the weights are recomputed by
 * akra_plan_set_weights.  Errors: EINVAL. */
typedef enum { AKRA_PRECOND_SCALAR = 0, AKRA_PRECOND_PER_L = 1 } akra_precond;
akra_status akra_plan_set_preconditioner(akra_plan plan, akra_precond kind);

/* Field-restricted solves (App. A, "Conditional B-mode solve").  With b = A^T W y as in
 * akra_cg_solve and H_EE, H_BB, H_BE the E/B blocks of the joint operator (Eqs. A3-A6):
 *   AKRA_SOLVE_E: the E-mode normal equations H_EE κ_E = b_E (κ_B held at zero; the B rows
 *     are dropped).  d_x [R][2][ntri] receives (κ̂_E, 0).
 *   AKRA_SOLVE_B_GIVEN_E: the reduced B-mode equation H_BB κ_B = b_B - H_BE κ̂_E (Eq. A8),
 *     with κ̂_E read from the E field of d_x on input (e.g. from an AKRA_SOLVE_E call); the
 *     correction H_BE κ̂_E costs one H application (FP64 unless prec is F32).  d_x keeps its
 *     E field and receives κ̂_B in its B field.
 * Precisions, layouts, blocking behaviour and statuses as akra_cg_solve; info->relres is
 * relative to the reduced right-hand side (b_E, or b_B - H_BE κ̂_E).  Errors: as
 * akra_cg_solve, and EINVAL for any other value of fields. */
typedef enum { AKRA_SOLVE_E = 1, AKRA_SOLVE_B_GIVEN_E = 2 } akra_fields;
akra_status akra_cg_solve_fields(akra_plan plan, akra_prec prec, akra_fields fields,
                                 const void *d_shear, void *d_x, int R, double tol, int maxiter,
                                 akra_cg_info *info, void *stream);

/* Noise-realisation pipeline, shuffling step (Sec. IV, "Power spectrum results": the observed
 * shear values are shuffled among the unmasked pixels, which keeps the survey geometry and
 * noise level and destroys the signal's spatial correlations).  d_shear [2][npix] (γ1, γ2),
 * d_perm [R][npix] int32 source pixel per output pixel (a permutation of the unmasked pixels
 * onto themselves, masked pixels mapping to themselves, for the paper's procedure; any gather
 * is computed as given), d_out [R][2][npix]: out[r][c][p] = shear[c][perm[r][p]].  prec F64 or
 * F32 selects the map type.  The random permutations are the caller's (the library draws no
 * random numbers).  Blocking (reads back an index check).  Errors: EINVAL (arguments, or any
 * perm entry outside [0, npix): those outputs are 0), ENOMEM, ECUDA. */
akra_status akra_shuffle_shear(akra_plan plan, akra_prec prec, const void *d_shear,
                               const int *d_perm, void *d_out, int R, void *stream);

/* E/B power spectra of reconstructed convergence alm (Sec. IV, "Power spectrum results"):
 *   C_l^{XY} = [Re a_X,l0 Re b_Y,l0 + 2 Re Σ_{m>0} a_X,lm conj(b_Y,lm)] / (2l + 1),
 * for (X, Y) = (E,E), (E,B), (B,E), (B,B), per RHS, accumulated in FP64 -- an auto spectrum with
 * d_b = d_a, a cross spectrum of two reconstructions otherwise.  d_a, d_b [R][2][ntri] complex
 * in prec (F64 or F32).  nbins = 0: d_out [R][4][lmax+1] receives C_l; nbins in [1, 64]:
 * d_out [R][4][nbins] receives band powers, the mean of C_l over l in (edges[b], edges[b+1]]
 * (0 for a bin holding no l), edges a host array of nbins + 1 increasing values.  Asynchronous
 * on `stream`.  Errors: EINVAL, ENOMEM (workspace), ECUDA. */
akra_status akra_cl_spectra(akra_plan plan, akra_prec prec, const void *d_a, const void *d_b, int R,
                            int nbins, const double *edges, double *d_out, void *stream);

/* Inner tolerance of the mixed-precision solves (Sec. II C: FP32 inner CG, FP64 refinement):
 * each outer step runs FP32 CG on the normalised FP64 residual to the relative tolerance
 * max(floor, min(0.1, inner_factor · tol / (‖r‖/‖b‖))), i.e. to what this step must gain
 * times a safety factor, but not below the floor.  After an outer step the FP64 residual is
 * about (FP32 tolerance + FP32 operator error) × the previous one, so iterating the FP32 CG
 * below the FP32 operator's relative error (~0.1-0.2 · 2^-24 · lmax) gains nothing.
 * inner_floor = 0 (default) selects that floor, 0.1 · 2^-24 · lmax within [5e-6, 1e-3];
 * inner_factor defaults to 0.5.  Process-wide: the pair is stored together (under a lock) and
 * a solve reads it once per outer step, so it never combines the floor of one call with the
 * factor of another; a solve already running picks up a new pair at its next outer step.
 * Errors: EINVAL unless 0 <= inner_floor < 0.1 and 0 < inner_factor <= 1. */
akra_status akra_set_mixed_policy(double inner_floor, double inner_factor);

/* Host-side wall-clock budget (seconds) for blocking solves; default 3600.  Process-wide
 * (any thread may set it; solves that start afterwards use the new value).  A solve that runs
 * out returns ETIMEOUT with the context still usable; the work it had already queued may
 * still be running, with the caller's stream ordered after it (see akra_cg_solve).
 * Errors: EINVAL unless seconds is finite and 0 < seconds <= 1e9. */
akra_status akra_set_timeout(double seconds);

/* Pick the Legendre tile shapes for this plan, precision and RHS count by timing the
 * candidates on `stream`: ring pairs per thread of the synthesis and, separately, of the
 * adjoint, with a common number of RHS per block.  The choice is cached in the plan and used
 * by every later call with the same (prec, R).  Blocking. */
akra_status akra_autotune(akra_plan plan, akra_prec prec, int R, void *stream);

/* Legendre tile shape used for (prec, R), prec AKRA_F64 or AKRA_F32: ring pairs per thread of
 * the synthesis (*P) and of the adjoint (*PA), RHS per block (*RG) -- the autotuned or forced
 * choice if there is one, else the default.  Errors: EINVAL. */
akra_status akra_plan_get_shape(akra_plan plan, akra_prec prec, int R, int *P, int *PA, int *RG);

/* Force the Legendre tile shape for (prec, R), replacing a default or autotuned choice (for
 * reproducible timing, or to test every compiled shape).  Compiled shapes: (P, RG) and
 * (PA, RG) in {(1,1), (2,1), (4,1), (1,2), (2,2), (1,4)}, and for AKRA_F32 also (3,1), (5,1),
 * (6,1) and (8,1).
 * The results do not depend on the shape beyond rounding order.  Errors: EINVAL. */
akra_status akra_plan_set_shape(akra_plan plan, akra_prec prec, int R, int P, int PA, int RG);

/* The adjoint's own tile shape for (prec, R): ring pairs per thread PA and RHS per block RGA,
 * which may differ from the synthesis' RG (the synthesis amortises its recurrence over the RHS
 * of a block, the adjoint's per-step warp reduction grows with them).  akra_plan_set_shape sets
 * RGA = RG; akra_autotune picks synthesis and adjoint shapes independently; the defaults take
 * PA = 5, RGA = 1 (FP32) and PA = 2, RGA = 2 (FP64) for several RHS.  (PA, RGA) must be a
 * compiled shape (list above).  Errors: EINVAL. */
akra_status akra_plan_set_adjoint_shape(akra_plan plan, akra_prec prec, int R, int PA, int RGA);
akra_status akra_plan_get_adjoint_shape(akra_plan plan, akra_prec prec, int R, int *PA, int *RGA);

/* FP32 Legendre synthesis on the tensor core (the paper has no counterpart; an implementation
 * choice of the FP32 operator).  group = 4, 8, 16 or 32 runs the synthesis of every FP32
 * operator with (prec, R) = (AKRA_F32, R) on tcgen05 tensor cores, RHS taken `group` at a time:
 * the recurrences stay on the CUDA cores, their values split into a TF32 head and an FP32
 * remainder, and the l-sum is three TF32 products (head·head, head·rest, rest·head) accumulated in
 * FP32 -- about 21 bits per product, within the FP32 operator's tolerance.  group = 0 selects the
 * CUDA-core synthesis.  akra_autotune considers both; akra_plan_set_shape resets the choice to
 * the CUDA-core synthesis.  If a tensor-core completion wait exceeds its bound (it should not),
 * the next blocking call (a solve, akra_autotune, akra_time_H_stages) returns ECUDA.
 * Errors: EINVAL (group, R, flat-sky plan). */
akra_status akra_plan_set_tc_synthesis(akra_plan plan, int R, int group);
/* The group set for (AKRA_F32, R): 0 (CUDA-core synthesis) or 4, 8, 16, 32.  Errors: EINVAL. */
akra_status akra_plan_get_tc_synthesis(akra_plan plan, int R, int *group);

/* Measured FMA rate of the current device in TFLOP/s (2 flops per FMA) for prec AKRA_F32 or
 * AKRA_F64: a saturating kernel of independent FMA chains on every SM, timed with CUDA events
 * (tens of milliseconds; blocking).  The denominator of the Legendre kernels' pipe fractions;
 * the paper has no counterpart.  Errors: EINVAL, ENOMEM, ECUDA. */
akra_status akra_fma_rate(akra_prec prec, double *tflops);

/* Work accounting of one Legendre launch (diagnostic; the paper has no counterpart).  For the
 * plan's ring pairs (its active ones once weights are set) laid out as the synthesis
 * (adjoint = 0) or the adjoint (adjoint = 1) lays them out with P ring pairs per thread and NT
 * threads per block, *steps = the (l, m, ring pair) steps from each pair's start point to lmax
 * (the work counted in roofline figures; akra_plan_desc.legendre_steps_*), *lane_steps = the
 * steps the lanes execute: a warp runs all 32 P of its slots from the first 64-step l-tile that
 * holds its earliest start (tiles counted from the block's earliest start) to lmax.  The ratio
 * is the fraction of executed lane-steps that carry counted work.  Blocking.
 * Errors: EINVAL (P outside 1..64, NT not a multiple of 32 in 32..1024, flat-sky plan), ENOMEM,
 * ECUDA. */
akra_status akra_legendre_lane_steps(akra_plan plan, akra_prec prec, int adjoint, int P, int NT,
                                     long long *lane_steps, long long *steps);

/* Time the four stages of one H application (Legendre synthesis, ring FFT x W x FFT,
 * Legendre adjoint, epilogue) with CUDA events on `stream`, averaged over `reps` runs after
 * one warm-up, on the plan's own scratch input.  ms_out[0..3] receive the per-stage
 * milliseconds and ms_out[4] the whole H.  Blocking.  Errors: EINVAL, ENOWEIGHTS, ENOMEM,
 * ECUDA. */
akra_status akra_time_H_stages(akra_plan plan, akra_prec prec, int R, int reps, void *stream,
                               double *ms_out);

#ifdef __cplusplus
}
#endif
#endif /* AKRA_H */
