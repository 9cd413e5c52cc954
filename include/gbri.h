/*
 * gbri.h -- C ABI of the GB300-native sparse radio-interferometric imaging library.
 *
 * The library implements, for one GPU (sm_103a), the measurement operator of
 * Sec. 2 / Eq. 2 of the paper (Phi = W G F Z S: Kaiser-Bessel correction S,
 * zero padding Z, oversampled FFT F, degridding G with a pre-sampled kernel
 * table (Sec. 8.1), noise weights W), its adjoint Phi^dagger = S^T Z^T F^H G^T W^T,
 * the SARA wavelet dictionary Psi / Psi^dagger (Sec. 3.1, Sec. 6.4), the proximal
 * operators of Sec. 4 (soft thresholding, l2-ball projection), the power method
 * for ||Phi||^2 (Sec. 6.3.1) and the solvers of the constrained analysis problem
 * min ||Psi^dagger x||_1 s.t. ||y - Phi x||_2 <= eps, x >= 0: primal-dual
 * (Appendix A.4, Algorithm 7) and Dual Forward-Backward ADMM (Sec. 5,
 * Algorithm 1).
 *
 * Conventions (every call):
 *   - Pointers named d_* are DEVICE pointers on the current CUDA device, owned by
 *     the caller; the library never frees them and never keeps them after the
 *     call returns (except where a create call documents a copy).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; nothing synchronises unless the call says so.
 *   - Precision is fixed per object (plan, wavelet; a solver takes its plan's):
 *     GBRI_F32 = float images and interleaved complex64 {re, im} visibilities,
 *     FP32 arithmetic for the bulk with FP64 global norms, ball test, power
 *     method and convergence test (the mixed-precision path); GBRI_F64 = double
 *     images and complex128 visibilities, FP64 throughout (the plain FP64 path).
 *     Data pointers are void*: their element type is the object's precision.
 *     Images are row-major [n_side][n_side].
 *   - Return value: GBRI_OK (0) or a negative gbri_status.  On error nothing has
 *     been enqueued unless the status is GBRI_ECUDA / GBRI_ECUFFT, in which case
 *     the stream may hold partial work.  gbri_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread).
 *   - Objects (plan, wavelet, solver) are not thread-safe: one object may be used
 *     by one stream at a time.  Different objects are independent.
 */
#ifndef GBRI_H
#define GBRI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------------- */
#define GBRI_OK 0
#define GBRI_EINVAL (-1)      /* bad argument (null pointer, size, unsupported shape) */
#define GBRI_ENOMEM (-2)      /* device or host allocation failed */
#define GBRI_ECUDA (-3)       /* a CUDA runtime call or kernel launch failed */
#define GBRI_ECUFFT (-4)      /* a cuFFT call failed */
#define GBRI_ETIMEOUT (-5)    /* a bounded device wait gave up */
#define GBRI_ENONFINITE (-6)  /* non-finite input rejected */
#define GBRI_ENOTCONV 1       /* warning: solver stopped at max_iter before rel_tol */

#define GBRI_F32 0
#define GBRI_F64 1

/* flags for phi / phi_adjoint / solver_create */
#define GBRI_PLAN_ORDER 1u   /* visibility buffers are in the plan's sorted order (no permutation) */

typedef struct gbri_plan gbri_plan;
typedef struct gbri_wavelet gbri_wavelet;
typedef struct gbri_solver gbri_solver;
typedef struct gbri_wstack gbri_wstack;

/* ---- measurement operator plan (Sec. 2, Eq. 2; Sec. 8.1) ------------------ */
typedef struct {
  int32_t n_side;            /* image side N_side (image is N_side x N_side); even, >= 16 */
  int32_t oversample;        /* grid oversampling alpha per axis, 2..4; K = alpha * N_side must be a multiple of 16 */
  int32_t J;                 /* kernel support in grid cells: 4 or 6 */
  int32_t samples_per_unit;  /* table samples per grid cell S: power of two, 16 <= S <= 4096 */
  double kb_beta;            /* Kaiser-Bessel shape; <= 0 selects 2.34 * J */
  int64_t M;                 /* number of visibilities, >= 0 */
  int32_t precision;         /* GBRI_F32 or GBRI_F64: tables, grids and data in float or double */
  int32_t vis_per_run;       /* longest run of one grid cell's visibilities a gridding thread sums in
                                registers before one shared-memory update: 1..1024; 0 selects 64 */
  int32_t autotune;          /* 1: time the run lengths 8, 16, 64 and the resident blocks per SM of the
                                visibility kernels at plan creation and keep the fastest (cached per
                                problem shape for the process); 0: vis_per_run and the occupancy limit */
  int32_t interp_order;      /* kernel-table interpolation (Sec. 8.1 names zeroth and first order):
                                0: zeroth order, k~ = round(k S), each tap takes the nearest table
                                sample; 1: first order, k is quantised 256 S steps per cell and each
                                tap interpolates linearly between its two table samples (8 bits of
                                fraction per axis kept beside the metadata: 2 more bytes per visibility) */
  int32_t deterministic;     /* 1: gridding results are bitwise reproducible from run to run (and the
                                same alone or inside a batch): work items are taken in a fixed order,
                                every gridding work item writes its whole window to a slot of its own,
                                and a second pass sums, for every grid cell, the windows covering it in
                                a fixed order, instead of float atomics on the cells tiles share; the
                                slots take 8 (T + J - 1)^2 bytes per work item (FP32; 16 for FP64);
                                plan creation orders each cell's visibilities by caller index, and
                                autotune is ignored (timed choices would change the layout); local
                                l2 balls (n_balls > 1) still sum their block norms with shared-memory
                                atomics and are not covered;
                                0: atomics (faster, last-bit differences between runs) */
  int32_t layout;            /* order of the visibilities inside a grid tile: 0 = automatic, the step
                                layout for FP32 plans whose taps come from the kernel's polynomial fit
                                with J = 4 (each 32-run group stored step-major: the k-th visibility of
                                every run side by side; the layout of the fused degridding + gridding
                                pass of the primal-dual iteration and FISTA) and the run layout
                                otherwise; 1 = the run layout (each run of one cell's visibilities
                                consecutive; faster for Phi and Phi^dagger applied alone, ADMM and
                                local l2 balls) */
} gbri_plan_desc;

/* Build a plan: quantises every (u, v) once in FP64 to the fixed-point grid
 * coordinate k~ = round_half_away(u * K * S / (2 pi)) (Sec. 8.1 zeroth-order
 * pre-sampling), sorts the visibilities by grid tile and cell, packs per-visibility
 * metadata, builds the kernel table and the correction 1/ghat, and creates the
 * cuFFT plan.  d_uvw_weight: [M][4] float rows {u, v, w, weight}, u and v in
 * radians per pixel, normally |u|, |v| <= pi; values outside wrap around the
 * grid, as the DFT is 2 pi periodic (w is ignored: coplanar array).  The plan
 * copies what it needs; d_uvw_weight may be freed after the call returns.
 * Synchronises `stream`.  Errors: EINVAL (shape; |u| or |v| > 16 pi), ENOMEM,
 * ENONFINITE (non-finite u, v or weight), ECUDA, ECUFFT. */
int32_t gbri_plan_create(gbri_plan** out, const gbri_plan_desc* desc, const float* d_uvw_weight,
                         void* stream);
int32_t gbri_plan_destroy(gbri_plan* plan);

/* Launch configuration the plan uses (after autotuning, if requested): visibilities per run and
 * persistent blocks of the degridding and gridding kernels.  Any pointer may be NULL. */
int32_t gbri_plan_launch_config(const gbri_plan* plan, int32_t* vis_per_run, int32_t* degrid_blocks,
                                int32_t* grid_blocks);

/* Bounds-check report of a library built with GBRI_DEBUG (paper_1903_04502_gb300/build.py,
 * debug=True: libgbri_debug.so; the paper has no counterpart).  In that build every visibility
 * kernel checks its window, accumulator, grid, half-spectrum, slot and visibility indices; an
 * index that would leave its buffer sets a bit in the plan's device error word (1 window,
 * 2 accumulator, 4 grid, 8 visibility position, 16 half spectrum, 32 deterministic slot),
 * records the first such index, and the access is skipped (no trap).  Copies the bits and that
 * index (may be NULL) to the host and clears the word when reset != 0; synchronises `stream`.
 * Errors: EINVAL (null arguments, or a library built without the checks). */
int32_t gbri_plan_debug_word(const gbri_plan* plan, uint32_t* bits, int64_t* first_index, int32_t reset,
                             void* stream);

/* How the plan's visibility kernels get the Kaiser-Bessel tap weights (Sec. 8.1):
 * 0 = the zeroth-order pre-sampled table in shared memory; 1 = first-order interpolation
 * between table samples (interp_order = 1); 2 = FP32 zeroth-order plans: a polynomial fit of
 * the kernel on each unit segment of its support, evaluated at the same quantised positions
 * the table is sampled at (the table's weights to within 3e-7; chosen when the fit reaches
 * that bound, which it does for J = 4 and 6 with the default beta; the environment variable
 * GBRI_TAP_TABLE=1 at plan creation keeps the table instead).  Errors: EINVAL (null). */
int32_t gbri_plan_tap_mode(const gbri_plan* plan, int32_t* mode);

/* Plan facts: K, M, number of non-empty 16 x 16 grid tiles, device bytes held. Any pointer may be NULL. */
int32_t gbri_plan_info(const gbri_plan* plan, int64_t* K, int64_t* M, int64_t* n_tiles,
                       int64_t* device_bytes);

/* ---- non-coplanar measurement operator by w-stacking (Sec. 7.1 names w-stacking as the
 * software's wide-field method and defers its definition to the wide-field paper; reading R14) --
 * y_i = w_i sum_{q,p} x[q,p] exp(-i (u_i p' + v_i q')) exp(-2 pi i w_i (n - 1)), n = sqrt(1 - l^2 - m^2),
 * l = p' pixel_size, m = q' pixel_size: u, v in radians per pixel as for the coplanar plan, w (the
 * third column of d_uvw_weight) in wavelengths.  The w range is cut into n_planes equal bins;
 * each visibility's w is replaced by its bin centre w_k, and plane k applies a coplanar plan
 * (desc, with M the plane's count) to the image times C_k = exp(-2 pi i w_k (n - 1)); the adjoint
 * sums Re(conj(C_k) (plane k's adjoint)).  The phase error of the binning is at most
 * 2 pi (dw / 2) max|n - 1| per visibility.  Creation copies the coordinates to the host, bins
 * them in FP64 and builds one plan per non-empty plane (synchronises `stream`); every plan owns
 * its grids (about 60 bytes per grid cell in FP32).  Errors: EINVAL (n_planes outside [1, 4096],
 * pixel_size <= 0, a field of view reaching the horizon, the plan errors), ENONFINITE, ENOMEM, ECUDA. */
int32_t gbri_wstack_create(gbri_wstack** out, const gbri_plan_desc* desc, const float* d_uvw_weight,
                           int32_t n_planes, double pixel_size, void* stream);
int32_t gbri_wstack_destroy(gbri_wstack* w);
/* Planes, and (host arrays of n_planes entries, may be NULL) visibilities per plane and plane centres w_k. */
int32_t gbri_wstack_info(const gbri_wstack* w, int32_t* n_planes, int64_t* counts, double* centres);
/* y = Phi x (caller order): x real [n_side][n_side], y complex [M], desc's precision.  Two coplanar
 * applications per non-empty plane (the screened image's real and imaginary parts). */
int32_t gbri_wstack_phi(gbri_wstack* w, const void* d_x, void* d_y, void* stream);
/* x = Phi^dagger y (x overwritten).  Two coplanar adjoints per non-empty plane. */
int32_t gbri_wstack_phi_adjoint(gbri_wstack* w, const void* d_y, void* d_x, void* stream);

/* Copy the plan's permutation (plan position -> caller's visibility index) to d_perm [M] int32. */
int32_t gbri_plan_permutation(const gbri_plan* plan, int32_t* d_perm, void* stream);

/* Reorder a complex visibility vector [M] between the caller's order and plan order.
 * to_plan = 1: d_out[pos] = d_in[perm[pos]]; to_plan = 0: d_out[perm[pos]] = d_in[pos].
 * d_in and d_out must not overlap. */
int32_t gbri_vis_reorder(const gbri_plan* plan, const void* d_in, void* d_out, int32_t to_plan,
                         void* stream);

/* y = Phi x = W G F Z S x (Sec. 2, Eq. 2).  d_x: [n_side][n_side] real image.
 * d_y: [M] complex, written (caller's order unless flags has GBRI_PLAN_ORDER). */
int32_t gbri_phi(gbri_plan* plan, const void* d_x, void* d_y, uint32_t flags, void* stream);

/* x = Phi^dagger y = Re(S^T Z^T F^H G^T W^T y) (Sec. 2; real part because the sky
 * is real).  d_y: [M] complex (caller's order unless GBRI_PLAN_ORDER); d_x:
 * [n_side][n_side] real, overwritten. */
int32_t gbri_phi_adjoint(gbri_plan* plan, const void* d_y, void* d_x, uint32_t flags, void* stream);

/* ||Phi||^2 by the power method on Phi^dagger Phi (Sec. 6.3.1), FP64 norms.
 * Start vector 0.5 + U[0,1) with U from SplitMix64 at counters seed + k * 0x9E3779B97F4A7C15
 * (k = 1..N, top 53 bits).  Stops when the relative change of the estimate is
 * <= tol or after max_iter iterations.  Synchronises `stream` each iteration.
 * Writes the estimate to *op_norm_sq and the iteration count to *iters (host,
 * iters may be NULL). */
int32_t gbri_op_norm(gbri_plan* plan, int32_t max_iter, double tol, uint64_t seed, double* op_norm_sq,
                     int32_t* iters, void* stream);

/* ---- SARA wavelet dictionary (Sec. 3.1, Sec. 6.4, Sec. 7.5) --------------- */
/* db_orders[n_w] (host): 0 = Dirac basis, N in 1..10 = Daubechies dbN (2N taps,
 * minimum phase, derived in the library by spectral factorisation).  Periodic
 * boundaries, rows then columns per level, Mallat layout, `levels` levels; the
 * stack is scaled by 1/sqrt(n_w) so that Psi Psi^dagger = I.  n_side must be
 * divisible by 2^levels and n_side >> levels >= 2. */
int32_t gbri_wavelet_create(gbri_wavelet** out, int32_t n_side, int32_t levels, const int32_t* db_orders,
                            int32_t n_w, int32_t precision);
int32_t gbri_wavelet_destroy(gbri_wavelet* wav);

/* x = Psi alpha = sum_b IDWT_b(alpha_b) / sqrt(n_w).  d_alpha: [n_w][n_side][n_side]; d_x: image. */
int32_t gbri_psi(gbri_wavelet* wav, const void* d_alpha, void* d_x, void* stream);

/* alpha = Psi^dagger x: alpha_b = DWT_b(x) / sqrt(n_w). */
int32_t gbri_psi_adjoint(gbri_wavelet* wav, const void* d_x, void* d_alpha, void* stream);

/* ---- proximal operators (Sec. 4) ------------------------------------------ */
/* Soft thresholding (Sec. 4.3): out_i = 0 if |in_i| <= lambda, else in_i (|in_i| - lambda) / |in_i|.
 * n elements of real (is_complex = 0) or complex (is_complex = 1) type of the given precision.
 * d_in == d_out allowed. */
int32_t gbri_prox_l1(const void* d_in, void* d_out, int64_t n, double lambda, int32_t is_complex,
                     int32_t precision, void* stream);

/* Weighted soft thresholding (the reweighted l1 prox): threshold lambda * w_i per element.
 * d_w: n non-negative real weights of the same precision (real even for complex input).
 * d_in == d_out allowed. */
int32_t gbri_prox_l1_weighted(const void* d_in, const void* d_w, void* d_out, int64_t n, double lambda,
                              int32_t is_complex, int32_t precision, void* stream);

/* Projection onto the l2 ball of radius eps centred at d_center (Sec. 4.2 and the
 * global constraint of Sec. 6.8): out = z if ||z - c|| <= eps, else c + eps (z - c) / ||z - c||.
 * Complex vectors of length M in the given precision; the norm is accumulated in
 * FP64 (GBRI_F32: per-thread partial sums in FP32, compensated).  d_norm_out (device
 * double, may be NULL) receives ||z - c||.  d_out may alias d_z.  Uses a temporary
 * device buffer from the stream-ordered allocator. */
int32_t gbri_proj_l2ball(const void* d_z, const void* d_center, void* d_out, int64_t M, double eps,
                         double* d_norm_out, int32_t precision, void* stream);

/* Allocation-free variant of gbri_proj_l2ball for GBRI_F32 complex64 vectors (the paper
 * has no counterpart; this is a library convenience).  Same arguments (without the
 * precision), result and error behaviour, but the FP64
 * reduction scratch is a fixed 1024-entry (8 KB) device array inside the library
 * instead of a stream-ordered allocation, for callers that cannot allocate device
 * memory at that point (their own pool already holds the memory, an out-of-memory
 * handler, a loop that must not synchronise).  No cudaMalloc or cudaFree is made.
 *  - The array lives on every GPU that loads the library until the process exits.
 *  - The first call on a device resolves the array's device address for that device
 *    (cudaGetSymbolAddress, with the device current) and caches it; make that first
 *    call before any stream capture.  The cached address belongs to the device's
 *    primary context: after cudaDeviceReset on that device it is stale, so do not
 *    call this entry point on that device again in the same process.
 *  - The number of reduction blocks follows the SM count of the current device.
 *  - Every call shares the one array: calls that overlap on the GPU (different
 *    streams, or devices sharing nothing but the same call in flight) race.  Each
 *    call writes every scratch entry it reads, so nothing needs clearing.
 *  - Returns GBRI_EINVAL if a launch would need more than 1024 partials (one per
 *    reduction block; at most 4 per SM, so only GPUs with more than 256 SMs). */
int32_t gbri_proj_l2ball_noalloc(const float* d_z, const float* d_center, float* d_out, int64_t M, double eps,
                                 double* d_norm_out, void* stream);

/* ---- solvers (Appendix A.4 Algorithm 7; Sec. 5 Algorithm 1; Algorithm 4) --- */
#define GBRI_ALGO_PD 0
#define GBRI_ALGO_ADMM 1
/* FISTA (Algorithm 4) on the unconstrained analysis problem (Sec. 3.1, the MAP estimate)
 * min_x 1/2 ||y - Phi x||^2 + gamma ||Psi^dagger x||_1, x >= 0 (the paper's 1 / (2 sigma^2)
 * data weight folded into gamma); prox of lambda * (gamma ||Psi^dagger .||_1 + iota_{R+}) by the
 * Dual Forward-Backward function of Algorithm 1 (eta, dualfb_iters); eps is not used. */
#define GBRI_ALGO_FISTA 2

typedef struct {
  int32_t algo;          /* GBRI_ALGO_PD, GBRI_ALGO_ADMM or GBRI_ALGO_FISTA */
  int32_t max_iter;      /* iterations run by gbri_solve */
  double rel_tol;        /* stop when ||x+ - x|| / ||x+|| < rel_tol (Sec. 6.6); 0 = never */
  double eps;            /* l2-ball radius epsilon (> 0; PD and ADMM) */
  double gamma;          /* l1 weight; <= 0 selects 1e-3 max|Psi^dagger Phi^dagger y| / ||Phi||^2 (PD, ADMM)
                            or 1e-3 max|Psi^dagger Phi^dagger y| (FISTA) */
  double op_norm_sq;     /* ||Phi||^2; <= 0 runs the power method (200 iterations, tol 1e-8, seed) */
  double tau;            /* PD primal step; <= 0 selects 0.49 */
  double sigma1;         /* PD step of the l1 dual; <= 0 selects 1 */
  double sigma2;         /* PD step of the l2-ball dual; <= 0 selects 1 / ||Phi||^2 */
  double theta;          /* PD extrapolation in [0, 1]; < 0 selects 1 */
  double rho;            /* ADMM / FISTA gradient step (FISTA: lambda); <= 0 selects 1 / ||Phi||^2 */
  double varrho;         /* ADMM multiplier step; <= 0 selects 1 */
  double eta;            /* DualFB step (ADMM, FISTA); <= 0 selects 1 */
  int32_t dualfb_iters;  /* DualFB inner iterations (ADMM, FISTA; >= 1; 0 selects 1) */
  int32_t check_every;   /* host reads the convergence test every k iterations (0 selects 10) */
  uint64_t seed;         /* power-method start vector seed */
  int32_t n_balls;       /* PD / ADMM fidelity constraint: 0 or 1 = the global l2 ball of radius eps;
                            2..64 = local l2 balls (Sec. 6.9): the plan order is cut at tile boundaries
                            into n_balls consecutive ranges -- walking the non-empty tiles in plan order
                            with cumulative visibility count C, ball j (< n_balls - 1) ends after the
                            first tile at which C * n_balls >= (j + 1) * M (at most one ball ends per
                            tile) -- and ball j constrains ||y_j - Phi_j x|| <= eps * sqrt(M_j / M), so
                            that the radii add up to eps in quadrature.  EINVAL if fewer non-empty balls
                            result. */
  int32_t reserved;      /* must be 0 */
} gbri_solve_params;

typedef struct {
  int32_t iters;             /* iterations run */
  int32_t status;            /* GBRI_OK or GBRI_ENOTCONV */
  double rel_change;         /* last ||x+ - x|| / ||x+|| (FP64) */
  double residual_norm;      /* ||y - Phi x|| at exit (FP64) */
  double op_norm_sq;         /* ||Phi||^2 used */
  double gamma;              /* gamma used */
  double ms_total;           /* wall time of the solve on the device, ms */
} gbri_solve_report;

/* Stateful solver: keeps the iterate and dual variables resident on the device.
 * The plan and the wavelet object must have the same precision, which the solver
 * takes.  d_y: [M] complex data (caller's order unless GBRI_PLAN_ORDER); it is copied.
 * Synchronises `stream` (power method / gamma when requested). */
int32_t gbri_solver_create(gbri_solver** out, gbri_plan* plan, gbri_wavelet* wav, const void* d_y,
                           const gbri_solve_params* params, uint32_t flags, void* stream);
int32_t gbri_solver_destroy(gbri_solver* s);
/* Run n_iter iterations without any host synchronisation.  All work is ordered on
 * `stream`: a primal-dual iteration forks its wavelet half (Psi^dagger with the dual update,
 * then Psi) onto a solver-owned stream after the previous iteration and joins it back
 * before the primal update (a graph edge when the iteration is a captured CUDA graph), so
 * the call returns with every iteration enqueued behind `stream`'s earlier work and ahead
 * of its later work.  A solver is stepped by one host thread at a time. */
int32_t gbri_solver_step(gbri_solver* s, int32_t n_iter, void* stream);
/* Capture the solver's iteration as a CUDA graph now (stream capture on a stream of the
 * solver's own, thread-local capture mode); otherwise the first graph step or the first batch
 * step that holds the solver does it.  A program that sets solvers up on one thread while
 * another thread synchronises or frees device memory should capture on the set-up thread, so
 * that no capture runs while those calls do.  Idempotent.  Errors: EINVAL (null solver, or kernel
 * timing on), ECUDA. */
int32_t gbri_solver_capture(gbri_solver* s);
/* Reweighted l1 (SARA's reweighting, Sec. 3.1; the weights' formula follows the SARA
 * paper the text cites): sets per-coefficient weights w_i = delta / (delta + |(Psi^dagger x)_i|)
 * from the current iterate x; from then on the l1 prior is gamma sum_i w_i |(Psi^dagger x)_i|
 * (every l1 bound gamma becomes gamma w_i: the PD dual clip, the DualFB step of ADMM and
 * FISTA).  The dual variables are kept.  delta > 0.  The first call allocates the weights
 * and drops the solver's captured iteration (captured again at the next step; a batch
 * holding the solver rebuilds its graph).  No host synchronisation. */
int32_t gbri_solver_reweight(gbri_solver* s, double delta, void* stream);
/* Copy the current iterate x to d_x (image). */
int32_t gbri_solver_get_x(gbri_solver* s, void* d_x, void* stream);
/* Iterations run and the last FP64 relative change ||x+ - x|| / ||x+|| (host; INFINITY before the
 * first iteration).  Reads one device scalar: synchronises `stream`, no other work. */
int32_t gbri_solver_status(gbri_solver* s, int32_t* iters, double* rel_change, void* stream);
/* Fill *report (host) with the iteration count, last relative change and residual. Synchronises. */
int32_t gbri_solver_report(gbri_solver* s, gbri_solve_report* report, void* stream);

/* One-shot solve: create, iterate up to max_iter (checking rel_tol every check_every
 * iterations on the host), write x to d_x_out, fill *report (host, may be NULL), destroy.
 * Returns GBRI_OK, GBRI_ENOTCONV (max_iter reached with rel_tol > 0) or an error. */
int32_t gbri_solve(gbri_plan* plan, gbri_wavelet* wav, const void* d_y, const gbri_solve_params* params,
                   void* d_x_out, gbri_solve_report* report, uint32_t flags, void* stream);

/* ---- batched execution (many independent problems in one graph launch) ----- */
/* A batch holds resident solvers of independent problems (each with its own plan
 * and wavelet object; sizes, visibility counts and kernel supports may differ).
 * gbri_batch_step runs n_iter iterations of every member: each iteration is one
 * launch of a CUDA graph whose branches are the members' captured iterations, so
 * the problems share the device.  Members may be added and removed between steps
 * (continuous batching; the graph is rebuilt on the next step).  Remove a solver
 * before destroying it.  No paper counterpart: the paper distributes one problem
 * over cluster nodes (Sec. 6); on one GPU the independent problems share it. */
typedef struct gbri_batch gbri_batch;
int32_t gbri_batch_create(gbri_batch** out);
int32_t gbri_batch_destroy(gbri_batch* b);
/* Errors: EINVAL if the solver is already a member or shares a plan or wavelet object with one. */
int32_t gbri_batch_add(gbri_batch* b, gbri_solver* s);
int32_t gbri_batch_remove(gbri_batch* b, gbri_solver* s);
int32_t gbri_batch_size(const gbri_batch* b);
/* No host synchronisation.  EINVAL while kernel timing (gbri_profile_enable) is on. */
int32_t gbri_batch_step(gbri_batch* b, int32_t n_iter, void* stream);
/* Shared pass (on by default): members that are primal-dual solvers with a global l2 ball on
 * FP32 plans of the step layout (gbri_plan_desc.layout) with the same kernel, not
 * deterministic, share one launch of the fused degridding + gridding pass per iteration: a
 * work list over all of their gridding items, taken from one counter (up to 256 members,
 * heaviest first; at least two).  Each such member's iteration runs in two phases around it
 * (up to its forward FFT; from its inverse FFT on); the other members keep their own
 * captured iterations.  Results equal the members stepped alone up to the summation order of
 * the l2-ball norm.  enable: 0 or 1 (EINVAL otherwise); takes effect at the next step. */
int32_t gbri_batch_set_shared_pass(gbri_batch* b, int32_t enable);
/* Members in the shared pass at the last step (0 when none). */
int32_t gbri_batch_shared_members(const gbri_batch* b);

/* ---- diagnostics ------------------------------------------------------------ */
/* Kernel timing with CUDA events recorded around each library kernel launch on its
 * own stream.  capacity = events per kind to keep (0 disables).  Kinds: */
#define GBRI_K_PAD 0
#define GBRI_K_FFT_FWD 1
#define GBRI_K_DEGRID 2
#define GBRI_K_GRID 3
#define GBRI_K_FFT_INV 4
#define GBRI_K_CROP 5
#define GBRI_K_PSI_ADJ 6
#define GBRI_K_PSI 7
#define GBRI_K_UPDATE 8
#define GBRI_K_OTHER 9
#define GBRI_K_DEGRID_GRID 10   /* degridding fused with the gridding of its output */
#define GBRI_K_COUNT 11
int32_t gbri_profile_enable(int32_t capacity);
/* Sum of recorded durations (ms) and number of launches of one kind. Synchronises the device. */
int32_t gbri_profile_read(int32_t kind, double* total_ms, int64_t* launches);
/* Test hook for allocation-failure handling (the paper has no counterpart): the after_n-th
 * device allocation the library makes from now on (plan, solver state) fails as if the device
 * were out of memory, and the call that made it returns GBRI_ENOMEM after releasing what it had
 * allocated; 0 disarms.  No GPU fault is involved.  Errors: EINVAL (after_n < 0). */
int32_t gbri_debug_inject_alloc_failure(int32_t after_n);
/* Total number of library kernel launches since the last gbri_profile_enable / reset. */
int64_t gbri_launch_count(void);
void gbri_launch_count_reset(void);

const char* gbri_last_error(void);
const char* gbri_version(void);

#ifdef __cplusplus
}
#endif
#endif /* GBRI_H */
