/*
 * libfmm — natively periodic Fast Multipole Method on one GB300 (sm_103a).
 *
 * The method is Gnedin, "Natively Periodic Fast Multipole Method:
 * Approximating the Optimal Green's Function" (arXiv:2011.07099).  A density
 * field on a periodic N^3 mesh over the unit box is solved for the potential
 * Phi (lap Phi = rho - mean rho, Sec. 1: G_0 = -1/(4 pi r)) and the
 * acceleration g = -grad Phi, by an FMM whose interaction-zone Green's
 * function is the approximately optimal periodic G_S1 of eq. gfs1 (Sec. 4):
 *
 *   G_S1(x) = -1/(4 pi |xhat|),  xhat_i = (9/(8 pi)) sin(pi x_i) - (1/(24 pi)) sin(3 pi x_i).
 *
 * Conventions shared by every entry point
 *   - Mesh arrays are float32, C order [z][y][x] (x fastest), N^3 elements.
 *     Cell (i,j,k) has its centre at ((i+1/2)/N, (j+1/2)/N, (k+1/2)/N).
 *   - accel is structure-of-arrays: ax[N^3] | ay[N^3] | az[N^3].
 *   - Device pointers must be 16-byte aligned device memory owned by the
 *     caller; the library never frees them.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  fmm_solve only enqueues work; it does not synchronise.
 *   - Every int-returning call returns FMM_OK (0) or an FMM_ERR_* code; the
 *     same code is kept per host thread and readable by fmm_last_error().
 *   - A plan is not thread-safe: one host thread and one stream at a time.
 *
 * Tree (Sec. 2): level l has 2^l nodes per dimension; L is the leaf level,
 * each leaf holds S^3 cells, S = N / 2^L.  Each node carries a gridlet of
 * order^3 effective masses (order = N_g of the paper) on a cell-centred
 * uniform mini-mesh.
 */
#ifndef FMM_H
#define FMM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_plan fmm_plan;

/* ---- error codes ---------------------------------------------------- */
#define FMM_OK              0
#define FMM_ERR_ARG         1   /* invalid argument (sizes, pointers, alignment, mode) */
#define FMM_ERR_CUDA        2   /* a CUDA runtime call failed */
#define FMM_ERR_TIMEOUT     3   /* a bounded device-side wait gave up */
#define FMM_ERR_INTERNAL    4   /* a device-side consistency check failed */
#define FMM_ERR_ALLOC       5   /* device or host allocation failed */
#define FMM_ERR_UNSUPPORTED 6   /* valid request this build does not implement */

/* ---- M2L precision modes (fmm_plan_set_precision) -------------------- */
#define FMM_PREC_FP32    0  /* plain form: CUDA cores, FP32 with the extended-
                               precision coarse levels described below        */
#define FMM_PREC_BF16    1  /* M2L levels >= 4 (order >= 7: the leaf level) on
                               tcgen05 tensor cores, BF16 operands, FP32
                               accumulation in TMEM                           */
#define FMM_PREC_BF16X3  2  /* as BF16 with split products hi*hi+hi*lo+lo*hi */

/* ---- plan lifecycle -------------------------------------------------- */

/* Create a plan for an N^3 periodic mesh, leaf level L and gridlet order.
 *   N     mesh cells per dimension; N = S * 2^L with S in {1, 2, 3, 4, 6, 8, 16}
 *         (16 is the sub-grid of the paper's accuracy experiment, Sec. 3).
 *   L     leaf level, 2 <= L <= 8 (L = 2 is the two-level special case of
 *         Sec. 3, exact when order == S; the general case is L >= 3, Sec. 2).
 *   order gridlet points per dimension (N_g), 1 <= order <= 8.
 * Allocates the plan's device buffers on the current device and tabulates
 * G_S1 and grad G_S1 in FP64 for every level (Sec. 3 eq. fmm2, Sec. 4
 * eq. gfs1).  Synchronises the device before returning.
 * Returns NULL on error (fmm_last_error() gives the code). */
fmm_plan* fmm_plan_create(int N, int L, int order);

/* Release every resource of the plan (NULL is allowed).  Synchronises the
 * device first so that no enqueued solve still uses the plan's buffers. */
void fmm_plan_destroy(fmm_plan* plan);

/* ---- solve ------------------------------------------------------------ */

/* One full solve, enqueued on `stream`:
 *   density   device, N^3 float32, read only.
 *   potential device, N^3 float32, written (every element).
 *   accel     device, 3*N^3 float32 SoA, written (every element).
 * Steps (Sec. 2, Sec. 3 eqs. fmm1-fmm3): mean removal and P2M at the leaves,
 * M2M up to level 2, M2L over the interaction zone at every level 2..L
 * (37 periodic nodes at level 2, 189 below) with G_S1, L2L down the tree,
 * and at each leaf L2P plus the direct near-zone sum over its 27 periodic
 * neighbour leaves.  Buffers must not overlap.  Returns FMM_ERR_ARG for NULL
 * or misaligned pointers, FMM_ERR_CUDA if a launch fails.  The return value
 * covers the enqueueing only: a bounded device-side wait of the tensor-core
 * M2L that runs out (fmm_plan_set_timeout_ms) is recorded in the plan's
 * device error word, so the outputs are valid only once fmm_plan_check()
 * has returned FMM_OK after the solve. */
int fmm_solve(fmm_plan* plan, const float* density, float* potential,
              float* accel, void* stream);

/* End-to-end variant with HOST buffers (same shapes as fmm_solve).  Copies
 * density host->device, solves, copies potential and accel device->host on
 * `stream`, and synchronises the stream before returning.  The host buffers
 * should be page-locked for full copy bandwidth; pageable memory works but is
 * slower.  Device staging buffers are owned by the plan (allocated on first
 * use). */
int fmm_solve_host(fmm_plan* plan, const float* density_host,
                   float* potential_host, float* accel_host, void* stream);

/* ---- configuration ------------------------------------------------------ */

/* Select the M2L arithmetic (FMM_PREC_*).  Takes effect at the next solve.
 * FMM_PREC_BF16 / FMM_PREC_BF16X3 apply to levels >= 4 (see
 * fmm_plan_set_tc_min_level).  In every mode the coarse levels, whose
 * long-range sums cancel most, run on the CUDA cores in extended precision:
 * level 2 in double-float (error-free products and sums), level 3 with split
 * tables, both reduced in FP64 into FP64 local fields.  At order >= 7 every
 * level above the leaves keeps FP64 local fields: in the tensor-core modes
 * levels >= 5 of them run "bf16x6" (both operands split in three BF16 parts,
 * six products, partials of each 32-deep stage added into a double-float
 * total, written in FP64), the coarser ones the double-float CUDA-core
 * kernel, and the leaf level the selected mode.  The first tensor-core
 * selection allocates and tabulates the split BF16 tables, translation tiles
 * and multipole buffers (synchronous).  Order 1 ignores the tensor-core
 * modes.  FMM_ERR_ARG for an unknown mode. */
int fmm_plan_set_precision(fmm_plan* plan, int mode);

/* Boundary of the problem.  FMM_BOUNDARY_PERIODIC (default) is the natively
 * periodic method.  FMM_BOUNDARY_ISOLATED is the non-periodic problem of
 * Sec. 3's accuracy experiment (eq. gerr), which separates the multipole-
 * expansion error from the Green's-function error: every table holds the
 * Newtonian G_0 = -1/(4 pi r) (same cell self term), no mean is removed
 * (m = rho / N^3), and the interaction and near zones keep only nodes inside
 * the box (Sec. 2 zones without the wrap).  Corrections (network, grid) and
 * the G_S ansatz are not applied while isolated.  Re-tabulates
 * (synchronous).  FMM_ERR_ARG for an unknown value. */
#define FMM_BOUNDARY_PERIODIC 0
#define FMM_BOUNDARY_ISOLATED 1
int fmm_plan_set_boundary(fmm_plan* plan, int boundary);

/* The periodic Green's function of the tables and the near zone.
 * FMM_GREEN_S1 (default): G_S1 of eq. gfs1.  FMM_GREEN_S: the ansatz G_S of
 * Sec. 3, xi_n(t) = sin(pi t)/pi + sum_k a_k (sin((2k+1) pi t)/((2k+1) pi)
 * - sin(pi t)/pi) with a[0..na-1] = a_1..a_na, 1 <= na <= 4 (G_S1 is na = 1,
 * a_1 = -1/8); used to fit a_k (Table 1).  FMM_GREEN_X: the exact-in-real-
 * space G_X = -1/(4 pi |x <> L|) of eq. gfx (a and na ignored), whose kink
 * at half the box aliases (Fig. errex).  Corrections (network, grid) apply
 * to G_S1 only.  Re-tabulates (synchronous).  FMM_ERR_ARG otherwise. */
#define FMM_GREEN_S1 0
#define FMM_GREEN_S  1
#define FMM_GREEN_X  2
int fmm_plan_set_green(fmm_plan* plan, int kind, const double* a, int na);

/* Any periodic Green's function given on the N^3 mesh, e.g. the exact-in-
 * Fourier-space G_K of eq. gfk (whose real-space values have no closed form):
 * mesh (device or host, 4 N^3 doubles, copied) holds G, -dG/dx, -dG/dy,
 * -dG/dz at the offsets d/N, d in [0, N)^3, x fastest, d = 0 holding the cell
 * self term (the layout fmm_plan_mesh_green writes).  Every table entry is
 * then a mesh value, which needs every gridlet point on a cell centre: the
 * leaf size S must be a multiple of the order (FMM_ERR_ARG otherwise, and
 * for n != 4 N^3).  Re-tabulates (synchronous). */
int fmm_plan_set_green_mesh(fmm_plan* plan, const double* mesh, size_t n);

/* The plan's Green's function sampled on a mesh, for PM references (Sec. 3:
 * PM and FMM with the same G).  Periodic plans: M = N, entries at offsets
 * d/N, d in [0, N)^3.  Isolated plans: M = 2N, the zero-padded (Hockney)
 * mesh, G_0 at signed offsets k/N with k in [-N, N) stored in FFT order
 * (index k mod 2N).  d = 0 holds the cell self term.  `out` (device,
 * 4 M^3 doubles, written; evaluated in FP64): G, -dG/dx, -dG/dy, -dG/dz,
 * each M^3 with x fastest.  Enqueued on `stream`. */
int fmm_plan_mesh_green(const fmm_plan* plan, double* out, void* stream);

/* How M2L evaluates eq. fmm2 at the fine levels.  FMM_M2L_DENSE (default):
 * the dense contraction per offset (CUDA cores or, in the mixed forms, the
 * tensor cores).  FMM_M2L_FFT: the HPM form of Sec. 2, as an ablation: per
 * parent, the gridlet masses of its neighbours' children on a zero-padded
 * (8 order)^3 grid, one FFT convolution with the level table (cuFFT, FP32),
 * and the 27 near nodes' terms subtracted by direct sums; used at the levels
 * whose local fields are FP32 (the extended-precision coarse levels keep the
 * dense kernels) of periodic plans, whatever the precision mode.  Allocates
 * the FFT plans, buffers and table spectra (synchronous; about 7 parents x
 * (8 order)^3 x 16 bytes per level).  FMM_ERR_ARG for an unknown value. */
#define FMM_M2L_DENSE 0
#define FMM_M2L_FFT   1
int fmm_plan_set_m2l_algorithm(fmm_plan* plan, int algorithm);

/* How the leaf stage evaluates the near zone (Sec. 2, part 3 of the
 * potential).  FMM_NEAR_DIRECT (default): the direct sum over the 27
 * neighbour leaves.  FMM_NEAR_FFT: the same sum by FFT convolution under
 * non-periodic boundary conditions on a doubled grid, the approach Sec. 3
 * takes for the near zone of a regular grid: per pair of neighbour leaves
 * the 8^3 masses zero-padded to 16^3, the 27 x 4 kernel spectra of the near
 * table (FP64, rounded once), FP32 transforms and products; the inverse
 * transforms add the near field to the leaf's L2P far field.  Needs 8-cell
 * leaves (N = 8 * 2^L);
 * FMM_ERR_UNSUPPORTED otherwise.  Allocates the spectra (synchronous;
 * 2^(3L) x 92 KB: 3.0 GB at 256^3, L = 5) and computes the kernel spectra,
 * again after every re-tabulation.  FMM_NEAR_DIRECT frees them.  FMM_ERR_ARG
 * for an unknown value, FMM_ERR_ALLOC if the spectra do not fit. */
#define FMM_NEAR_DIRECT 0
#define FMM_NEAR_FFT    1
int fmm_plan_set_near_algorithm(fmm_plan* plan, int algorithm);

/* Limit of every bounded device-side wait (pipeline barriers of the
 * tensor-core M2L), in milliseconds, 1..600000; default 2000.  A wait that
 * runs out makes its kernel skip the rest of its work, wait (bounded) for the
 * copies and MMAs it already issued, free its tensor memory and return;
 * fmm_plan_check() then reports FMM_ERR_TIMEOUT and the outputs of that solve
 * are not valid. */
int fmm_plan_set_timeout_ms(fmm_plan* plan, int ms);

/* Test hook for the failure path (no GPU fault is involved):
 * FMM_FAULT_TC_STALL makes the tensor-core MMA issuer of later solves do
 * nothing, so the dependent bounded waits expire; FMM_FAULT_NONE clears it. */
#define FMM_FAULT_NONE     0
#define FMM_FAULT_TC_STALL 1
int fmm_plan_inject_fault(fmm_plan* plan, int kind);

/* Tensor-core M2L: number of interaction offsets (1..189) accumulated in one
 * TMEM partial sum before it is added to the compensated FP32 total on the
 * CUDA cores.  Smaller is more accurate, larger is faster; default 2.
 * FMM_ERR_ARG outside 1..189. */
int fmm_plan_set_m2l_group(fmm_plan* plan, int offsets_per_partial);

/* Mixed-precision forms: the first tree level whose M2L (eq. fmm2) runs on
 * the tensor cores; coarser levels run the CUDA-core kernels.  Default and
 * minimum 4 (levels 2 and 3 always use the extended-precision CUDA-core
 * kernels); at order >= 7 the default is level 5 (or the leaf level, if
 * coarser).  A value above the leaf level L keeps every level on the CUDA
 * cores.  At order >= 7 the levels above the leaves keep FP64 local fields
 * (the L2L interpolation to the children extrapolates beyond the parent
 * gridlet: absolute weight sums ~1100 at p = 8) and those on the tensor
 * cores run the bf16x6 mode (fmm_plan_set_precision); a level set here is
 * taken as given, also at order >= 7 (measured on the 512^3 order-8
 * clustered workload, bf16x6 at level 4 costs 6.1e-5 against the FP64
 * oracle, at level 5 2.6e-6).  Lowering the level after the first
 * mixed-precision solve builds the translation tiles of the new levels
 * (synchronously).  FMM_ERR_ARG outside 4..9. */
int fmm_plan_set_tc_min_level(fmm_plan* plan, int level);

/* Tensor-core tile of one level: targets per CTA, 256 (default: an
 * 8 x 8 x 4 box of parents, MMA N = 256) or 128 (8 x 4 x 4, N = 128: twice
 * the CTAs, for levels whose 256-target grid leaves SMs idle).  The results
 * do not depend on it (each target's sums run in the same order).  The bf16x6
 * levels always take 128.  level in 4..L; FMM_ERR_ARG otherwise. */
int fmm_plan_set_tc_tile(fmm_plan* plan, int level, int targets);

/* Autotune the tensor-core tile of every level of the plan's mixed form:
 * times each tensor-core level's M2L with both tiles (stage-timed solves of
 * `density`, one warm-up and the faster of two, enqueued on `stream`; the
 * plan's precision must already be set), keeps the faster per level, and
 * writes the chosen targets per CTA to tiles[l] for l < n (0 for levels not
 * on the tensor cores; n may be 0).  Allocates scratch outputs for its
 * solves (4 N^3 floats) and synchronises.  FMM_ERR_ARG for NULL or
 * misaligned pointers, FMM_ERR_ALLOC, FMM_ERR_CUDA. */
int fmm_plan_autotune_tiles(fmm_plan* plan, const float* density, int* tiles, int n, void* stream);

/* Synchronise the device and read the plan's device error word: FMM_OK, or
 * FMM_ERR_TIMEOUT if a bounded device-side wait of an earlier solve gave up
 * (the word is then cleared).  Solves never block forever. */
int fmm_plan_check(fmm_plan* plan);

/* Query plan parameters: writes N, L, order, S (any pointer may be NULL). */
int fmm_plan_get_shape(const fmm_plan* plan, int* N, int* L, int* order, int* S);

/* ---- per-stage timing --------------------------------------------------- */

#define FMM_TIME_MEAN   0   /* a0 mean density                                   */
#define FMM_TIME_P2M    1   /* a3 leaf gridlet masses                             */
#define FMM_TIME_M2M    2   /* a4 all M2M levels                                  */
#define FMM_TIME_M2L    3   /* a5/a6 all M2L levels                               */
#define FMM_TIME_L2L    4   /* a7 all L2L levels                                  */
#define FMM_TIME_P2P    5   /* a8+a9 fused L2P and near-zone sum                  */
#define FMM_TIME_M2L_LEVEL0 6  /* slot 6 + l: M2L of level l alone (l = 2..8)     */
#define FMM_TIME_SLOTS  16

/* Enable (1) or disable (0) CUDA-event timing of every stage of later solves.
 * Events are recorded on the solve's stream, so they bracket exactly the
 * kernels of each stage.  Plan-owned events; no effect on results. */
int fmm_plan_set_timing(fmm_plan* plan, int enable);

/* Stage durations of the most recent timed solve in milliseconds, indexed by
 * FMM_TIME_*; writes min(n, FMM_TIME_SLOTS) floats (unused slots 0).  Waits for
 * that solve to finish.  FMM_ERR_ARG if timing was never enabled. */
int fmm_plan_stage_times(fmm_plan* plan, float* ms, int n);

/* ---- batches of independent fields ------------------------------------------ */
/* Many periodic fields of uneven size solved together: one plan per field,
 * and every solve of the batch is a single CUDA-graph launch whose parallel
 * branches are the fields (largest first, up to 8 concurrent branches). */
typedef struct fmm_batch fmm_batch;

/* nfields >= 1 fields with mesh sizes N[i], leaf levels L[i] and orders
 * order[i] (each as in fmm_plan_create).  L[i] <= 0 picks the level with
 * fmm_autotune_levels (mixed-precision M2L, cache file from the environment
 * variable FMM_AUTOTUNE_CACHE if set).  Tensor-core precision is off until
 * fmm_batch_set_precision.  NULL on error (fmm_last_error()). */
fmm_batch* fmm_batch_create(int nfields, const int* N, const int* L, const int* order);

/* M2L arithmetic of every field (FMM_PREC_*). */
int fmm_batch_set_precision(fmm_batch* batch, int mode);

/* The near-zone algorithm (FMM_NEAR_DIRECT / FMM_NEAR_FFT, see
 * fmm_plan_set_near_algorithm) of every field of the batch that supports it:
 * with FMM_NEAR_FFT the fields with 8-cell leaves take the FFT form, the
 * others keep the direct sum.  Allocates the fields' spectra (synchronous)
 * and drops the captured graph (the next solve captures again).  FMM_ERR_ARG
 * for an unknown value, FMM_ERR_ALLOC if the spectra do not fit. */
int fmm_batch_set_near_algorithm(fmm_batch* batch, int algorithm);

/* The leaf level chosen for each field (nfields ints). */
int fmm_batch_get_levels(const fmm_batch* batch, int* L);

/* Solve every field: host arrays of nfields device pointers (each as in
 * fmm_solve).  The first call with a given set of pointers captures the
 * fields' kernels into one graph (later calls with the same pointers only
 * launch it).  Enqueued on `stream`. */
int fmm_batch_solve(fmm_batch* batch, const float* const* density, float* const* potential,
                    float* const* accel, void* stream);

/* fmm_plan_check over every field. */
int fmm_batch_check(fmm_batch* batch);

/* Release the batch (NULL allowed); synchronises the device first. */
void fmm_batch_destroy(fmm_batch* batch);

/* Autotuner: the leaf level L (S = N / 2^L in {2, 3, 4, 6, 8}, L >= 3 when
 * possible) with the shortest solve of a synthetic N^3 field at this order
 * and precision, timed with CUDA events (median of 3).  Results are cached
 * per GPU model as JSON lines in `cache_path` (NULL: no cache).  Writes L and
 * (if not NULL) its time in ms.  Allocates temporary device memory. */
int fmm_autotune_levels(int N, int order, int precision, const char* cache_path, int* L_out, float* ms_out);

/* ---- learned table correction ------------------------------------------- */
/* Sec. 4 proposes parameterising the optimal Green's function G_* by many
 * parameters instead of the analytic G_S1.  Here a small MLP
 * (5 -> 64 -> 64 -> 64 -> 1, GELU) adds a learned correction to every M2L
 * table entry; the near zone keeps the exact G_S1 (it must match PM).
 * Inputs: the entry's offset in gridlet units (absolute values, sorted so
 * the cube symmetry holds), the level and the field class (G or a gradient
 * component, the latter times the sign of its own offset component); the
 * output is scaled by the entry's natural size at that level.  Parameter
 * layout (FP32): W1[64][5] b1[64] W2[64][64] b2[64] W3[64][64] b3[64] W4[64]
 * b4[1], FMM_MLP_PARAMS floats. */
#define FMM_MLP_PARAMS 8769
#define FMM_INFER_BF16 0      /* weights and activations rounded to BF16, FP32 accumulate */
#define FMM_INFER_FP32 1

/* Set (weights = device or host pointer to FMM_MLP_PARAMS floats, copied) or
 * clear (weights = NULL) the correction and re-tabulate every M2L table form
 * (synchronous).  FMM_ERR_ARG if n != FMM_MLP_PARAMS. */
int fmm_plan_set_correction(fmm_plan* plan, const float* weights, size_t n);

/* Inference arithmetic of the correction at the next fmm_plan_set_correction:
 * FMM_INFER_BF16 (default) or FMM_INFER_FP32 (used for training). */
int fmm_plan_set_correction_inference(fmm_plan* plan, int mode);

/* One training field: solve `density` (device, N^3) with the current
 * correction, compare with the target solution (device, N^3 potential and
 * 3 N^3 acceleration), and ADD to `grad` (device, FMM_MLP_PARAMS floats) the
 * gradient of J = w_phi |Phi - Phi*|^2 + w_g |g - g*|^2 with respect to the
 * correction's parameters, and J itself to `loss` (device, 1 float).  The
 * gradient runs through the adjoint of L2P and L2L, the table gradient of
 * eq. fmm2 and the MLP's backward pass, all on the GPU.  Requires a
 * correction to be set (FMM_ERR_ARG otherwise).  Enqueued on `stream`. */
int fmm_correction_grad(fmm_plan* plan, const float* density, const float* target_phi, const float* target_acc,
                        float w_phi, float w_g, float* grad, float* loss, void* stream);

/* One Adam update of n parameters (device arrays; m, v are the moment
 * estimates, step >= 1 the update count for bias correction). */
int fmm_adam_step(float* weights, const float* grad, float* m, float* v, size_t n, int step, float lr, float beta1,
                  float beta2, float eps, void* stream);

/* G_S1 and -grad G_S1 at the periodic mesh offsets d/N, d in [0, N)^3, with
 * the cell self term at d = 0: `out` (device) = 4 planes of N^3 floats in
 * [z][y][x] order (G, -dG/dx, -dG/dy, -dG/dz).  The kernel of the PM solution
 * with the same Green's function (Sec. 3 eq. pmconv). */
int fmm_mesh_green(int N, float* out, void* stream);

/* ---- errors --------------------------------------------------------- */
int fmm_last_error(void);
const char* fmm_error_string(int code);

/* ---- stage access (tests and diagnostics) ----------------------------- */

#define FMM_STAGE_MULTIPOLE 0   /* gridlet masses of `level`: 8^level x order^3  */
#define FMM_STAGE_LOCAL     1   /* local field of `level` after M2L and L2L:
                                   8^level x 4 x order^3 (Phi, gx, gy, gz)      */
#define FMM_STAGE_MEAN      2   /* mean density, 1 value (converted to float)    */

/* Copy an internal stage buffer of the last solve into `dst` (device memory,
 * `count` floats).  Node order is Morton: key = interleave(x, y, z) bits with
 * x in the lowest bit.  Per node, values are [field][sz][sy][sx].  Enqueued on
 * `stream`.  FMM_ERR_ARG if `count` is smaller than the stage. */
int fmm_plan_copy_stage(fmm_plan* plan, int stage, int level, float* dst,
                        size_t count, void* stream);

/* ---- error of a result against PM ---------------------------------------- */

/* Relative L2 error of a solution against the PM solution with the same
 * Green's function, over sampled cells.  Sec. 3 defines the optimal G_* as
 * the function with which PM and FMM give the same potential; PM is the
 * periodic convolution of the masses m = (rho - mean rho) / N^3 with G_S1
 * sampled at the mesh offsets d/N (eq. pmconv), and with the plan's self
 * term G(0) at d = 0.  At each sampled cell that convolution is evaluated
 * exactly, as a direct sum over all N^3 source cells (per-pair G_S1 in FP32,
 * sums in FP64: about 1e-7 relative), and compared with the given values.
 * The reference is always the plain G_S1, whatever precision mode or
 * learned correction the plan has, so that every form's error is stated
 * against the same target.
 *   plan        the plan (its N; its mean scratch is overwritten).
 *   density     device, N^3 floats, [z][y][x] (x fastest), read only.
 *   potential   device, N^3 floats, the result to assess.
 *   accel       device, 3 N^3 floats (SoA ax | ay | az), the result to assess.
 *   samples     1 .. 1024 target cells: the first `samples` outputs of
 *               splitmix64 seeded with `seed`, each modulo N^3 (a cell index
 *               x + N (y + N z); drawn with replacement).
 *   seed        generator seed.
 *   out         host, 2 doubles, written: out[0] = ||dPhi|| / ||Phi_PM||,
 *               out[1] = ||dg|| / ||g_PM|| (all three components) over the
 *               sampled cells.
 *   stream      cudaStream_t as void*.  The call is synchronous: it returns
 *               after the work it enqueued on `stream` has finished.
 * Cost: samples x N^3 pair evaluations (on one GB300 0.14 s for 512 samples
 * at 256^3, 0.27 s for 1024); scratch of up to 10 MB is allocated and freed
 * by the call; the statement's density mean goes to that scratch too, so
 * the plan's mean stage (FMM_STAGE_MEAN) still holds the last solve's.  Do
 * not run it concurrently with a solve of the same plan.
 * Returns FMM_OK, FMM_ERR_ARG (NULL or misaligned pointers, samples out of
 * range), FMM_ERR_ALLOC or FMM_ERR_CUDA. */
int fmm_plan_error_stats(fmm_plan* plan, const float* density, const float* potential,
                         const float* accel, int samples, unsigned long long seed,
                         double* out, void* stream);

/* ---- grid model of G_* --------------------------------------------------- */
/* Sec. 4's other proposal: parameterise G_* as a grid of values, every value
 * its own parameter.  Here each level l = 2..L carries one free value per
 * folded table entry and field: theta[l - 2][f][az][ay][ax] with a_i in
 * [0, 4p) (the (4 N_g)^3 samples Sec. 4 counts), f = 0 for G and 1..3 for
 * -dG/dx, -dG/dy, -dG/dz.  The M2L table entry at offset n (gridlet units,
 * taken to its nearest periodic image) becomes G_S1 + theta[0][|n|] for G
 * and -dG/dx_i + sign(n_i) theta[i][|n|] for the gradients (sign 0 at half
 * the box), so the table keeps the parity and periodicity of G_S1 and the
 * solve keeps zero net force.  The near zone keeps the exact G_S1.  The
 * grid adds to the MLP correction when both are set. */

/* Number of grid parameters of the plan: (L - 1) x 4 x (4 order)^3. */
int fmm_plan_table_grid_size(const fmm_plan* plan, size_t* n);

/* Set (theta = device or host pointer to fmm_plan_table_grid_size floats,
 * copied) or clear (theta = NULL) the grid and re-tabulate every M2L table
 * form (synchronous).  FMM_ERR_ARG if n is not the plan's grid size. */
int fmm_plan_set_table_grid(fmm_plan* plan, const float* theta, size_t n);

/* One training field for the grid model: solve `density` with the current
 * tables, compare with the target solution (device, N^3 potential and 3 N^3
 * acceleration) and ADD to `grad` (device, grid-size floats) the gradient of
 * J = w_phi |Phi - Phi*|^2 + w_g |g - g*|^2 with respect to theta, and J to
 * `loss` (device, 1 float): the adjoint of L2P and L2L, the table gradient
 * of eq. fmm2 and its fold onto the grid entries, all on the GPU.  Enqueued
 * on `stream`.  A grid need not be set (the gradient is then taken at
 * theta = 0). */
int fmm_table_grid_grad(fmm_plan* plan, const float* density, const float* target_phi, const float* target_acc,
                        float w_phi, float w_g, float* grad, float* loss, void* stream);

/* ---- measurement aid ----------------------------------------------------- */

/* FP32 FMA throughput probe; the paper has no counterpart.  Enqueues on
 * `stream` one kernel of `blocks` CTAs x 1024 threads, each thread running 8
 * independent chains of iters x 16 dependent FMAs, and stores one float per
 * CTA to `out` (device, `blocks` floats).  fmm_probe_fma_flops(blocks, iters)
 * returns the flops one launch performs (2 per FMA), so a caller that times
 * the launch with CUDA events measures the FP32 CUDA-core peak, the roofline
 * of the FMA-bound steps (the near-zone sum, CUDA-core M2L).  FMM_ERR_ARG for a NULL
 * pointer or counts < 1. */
int fmm_probe_fma(float* out, int blocks, int iters, void* stream);
double fmm_probe_fma_flops(int blocks, int iters);

/* ---- allocation-free entry point ----------------------------------------- */

/* Mean of a device float array, without any allocation by the library.  The
 * paper has no counterpart: this is a service for callers that cannot let a
 * library call cudaMalloc / cudaFree (embedders whose own allocator owns all
 * device memory; host loops that must not take the device-wide
 * synchronisation those calls may cause).  It computes the same FP64 mean of
 * the density as the first step of fmm_solve.
 *   density  device, `count` floats, read only.
 *   count    1 .. 134217728 (= 512^3); larger counts return FMM_ERR_ARG.
 *   mean     device, one double, written.
 *   stream   cudaStream_t as void* (NULL = legacy default stream); the call
 *            only enqueues work.
 * Scratch: a file-scope static device array of 16384 doubles (128 KB) that
 * every GPU which loads this library holds until the process exits.  Every
 * call on a device shares it and it keeps the last call's contents (each call
 * overwrites the slots it reads), so calls whose work overlaps on the GPU
 * (different streams, or different host threads on one device) race and must
 * be serialised by the caller.  The first call on each device looks up the
 * array's device address with that device current (a one-time set-up); make
 * that first call before any stream capture.  Host threads may make their
 * first calls concurrently: the looked-up address is published atomically.
 * Returns FMM_OK, FMM_ERR_ARG (NULL pointers, count 0 or above the maximum),
 * FMM_ERR_UNSUPPORTED (device ordinal >= 64) or FMM_ERR_CUDA. */
int fmm_mean_density_noalloc(const float* density, size_t count, double* mean, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FMM_H */
