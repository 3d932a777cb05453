/*
 * blockoa.h -- C ABI of libblockoa.so, the GB300 (sm_103a) hot path of
 * BlocKOA: block Krylov basis solve, combination, operator action.
 *
 * Paper: "Accelerating IC Thermal Simulation Data Generation via Block
 * Krylov and Operator Action" (arXiv 2510.23221).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Unknowns are excess temperature theta = T - t_ambient in K; rows of the
 *   operator are in W/K; right-hand sides are cell powers in W.
 * - Cells of one chip are numbered a = (z * ny + y) * nx + x, z = 0 is the
 *   top (silicon) layer.  Several chips are concatenated chip after chip;
 *   blockoa_operator_size() gives each chip's cell offset.
 * - Block vectors (B, X, U) are cell-major with the s columns fastest:
 *   element (cell a of chip c, column j) sits at [(off_c + a) * s + j].
 * - Fields (T, q) are field-major per chip: element (field m, cell a of
 *   chip c) sits at [off_c * M + m * n_c + a].
 * - Coefficients C are [chip][s][M] row-major, float64 values that are
 *   exactly representable in bfloat16 when the MIXED path is used.
 * - Every pointer named "device" is a CUDA device pointer owned by the
 *   caller; the library never frees or reallocates it.  Pointers named
 *   "host" are ordinary host memory.  The operator object is owned by the
 *   library and holds its own device workspace until blockoa_destroy().
 * - Calls are asynchronous on `stream` unless stated otherwise.
 * - Every call returns a blockoa_status; nothing crosses the ABI as an
 *   exception and the library never exits the process.  On error, outputs
 *   are unspecified but statistics structures are filled in.
 */
#ifndef BLOCKOA_H
#define BLOCKOA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st *blockoa_stream;

typedef enum {
  BLOCKOA_OK = 0,
  BLOCKOA_ERR_INVALID = 1,        /* bad argument, checked on the host before any launch */
  BLOCKOA_ERR_CUDA = 2,           /* a CUDA runtime call failed */
  BLOCKOA_ERR_BREAKDOWN = 3,      /* NaN/Inf, or Gram matrix of rank 0 with columns unconverged */
  BLOCKOA_ERR_NOT_CONVERGED = 4,  /* iteration limit reached before every column met rtol */
  BLOCKOA_ERR_TIMEOUT = 5,        /* a bounded device wait gave up */
  BLOCKOA_ERR_OOM = 6             /* device allocation failed */
} blockoa_status;

/* Arithmetic of a call. */
typedef enum {
  BLOCKOA_FP64 = 0,   /* every step in float64 */
  BLOCKOA_MIXED = 1   /* float32 vectors and stencil, float64 Gram/Cholesky and
                         refinement, bfloat16x3 tensor-core combination */
} blockoa_precision;

/*
 * One layered chip (Sec. V-A; the steady heat equation of Eq. 1 on a
 * rectangular prism with the Robin condition of Sec. II-A).
 * All pointers are host pointers read during blockoa_assemble() only.
 */
typedef struct {
  int nx, ny;                 /* lateral cells, >= 1 */
  int n_layers;               /* >= 1 */
  const int *layer_nz;        /* [n_layers] cells per layer along z, >= 1 */
  const double *layer_dz;     /* [n_layers] thickness of one cell of the layer, m, > 0 */
  const double *layer_k;      /* [n_layers] conductivity, W/m/K, > 0; ignored if k_cell != NULL */
  const double *k_cell;       /* optional [nz][ny][nx] per-cell conductivity, W/m/K */
  double dx, dy;              /* lateral cell size, m, > 0 */
  double h_top, h_bottom, h_side; /* convective coefficients, W/m^2/K; 0 = adiabatic;
                                     * +INFINITY = Dirichlet face held at t_ambient
                                     * (theta = 0 on the face: Gb = 2 k A / d, the
                                     * half-cell conductance to the face) */
  double t_ambient;           /* K; reporting only (unknowns are excess temperature) */
} blockoa_chip_desc;

typedef struct {
  double rtol;          /* per-column ||B_j - A X_j|| / ||B_j|| target, > 0 */
  int maxiter;          /* limit on block iterations (summed over refinement steps) */
  int precision;        /* blockoa_precision */
  double inner_rtol;    /* MIXED: residual reduction asked of each float32 inner solve (<= 0: 1e-4) */
  int max_refine;       /* MIXED: limit on float64 refinement steps (<= 0: 12) */
  double deflate_tol;   /* pivot threshold on the scaled Gram (<= 0: 1e-14 FP64, 1e-6 float32 inner) */
  const double *x0;     /* device [n_total][s] initial guess, or NULL for zero */
  int check_every;      /* block iterations between convergence polls by the host (<= 0: 8) */
  int precond;          /* BLOCKOA_PRECOND_NONE (the paper's unpreconditioned block CG),
                           BLOCKOA_PRECOND_JACOBI (diagonal: directions from D^-1 R) or
                           BLOCKOA_PRECOND_ZLINE (z-line: directions from M^-1 R, M the
                           tridiagonal coupling of each (x, y) cell column) or
                           BLOCKOA_PRECOND_ZLINE2 (two-step z-line: directions from
                           M^-1 (2 R - A M^-1 R), the polynomial 2 - x of M^-1 A on
                           M^-1 R; symmetric positive definite because the z-line
                           splitting puts the spectrum of M^-1 A in (0, 2)).  Both
                           z-line forms need nz <= the block tile's cells. */
  int small_solve;      /* BLOCKOA_SMALL_AUTO or BLOCKOA_SMALL_FP64_CHOLESKY (below) */
  int independent;      /* 0: block CG (the s columns share one Krylov space);
                           1: the s columns iterate as s independent (single
                           right-hand side) CG solves -- the per-sample "direct"
                           baseline: every off-diagonal entry of Gamma, P^T R and
                           Q^T Z is dropped, so alpha_jj = (p_j . r_j) / (p_j . A p_j)
                           and beta_jj = -(A p_j . z_j) / (p_j . A p_j) */
  int deterministic;    /* 0: the loop kernels' partial sums reach the float64
                           accumulators by atomics in whatever order the CTAs
                           finish (results can differ in the last bits, and the
                           iteration count by a few, from run to run);
                           1: bitwise reproducible on a given GPU and operator --
                           static unit schedules, every partial sum stored and
                           reduced in a fixed order (the stencil pass, the
                           update, the second z-line step, ||B_j||^2 and the
                           float64 residual), float64 Cholesky small solves;
                           two or three more kernel launches per iteration */
} blockoa_solve_opts;

enum { BLOCKOA_PRECOND_NONE = 0, BLOCKOA_PRECOND_JACOBI = 1, BLOCKOA_PRECOND_ZLINE = 2,
       BLOCKOA_PRECOND_ZLINE2 = 3 };

/*
 * How the s x s systems Gamma alpha = rho and Gamma beta = -W are solved:
 *  BLOCKOA_SMALL_AUTO: FP64 form: float64 diagonal-pivoted Cholesky and
 *    substitution in kernels of their own.  MIXED form: in the last CTA per
 *    chip of the Gram kernels, by the symmetric sweep operator (Gauss-Jordan
 *    with the pivots and deflation test of the pivoted Cholesky) in
 *    double-float arithmetic (~48-bit significand, ~2^-44 relative), which
 *    leaves G_KK^-1 so that alpha and beta are plain s x s products.
 *  BLOCKOA_SMALL_FP64_CHOLESKY: float64 pivoted Cholesky and substitution
 *    in kernels of their own for both forms.
 */
enum { BLOCKOA_SMALL_AUTO = 0, BLOCKOA_SMALL_FP64_CHOLESKY = 1 };

typedef struct {
  int status;           /* blockoa_status of this chip */
  int iters;            /* block iterations (summed over refinement steps) */
  int refine_steps;     /* float64 true-residual evaluations after the start */
  int deflated_cols;    /* columns dropped by deflation, summed over iterations */
  double relres_max;    /* max_j ||B_j - A X_j|| / ||B_j|| from a float64 true residual */
} blockoa_solve_stats;

typedef struct blockoa_operator blockoa_operator;

/*
 * Discretise n_chips chips (Eq. 1 -> Eq. 2; Sec. II-B) with a cell-centred
 * 7-point finite-volume stencil in flux form:
 *   (A theta)_a = sum_b G_ab (theta_a - theta_b) + Gb_a theta_a,
 *   G_ab = S_f / (d_a/(2 k_a) + d_b/(2 k_b)),  Gb = S_f / (d/(2k) + 1/h).
 * Face conductances are computed on the device in float64 (and rounded to
 * float32 copies).  `chips` is a host array read before return.
 * On success *out receives a new operator (free with blockoa_destroy).
 * Errors: ERR_INVALID (bad descriptor), ERR_OOM, ERR_CUDA.
 */
int blockoa_assemble(const blockoa_chip_desc *chips, int n_chips, blockoa_stream stream,
                     blockoa_operator **out);

/*
 * Re-discretise an existing operator in place (Eq. 1 -> Eq. 2, same stencil
 * and arithmetic as blockoa_assemble) for chips of the same geometry: the
 * same chip count and, per chip, the same nx, ny and layer rows (layer
 * thicknesses, conductivities, cell sizes and film coefficients may
 * change).  The operator's arrays, its solve workspace and its captured
 * block-CG graph are kept, so a stream of same-shaped chips costs no
 * allocation or graph build.  Stream-ordered: work already queued on the
 * operator must be on `stream` or complete.
 * Errors: ERR_INVALID (bad descriptor or different geometry; the operator
 * is unchanged), ERR_OOM, ERR_CUDA.
 */
int blockoa_reassemble(blockoa_operator *op, const blockoa_chip_desc *chips, int n_chips,
                       blockoa_stream stream);

/* Sizes of chip `chip` (host outputs, any may be NULL).  Synchronous. */
int blockoa_operator_size(const blockoa_operator *op, int chip, int64_t *n_cells,
                          int64_t *cell_offset, int *nx, int *ny, int *nz);

/* Total cells over all chips and number of chips (host outputs). */
int blockoa_operator_total(const blockoa_operator *op, int64_t *n_total, int *n_chips);

/*
 * Right-hand sides b of Eq. 2: cell power = density * dx * dy in the top
 * cell row (z = 0), zero elsewhere.
 * density: device float64 [chip][s][ny][nx] (W/m^2), chips concatenated.
 * B: device float64 block vector [n_total][s] (written in full).
 */
int blockoa_build_rhs(const blockoa_operator *op, const double *density, double *B, int s,
                      blockoa_stream stream);

/*
 * Right-hand sides b of Eq. 2 from a volumetric heat source q (the q of
 * Eq. 1, per unit volume), for sources anywhere in the stack -- e.g. the
 * core and cache device layers of a 3-D IC (Sec. V-A):
 * b_j(a) = qv_j(a) * dx * dy * dz(a), dz(a) the thickness of cell a's layer
 * (the volume dx dy dz is formed first, then the product, in float64).
 * qv: device float64 [chip][s][nz][ny][nx] (W/m^3), chips concatenated;
 *     owned by the caller, only read.
 * B: device float64 block vector [n_total][s] (written in full).
 * Asynchronous on `stream`.  s = 0 is a no-op.
 * Errors: ERR_INVALID (op NULL, s < 0, qv or B NULL with s > 0), ERR_OOM,
 * ERR_CUDA.
 */
int blockoa_build_rhs_volume(const blockoa_operator *op, const double *qv, double *B, int s,
                             blockoa_stream stream);

/*
 * Block conjugate gradient on A_c X_c = B_c for every chip c at once
 * (Eq. 3-4, Sec. III-A): all s columns of a chip share one Krylov space.
 * Each iteration: Q = A P; Gamma = P^T Q; Jacobi-scaled pivoted Cholesky of
 * Gamma with deflation of pivots <= deflate_tol; alpha = Gamma^-1 P^T R;
 * X += P alpha; R -= Q alpha; beta = -Gamma^-1 Q^T R; P = R + P beta.
 * With BLOCKOA_PRECOND_JACOBI, Z = D^-1 R (D = diag(A)) replaces R in the
 * new directions: beta = -Gamma^-1 Q^T Z, P = Z + P beta (same solution);
 * with BLOCKOA_PRECOND_ZLINE, Z = M^-1 R with M the part of A that couples
 * the cells of one (x, y) column (solved by the Thomas recurrences per
 * column); it needs every chip's nz <= the solver's tile (64 cells for
 * s > 32, more for smaller s) and returns ERR_INVALID otherwise.
 * MIXED runs that loop in float32 (Gram products accumulated to float64)
 * inside float64 iterative refinement on the true residual B - A X.
 * Stops when every column meets ||B_j - A X_j|| <= rtol ||B_j||.
 * B, X: device float64 [n_total][s]; 1 <= s <= 64.  X is overwritten.
 * stats: host array [n_chips], always written.
 * Synchronous: returns after the solve, because it fills `stats`.
 * Errors: ERR_INVALID, ERR_NOT_CONVERGED, ERR_BREAKDOWN, ERR_OOM, ERR_CUDA
 * (the worst chip status is returned).
 */
int blockoa_block_solve(blockoa_operator *op, const double *B, double *X, int s,
                        const blockoa_solve_opts *opts, blockoa_solve_stats *stats,
                        blockoa_stream stream);

/*
 * Test support (no counterpart in the paper): arm a one-shot injection for
 * the next blockoa_block_solve on this operator.  Before the convergence
 * poll number after_polls (0 = before the first block of iterations) of
 * the first inner solve, chip `chip`'s device state is overwritten with
 * `status` and marked inactive -- the state a bounded device-side wait
 * leaves when it gives up (status ERR_TIMEOUT) -- so that the propagation
 * of such a status can be exercised without faulting or hanging a GPU.
 * The other chips are unaffected.  Errors: ERR_INVALID (chip out of range,
 * status not an error code, negative after_polls).
 */
int blockoa_inject_chip_status(blockoa_operator *op, int chip, int status, int after_polls);

/*
 * Launch tuning of the batched block-CG loop (the persistent launches of
 * blockoa_block_solve): work units are tiles_per_unit block tiles of one
 * chip for the loop kernels, and ztiles_per_unit column tiles for the
 * z-line kernels; 0 lets the library derive the size from the tile count.
 */
typedef struct {
  int tiles_per_unit;
  int ztiles_per_unit;
  double ms_per_iter;   /* blockoa_autotune: measured time of one block iteration */
} blockoa_tuning;

/*
 * Autotune the unit sizes of this operator for s columns in the given
 * precision and preconditioner form: for each candidate (1, 2, 4, 8, 16, 32
 * tiles; then, for the z-line forms, 1-32 column tiles) it times block
 * iterations of a solve on synthetic right-hand sides (the difference of a
 * 24- and an 8-iteration run, so set-up and refinement cancel), keeps the
 * fastest in the operator for later solves and reports it.  Synchronous;
 * uses the library's device pool for its right-hand sides.
 * Errors: ERR_INVALID, ERR_OOM, ERR_CUDA.
 */
int blockoa_autotune(blockoa_operator *op, int s, int precision, int precond, blockoa_tuning *out,
                     blockoa_stream stream);

/* Set (0 = derive from the tile count) or read the operator's unit sizes;
 * ms_per_iter is ignored / returned as 0.  Errors: ERR_INVALID (sizes
 * outside 0..64). */
int blockoa_set_tuning(blockoa_operator *op, const blockoa_tuning *t);
int blockoa_get_tuning(const blockoa_operator *op, blockoa_tuning *t);

/*
 * New temperature fields T = U C (Eq. 5, Sec. III-B, with the noise term
 * off and no normalisation: unknowns are excess temperatures, so every
 * combination keeps the homogeneous Robin/adiabatic conditions).
 * U: device float64 [n_total][s]; C: device float64 [chip][s][M].
 * T: device fields [chip][M][n_c], float64 for FP64, float32 for MIXED.
 * MIXED splits U into three bfloat16 planes and multiplies on the tensor
 * cores (tcgen05) with float32 accumulation; C must be bfloat16-exact.
 */
int blockoa_combine(blockoa_operator *op, const double *U, const double *C, void *T, int s,
                    int M, int dtype, blockoa_stream stream);

/*
 * Options of blockoa_combine_ex: the noise term epsilon and the normalised
 * weights of Eq. 5 (Sec. III-B).
 *
 * Noise.  BLOCKOA_NOISE_UNIFORM with noise_amp > 0 adds to every field value
 *   noise_amp * (2 u - 1),  u = (w >> 11) * 2^-53 in [0, 1),
 * w = word (m % 4) of Philox4x64-10 (Salmon et al., SC 2011) with counter
 * (a, m / 4, 0, 0) and key (noise_seed, 0), a the cell's index in the
 * operator's concatenated numbering: a uniform perturbation in
 * [-noise_amp, noise_amp) K that any kernel can reproduce.  MIXED (float32
 * fields) takes u from the top 24 bits of w, u = (w >> 40) * 2^-24, in
 * float32 (within noise_amp * 2^-23 of the float64 value).
 * BLOCKOA_NOISE_GAUSSIAN adds zero-mean Gaussian noise of standard
 * deviation noise_amp (the Gaussian noise of the noise study, Sec. V-D) by
 * Box-Muller (1958): words w1 = 2 (m % 2) and w2 = 2 (m % 2) + 1 of
 * Philox4x64-10 at counter (a, m / 2, 1, 0), key (noise_seed, 0), give
 * u1 = ((w1 >> 11) + 1/2) 2^-53, u2 = (w2 >> 11) 2^-53 and
 * epsilon = noise_amp sqrt(-2 ln u1) cos(2 pi u2); float32 fields evaluate
 * it in float32 from u1, u2 rounded once to float32.
 * Either way the operator action of the stored (noisy) T stays exact, so
 * pairs (T, A T) remain consistent.
 *
 * Normalised weights.  normalize = 1 combines with Eq. 5's weights
 * alpha_jm = C_jm / sum_i C_im (each field's weights sum to one), evaluated
 * as (U C)_m / sum_i C_im, with noise (if any) added afterwards.  Fields are
 * still excess temperatures: since the weights sum to one, the absolute
 * field is t_ambient + T_m, which keeps every boundary condition of the
 * basis (Robin ambient, held faces).  A field whose weights nearly cancel,
 * |sum_i C_im| <= normalize_min * sum_i |C_im| (normalize_min <= 0: 1e-6),
 * makes the call return ERR_INVALID (blockoa_last_error() says so); the
 * check synchronises the stream.
 */
typedef struct {
  uint64_t noise_seed;  /* Philox key word 0 */
  double noise_amp;     /* K, >= 0; 0 = no noise (half-width, or standard deviation) */
  int noise_kind;       /* BLOCKOA_NOISE_UNIFORM or BLOCKOA_NOISE_GAUSSIAN */
  int normalize;        /* 0: weights C as given; 1: Eq. 5's normalised weights */
  double normalize_min; /* guard on |sum_i C_im| / sum_i |C_im|; <= 0: 1e-6; < 1 */
} blockoa_combine_opts;

enum { BLOCKOA_NOISE_UNIFORM = 0, BLOCKOA_NOISE_GAUSSIAN = 1 };

/*
 * blockoa_combine with options (NULL opts: no noise, weights as given, same
 * as blockoa_combine).  Errors: as blockoa_combine, and ERR_INVALID for a
 * negative or non-finite noise_amp, an unknown noise_kind or normalize
 * value, normalize_min >= 1, or (normalize = 1) a field whose weights sum
 * to ~0.
 */
int blockoa_combine_ex(blockoa_operator *op, const double *U, const double *C, void *T, int s,
                       int M, int dtype, const blockoa_combine_opts *opts, blockoa_stream stream);

/*
 * The combination and the operator action in one pass (Eq. 5 then Eq. 6,
 * Sec. III-B/C, MIXED arithmetic): T = U C as blockoa_combine computes it
 * (bfloat16x3 on the tensor cores, float32 fields, C bfloat16-exact) and
 * q = A T from the same on-chip values, so T is never read back: for each
 * x-row of a chip the kernel also forms the four rows the 7-point stencil
 * reaches, y -+ 1 and z -+ 1, on the tensor cores.  T is bitwise the field
 * blockoa_combine stores; q differs from blockoa_apply_operator on that T
 * by float32 rounding order only.  Covers chips with nx <= 128 and s <= 32;
 * otherwise it runs blockoa_combine and blockoa_apply_operator in turn.
 * No noise or normalised weights (use the separate calls for those).
 * Measured slower than the two separate calls on a 128 x 128 x 8 chip with
 * s = 32 (2.2 ms against 1.6 ms for 5000 fields on one GB300).
 * U: device float64 [n_total][s]; C: device float64 [chip][s][M]; T, q:
 * device float32 fields [chip][M][n_c], not overlapping.  Synchronises the
 * stream (reads a timeout flag).  Errors: ERR_INVALID, ERR_OOM, ERR_CUDA,
 * ERR_TIMEOUT (a bounded wait gave up).
 */
int blockoa_combine_apply(blockoa_operator *op, const double *U, const double *C, float *T, float *q, int s,
                          int M, blockoa_stream stream);

/*
 * Operator action on the basis, AU = A U (Eq. 6 applied to the s basis
 * columns), float64.  U, AU: device float64 [n_total][s], cell-major like
 * blockoa_block_solve's X; they must not overlap.  By linearity
 * A (U C) = (A U) C, so blockoa_combine(op, AU, C, q, ...) yields the
 * operator action of T = U C carrying only the combination's rounding:
 * with float32 fields it is within ~1e-7 of A applied to the exact U C,
 * where blockoa_apply_operator on a float32 T inherits T's storage error
 * amplified by A (the q of the pair (T, q) -- consistent with the stored
 * T -- comes from blockoa_apply_operator).
 * Errors: ERR_INVALID (s < 1 or s > 4096, NULL pointers), ERR_OOM, ERR_CUDA.
 */
int blockoa_apply_basis(const blockoa_operator *op, const double *U, double *AU, int s,
                        blockoa_stream stream);

/*
 * Relative residual of a candidate solution of A X = B, per chip and column:
 * ratio[c * s + j] = ||B_j - A_c X_j|| / ||B_j|| (float64 operator action in
 * difference form, float64 sums; 0 for a zero column of B with a zero
 * residual, +inf for a zero column with a nonzero residual).  This is the
 * learned warm start's fallback test: block CG starts from X only if every
 * ratio of the chip is below the threshold.  B, X: device float64
 * [n_total][s]; ratio: device float64 [n_chips * s].  1 <= s <= 64.
 * Errors: ERR_INVALID (NULL pointers, s out of range), ERR_OOM, ERR_CUDA.
 */
int blockoa_residual_ratio(const blockoa_operator *op, const double *B, const double *X, int s,
                           double *ratio, blockoa_stream stream);

/*
 * Operator action q = A T (Eq. 6, Sec. III-C) on M fields of every chip.
 * T, q: device fields [chip][M][n_c]; float64 for FP64, float32 for MIXED.
 * T and q must not overlap.
 */
int blockoa_apply_operator(const blockoa_operator *op, const void *T, void *q, int M,
                           int dtype, blockoa_stream stream);

/*
 * Pair consistency of generated data (Sec. IV-B: the operator action adds
 * no solver error): e_pair[c*M + m] = ||A T_m - q_m|| / ||q_m|| with A
 * applied in float64 to the stored field T_m.
 * T, q: device fields as in blockoa_apply_operator (dtype selects float64
 * or float32 storage); e_pair: device float64 [n_chips * M].
 */
int blockoa_pair_check(const blockoa_operator *op, const void *T, const void *q, int M,
                       int dtype, double *e_pair, blockoa_stream stream);

/* Largest n_chips * M accepted by blockoa_pair_check_static. */
#define BLOCKOA_STATIC_PAIR_MAX 32768

/*
 * blockoa_pair_check without any device allocation.  The paper has no
 * counterpart.  blockoa_pair_check takes a small accumulator and a launch
 * table from the library's device pool on every call; this variant is for
 * callers that cannot allocate while they run: serving processes whose
 * device memory is reserved up front by their own pool (a stray allocation
 * competes with that budget and can fail or fragment it), deployments with
 * a fixed memory budget that forbid allocation after start-up, and loops
 * that must not stall on cudaMalloc / cudaFree, which can synchronise the
 * device.  Same arguments, layout and result as blockoa_pair_check.
 * Its accumulators live in a fixed library-owned device array of
 * 2 * BLOCKOA_STATIC_PAIR_MAX float64 values (512 KB on every GPU that
 * loads the library, held until the process exits); n_chips * M above
 * BLOCKOA_STATIC_PAIR_MAX returns ERR_INVALID before anything is launched
 * (blockoa_last_error() says why).  The first call on a device looks up
 * that array's device address (once per device, with that device
 * current).  All calls
 * on a device share the array, which keeps the last call's contents; each
 * call clears it on its stream first, so calls that overlap on the GPU
 * (different streams, or concurrent host threads) race and must be
 * serialised by the caller.
 */
int blockoa_pair_check_static(const blockoa_operator *op, const void *T, const void *q, int M,
                              int dtype, double *e_pair, blockoa_stream stream);

/*
 * Copy chip `chip`'s float64 face conductances to host arrays laid out like
 * the oracle's: gx [nz][ny][nx-1], gy [nz][ny-1][nx], gz [nz-1][ny][nx],
 * gb [nz][ny][nx] (any pointer may be NULL).  Synchronous.  For tests.
 */
int blockoa_export_conductances(const blockoa_operator *op, int chip, double *gx, double *gy,
                                double *gz, double *gb);

/*
 * Live per-kernel timing (tracing; no counterpart in the paper).  CUDA
 * events are recorded on the launching stream around the kernels of the
 * first block-CG iteration of every convergence poll (external event-record
 * nodes inside the captured graph), and around every float64 residual,
 * combination and operator-action launch.  Writes, for the first
 * max_kernels kernel classes (host arrays, any may be NULL): the summed
 * milliseconds of the timed launches, the number of timed launches, the
 * number of all launches, and a static name.  Returns the number of kernel
 * classes.  Synchronises on pending events.
 */
int blockoa_kernel_times(blockoa_operator *op, int max_kernels, double *timed_ms,
                         long long *timed_launches, long long *launches, const char **names);

/* Zero the per-kernel timing of the operator. */
int blockoa_reset_kernel_times(blockoa_operator *op);

/* Kernels launched by the library in this process so far (a graph launch
 * counts each of its kernel nodes).  Host only; never fails. */
long long blockoa_launch_count(void);

/* Free the operator and its workspace (NULL is a no-op).  Synchronises the device. */
void blockoa_destroy(blockoa_operator *op);

/* Static description of a status code. */
const char *blockoa_status_string(int status);

/* Text of the last CUDA error seen by the calling thread ("" if none). */
const char *blockoa_last_error(void);

/* ------------------------------------------------------------------------
 * Learned warm start: a 3-D Fourier neural operator that maps per-cell
 * inputs of one chip shape (e.g. normalised log k, power density and cell
 * coordinates) to a predicted basis solution, used as the initial guess of
 * block CG (blockoa_solve_opts.x0).  The paper trains neural operators on
 * data the method generates (Sec. V-C); the network follows the FNO
 * literature:
 *   v0 = P x + bP;  u_l = K_l(v_l) + W_l v_l + b_l,  v_{l+1} = gelu(u_l)
 *   (no gelu after the last layer);  y = Q2 gelu(Q1 v_L + c1) + c2,
 * K_l the spectral convolution over the retained modes kx in [-mx/2, mx/2),
 * ky in [-my/2, my/2), kz in [0, mz) with complex per-mode channel mixing:
 *   Yh_m = Xh_m R_m,  K(v) = 1/(nx ny nz) sum_m w_m Re(Yh_m e^{+i theta_m}),
 *   w_m = 1 for kz = 0 and 2 otherwise.
 * Weight matrices are used as bfloat16 copies of float32 masters; all
 * arithmetic is float32.
 *
 * Parameters are one float32 array in this order:
 *   P [width][c_in], bP [width], W [layers][width][width], b [layers][width],
 *   Rr, Ri [layers][mz*my*mx][width][width] (R[mode][in][out]; mode = (kz, ky, kx)
 *   row-major with kx fastest), Q1 [hidden][width], c1 [hidden], Q2 [hidden], c2 [1].
 * Gradients use the same layout.
 * ------------------------------------------------------------------------ */
typedef struct blockoa_fno blockoa_fno;

typedef struct {
  int nx, ny, nz;          /* grid of every sample */
  int c_in;                /* input channels per cell, 1..8 */
  int width;               /* 32 */
  int hidden;              /* projection width, 128 */
  int layers;              /* Fourier layers, >= 1 */
  int mx, my, mz;          /* retained modes (even mx, my; mx <= nx, my <= ny, mz <= nz) */
  int max_batch;           /* samples per forward / backward call, >= 1 */
} blockoa_fno_shape;

/* Number of float32 parameters of a shape (host output).  ERR_INVALID for
 * an unsupported shape (width must be 32; hidden 32..256, a multiple of 32). */
int blockoa_fno_param_count(const blockoa_fno_shape *shape, int64_t *count);

/* Create a network with the given initial parameters (host float32 array of
 * blockoa_fno_param_count entries, read before return), zero gradients and
 * zero Adam moments.  Allocates its activations for max_batch samples. */
int blockoa_fno_create(const blockoa_fno_shape *shape, const float *params, blockoa_fno **out);

/* y = net(x).  x: device float32 [batch][nz][ny][nx][c_in]; y: device
 * float32 [batch][nz][ny][nx].  keep = 1 keeps the activations for
 * blockoa_fno_backward. */
int blockoa_fno_forward(blockoa_fno *net, const float *x, float *y, int batch, int keep,
                        blockoa_stream stream);

/* Mean squared error of y against target over batch samples, and its
 * gradient dy = 2 (y - target) / (batch nx ny nz).  loss: device float32 [1]
 * (overwritten); dy: device float32 like y. */
int blockoa_fno_mse(const blockoa_fno *net, const float *y, const float *target, int batch, float *dy,
                    float *loss, blockoa_stream stream);

/* Accumulate into the gradients the gradient of sum(dy * y) for the last
 * forward call made with keep = 1 (same batch). */
int blockoa_fno_backward(blockoa_fno *net, const float *dy, int batch, blockoa_stream stream);

/* Zero the gradients. */
int blockoa_fno_zero_grad(blockoa_fno *net, blockoa_stream stream);

/* One Adam step (Kingma & Ba, Algorithm 1; t counts from 1) on all
 * parameters from the accumulated gradients; refreshes the bfloat16 copies. */
int blockoa_fno_adam_step(blockoa_fno *net, float lr, float beta1, float beta2, float eps, int t,
                          blockoa_stream stream);

/*
 * The warm start's basis from network outputs: sample j of chip c of `op`
 * (y: device float32 [chip][s][n_c], i.e. y[off_c * s + j * n_c + a], the
 * layout of blockoa_fno_forward's output for the s samples of each chip)
 * times scale[c * s + j] (device float64 [n_chips * s]: the sample's input
 * normalisation undone) into X[(off_c + a) * s + j] (device float64
 * [n_total][s], the layout of blockoa_solve_opts.x0).
 * Errors: ERR_INVALID (NULL pointers, s < 1), ERR_OOM, ERR_CUDA.
 */
int blockoa_fno_basis(const blockoa_operator *op, const float *y, const double *scale, int s, double *X,
                      blockoa_stream stream);

/* Copy the float32 parameters or gradients to a host array.  Synchronous. */
int blockoa_fno_get_params(const blockoa_fno *net, float *params);
int blockoa_fno_get_grads(const blockoa_fno *net, float *grads);

/* Free the network (NULL is a no-op).  Synchronises the device. */
void blockoa_fno_destroy(blockoa_fno *net);

#ifdef __cplusplus
}
#endif
#endif /* BLOCKOA_H */
