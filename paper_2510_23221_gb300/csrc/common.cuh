// Internal declarations shared by the translation units of libblockoa.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "blockoa.h"

namespace blockoa {

// ---------------------------------------------------------------- chip table
struct ChipDev {
  int nx, ny, nz;
  int layered;    // 1: conductivity constant within every z-row (layer tables valid)
  long long n;    // cells of the chip
  long long off;  // first cell of the chip in the concatenated numbering
  long long lz;   // first z-row of the chip in the layer tables
};

// Layer table of a layered chip, one record per z-row: the +x, +y, +z face
// conductances of interior faces and the Robin conductance of the 16 edge
// classes (class = 4 * cx + cy, c = 0 interior, 1 low face, 2 high face,
// 3 both faces of a one-cell-wide chip).  Values are identical to the
// per-cell assembly.
constexpr int kLT = 20;   // gx, gy, gz, unused, cb[16]

// A contiguous range of one chip's cells processed by one CTA.
struct Unit {
  int chip, pad;
  long long begin, end;  // global cell indices [begin, end)
};

// Per-chip state of a running block solve (device resident).
struct ChipSolveState {
  int active;       // 1 while the chip iterates
  int status;       // blockoa_status
  int iters;        // block iterations so far (this refinement step)
  int deflated;     // columns dropped by deflation so far
  int rank;         // kept columns in the current factorisation
  int pad0, pad1, pad2;
};
static_assert(sizeof(ChipSolveState) % 8 == 0, "chip states are read back in 8-byte words");

// Kernel classes with live event timing.
enum KernelClass {
  KC_SPMM_GRAM = 0, KC_ALPHA_SOLVE, KC_UPDATE_GRAM, KC_BETA_SOLVE, KC_P_UPDATE,
  KC_RESIDUAL64, KC_COMBINE_TC, KC_SPLIT, KC_APPLY, KC_COMBINE_FP64, KC_ZLINE2, KC_COMBINE_APPLY,
  KC_COUNT
};

struct KernelTimes {
  double ms[KC_COUNT] = {};           // summed duration of the timed launches
  long long samples[KC_COUNT] = {};   // timed launches
  long long launches[KC_COUNT] = {};  // all launches
  // event pairs recorded around launches, resolved when the times are read
  std::vector<int> pend_class;
  std::vector<cudaEvent_t> pend_ev;   // 2 per pending launch
};

// One cell's four float64 conductances (cx, cy, cz, cb) as stored in g64.
struct alignas(32) Coef64 {
  double x, y, z, w;
};

// Kernel launches issued by the library in this process (graph launches
// count every kernel node).
extern std::atomic<long long> g_launches;

// Programmatic dependent launch.  A kernel launched with
// launch_chained(..., chained = true) may be scheduled while the previous
// kernel on the stream is still running; it must call grid_wait_prior()
// before it touches memory that kernel writes (the wait returns once the
// prior grid has completed and its writes are visible, and immediately for
// a kernel launched without the attribute).  grid_release_next() lets the
// next chained kernel be scheduled as soon as SM space frees up.
#ifdef __CUDACC__
__device__ __forceinline__ void grid_wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_release_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                         cudaStream_t st, bool chained, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = chained ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}
#endif

}  // namespace blockoa

struct blockoa_operator {
  int device = 0;
  int n_chips = 0;
  long long n_total = 0;
  long long n_zrows = 0;                 // z-rows of all chips (layer table records)
  std::vector<blockoa::ChipDev> chips;   // host copy
  std::vector<double> cell_area;         // dx * dy per chip (m^2)
  std::vector<double> zrow_dz;           // [n_zrows] cell thickness of every z-row (m)
  blockoa::ChipDev *d_chips = nullptr;   // device copy
  double *g64 = nullptr;                 // [n_total][4]: cx, cy, cz, cb (float64)
  float *g32 = nullptr;                  // [n_total][4]: float32 copies
  double *dinv64 = nullptr;              // [n_total] 1 / diag(A) (Jacobi)
  float *dinv32 = nullptr;               // [n_total] float32 copy
  double *zinv64 = nullptr;              // [n_total] z-line preconditioner: 1 / (Thomas pivot) per cell
  float *zinv32 = nullptr;               // [n_total] float32 copy
  double *lt64 = nullptr;                // [sum nz][kLT] layer tables (float64)
  float *lt32 = nullptr;                 // [sum nz][kLT] float32 copies
  cudaMemPool_t pool = nullptr;          // stream-ordered pool for workspaces
  void *solve_ws = nullptr;              // block-solve workspace (blockcg.cu)
  blockoa::KernelTimes times;            // live per-kernel timing
  void *apply_blocks = nullptr;          // cached launch table of the operator action
  int n_apply_blocks = 0;
  void *apply_vec_blocks = nullptr;      // same for the vectorised form
  int n_apply_vec_blocks = 0;
  int *h_flag = nullptr;                 // pinned status word for small device -> host reads
  int tune_tpu = 0;                      // block-CG unit size in tiles (0: from the tile count)
  int tune_ztpu = 0;                     // z-line unit size in column tiles (0: from the tile count)
  // one-shot status injection for tests (blockoa_inject_chip_status)
  int inject_chip = -1, inject_status = 0, inject_after = 0;
};

namespace blockoa {

// ---------------------------------------------------------------- errors
void set_last_error(cudaError_t e, const char *where);
int cuda_status(cudaError_t e, const char *where);  // BLOCKOA_OK or ERR_CUDA/ERR_OOM

#define BLOCKOA_CUDA(call)                                   \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return ::blockoa::cuda_status(e_, #call); \
  } while (0)

// Small device -> host reads (a few KB) into pinned host memory, done by a
// one-block kernel writing through the mapping rather than by a copy:
// copies of other streams (e.g. results streaming back to the host) then
// never delay the read, which the solver issues at every convergence poll.
// `bytes` must be a multiple of 8 and both addresses 8-byte aligned; the
// data is on the host once `st` has been synchronised.
cudaError_t read_small(void *host_pinned, const void *dev, size_t bytes, cudaStream_t st);

// Stream-ordered allocation from the operator's pool.
int pool_alloc(blockoa_operator *op, void **p, size_t bytes, cudaStream_t st);
void pool_free(void *p, cudaStream_t st);

// Live timing: record an event pair around one launch on `st`.
void time_begin(blockoa_operator *op, cudaStream_t st, cudaEvent_t *ev);
void time_end(blockoa_operator *op, cudaStream_t st, int kclass, cudaEvent_t ev0);
void add_time(blockoa_operator *op, int kclass, double ms);
void add_launches(blockoa_operator *op, int kclass, long long n);

// Work units: every chip's cells split into ranges of at most `cells` cells.
std::vector<Unit> make_units(const blockoa_operator *op, long long cells);
long long pick_unit_cells(const blockoa_operator *op, long long align, long long min_cells,
                          int target_ctas);

// ---------------------------------------------------------------- kernels (host launchers)
// stencil.cu
int launch_apply_fields(const blockoa_operator *op, const void *T, void *q, int M, int dtype,
                        cudaStream_t st);
int launch_pair_check(const blockoa_operator *op, const void *T, const void *q, int M, int dtype,
                      double *e_pair, cudaStream_t st);
// R = B - A X (float64) on a padded block [n_total][S]; also accumulates
// per-chip column norms ||R_j||^2 into rn2 [chip][S] (must be zeroed).
int launch_residual64(const blockoa_operator *op, const double *B, const double *X, double *R,
                      int S, double *rn2, cudaStream_t st, bool det = false);
// ratio[chip][j] = ||B_j - A X_j|| / ||B_j|| for float64 blocks [n_total][s], s <= 64.
int launch_residual_ratio(const blockoa_operator *op, const double *B, const double *X, int s,
                          double *ratio, cudaStream_t st);
// AU = A U, float64 block of s columns [n][s] (blockoa_apply_basis).
int launch_apply_block64(const blockoa_operator *op, const double *U, double *AU, int s, cudaStream_t st);

// blockcg.cu
void free_solve_ws(void *ws);
// Deterministic reduction of per-unit or per-CTA partial sums (slots) into
// per-chip accumulators (ordered_reduce_kernel); state may be null (every
// chip).
cudaError_t launch_ordered_reduce(const double *slots, int n, const int *begin, const int *count,
                                  const ChipSolveState *state, int n_chips, int mode, int S, double *a, double *b,
                                  int diag, cudaStream_t st);

struct CombineEpi;   // noise.cuh

// combine_tc.cu (bfloat16x3 on tcgen05; fields in float32)
int launch_combine_tc(blockoa_operator *op, const double *U, const double *C, float *T, int s,
                      int M, const CombineEpi &epi, cudaStream_t st);

// combine_apply.cu (fused T = U C and q = A T; float32 fields)
bool fa_supported(const blockoa_operator *op, int s);
int launch_combine_apply(blockoa_operator *op, const double *U, const double *C, float *T, float *q, int s,
                         int M, cudaStream_t st);

// combine.cu
int launch_combine(blockoa_operator *op, const double *U, const double *C, void *T, int s, int M,
                   int dtype, const CombineEpi &epi, cudaStream_t st);

}  // namespace blockoa
