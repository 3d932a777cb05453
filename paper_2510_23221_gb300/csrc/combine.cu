// New temperature fields T = U C (Eq. 5, Sec. III-B) and the C-ABI entry
// points for the combination and the operator action (Eq. 6).
//
// FP64: float64 SIMT dot products of length s per output (this kernel).
// MIXED: bfloat16x3 on the tensor cores (combine_tc.cu).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "noise.cuh"

namespace blockoa {

struct CombTile {
  int chip, pad;
  long long begin;  // first cell (global numbering) of a 256-cell tile
};

constexpr int CT_CELLS = 256;
constexpr int CT_FIELDS = 32;

// T[m][a] = sum_j U[a][j] C[j][m] (+ epsilon) for a 256-cell tile and 32 fields.
template <typename T, int S>
__global__ void __launch_bounds__(CT_CELLS)
combine_simt_kernel(const CombTile *__restrict__ tiles, const ChipDev *__restrict__ chips,
                    const double *__restrict__ U, const double *__restrict__ C,
                    T *__restrict__ Tout, int s, int M, const CombineEpi epi) {
  const NoiseSpec &nz = epi.nz;
  __shared__ T sC[S][CT_FIELDS];
  const CombTile tile = tiles[blockIdx.x];
  const ChipDev ch = chips[tile.chip];
  const int m0 = blockIdx.y * CT_FIELDS;
  const int nf = min(CT_FIELDS, M - m0);
  const double *Cc = C + (long long)tile.chip * s * M;
  for (int e = threadIdx.x; e < S * CT_FIELDS; e += CT_CELLS) {
    const int j = e / CT_FIELDS, f = e % CT_FIELDS;
    sC[j][f] = (j < s && f < nf) ? (T)Cc[(long long)j * M + m0 + f] : T(0);
  }
  __syncthreads();
  const long long a = tile.begin + threadIdx.x;
  if (a >= ch.off + ch.n) return;
  T u[S];
#pragma unroll
  for (int j = 0; j < S; ++j) u[j] = j < s ? (T)U[a * s + j] : T(0);
  T *out = Tout + ch.off * (long long)M + (a - ch.off);
  const double *inv = epi.inv_sum ? epi.inv_sum + (long long)tile.chip * M + m0 : nullptr;
  for (int f0 = 0; f0 < nf; f0 += 4) {   // m0 is a multiple of 4: one noise block per 4 fields
    double eps[4] = {0.0, 0.0, 0.0, 0.0};
    if (nz.amp > 0.0 && nz.kind == NOISE_UNIFORM) {
      noise4(nz, a, (m0 + f0) / 4, eps);
    } else if (nz.amp > 0.0) {   // Gaussian: two blocks of two fields
      gauss2(nz, a, (m0 + f0) / 2, eps);
      gauss2(nz, a, (m0 + f0) / 2 + 1, eps + 2);
    }
    for (int f = f0; f < f0 + 4 && f < nf; ++f) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < S; ++j) acc += u[j] * sC[j][f];
      if (inv) acc *= (T)inv[f];   // normalised weights of Eq. 5
      out[(long long)(m0 + f) * ch.n] = acc + (T)eps[f - f0];
    }
  }
}

// Normalised weights of Eq. 5, alpha_jm = C_jm / sum_i C_im, applied as
// (U C)_m / sum_i C_im: inv[chip * M + m] = 1 / sum_i C_im (sum in float64,
// i ascending).  A field whose |sum| <= min_rel * sum |C_im| sets *bad.
__global__ void comb_inv_sum_kernel(const double *__restrict__ C, int n_chips, int s, int M,
                                    double min_rel, double *__restrict__ inv, int *__restrict__ bad) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)n_chips * M) return;
  const long long chip = i / M, m = i % M;
  const double *c = C + chip * s * (long long)M + m;
  double sum = 0.0, mag = 0.0;
  for (int j = 0; j < s; ++j) {
    const double v = c[(long long)j * M];
    sum += v;
    mag += fabs(v);
  }
  const bool ok = mag > 0.0 && fabs(sum) > min_rel * mag && isfinite(sum);
  inv[i] = ok ? 1.0 / sum : 0.0;
  if (!ok) atomicExch(bad, 1);
}

int launch_combine(blockoa_operator *op, const double *U, const double *C, void *Tout, int s, int M,
                   int dtype, const CombineEpi &epi, cudaStream_t st) {
  if (dtype == BLOCKOA_MIXED) return launch_combine_tc(op, U, C, (float *)Tout, s, M, epi, st);
  std::vector<CombTile> tiles;
  for (int c = 0; c < op->n_chips; ++c)
    for (long long b = 0; b < op->chips[c].n; b += CT_CELLS)
      tiles.push_back({c, 0, op->chips[c].off + b});
  void *d_tiles = nullptr;
  int rc = pool_alloc(op, &d_tiles, sizeof(CombTile) * tiles.size(), st);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(CombTile) * tiles.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)tiles.size(), (unsigned)((M + CT_FIELDS - 1) / CT_FIELDS));
    const CombTile *dt = (const CombTile *)d_tiles;
    const int S = s <= 8 ? 8 : s <= 16 ? 16 : s <= 32 ? 32 : 64;
#define BLOCKOA_COMB(TT, SS) \
  combine_simt_kernel<TT, SS><<<grid, CT_CELLS, 0, st>>>(dt, op->d_chips, U, C, (TT *)Tout, s, M, epi)
    cudaEvent_t ev;
    time_begin(op, st, &ev);
    g_launches += 1;
    switch (S) {
      case 8: BLOCKOA_COMB(double, 8); break;
      case 16: BLOCKOA_COMB(double, 16); break;
      case 32: BLOCKOA_COMB(double, 32); break;
      default: BLOCKOA_COMB(double, 64); break;
    }
#undef BLOCKOA_COMB
    e = cudaGetLastError();
    time_end(op, st, KC_COMBINE_FP64, ev);
  }
  pool_free(d_tiles, st);
  return cuda_status(e, "combine");
}

}  // namespace blockoa

using namespace blockoa;

static bool valid_dtype(int d) { return d == BLOCKOA_FP64 || d == BLOCKOA_MIXED; }

extern "C" int blockoa_combine_ex(blockoa_operator *op, const double *U, const double *C, void *T,
                                  int s, int M, int dtype, const blockoa_combine_opts *opts,
                                  blockoa_stream stream) {
  if (!op || s < 1 || s > 64 || M < 0 || !valid_dtype(dtype)) return BLOCKOA_ERR_INVALID;
  CombineEpi epi;
  bool normalize = false;
  double min_rel = 1e-6;
  if (opts) {
    if (!(opts->noise_amp >= 0.0) || !std::isfinite(opts->noise_amp)) return BLOCKOA_ERR_INVALID;
    if (opts->noise_kind != BLOCKOA_NOISE_UNIFORM && opts->noise_kind != BLOCKOA_NOISE_GAUSSIAN)
      return BLOCKOA_ERR_INVALID;
    if (opts->normalize != 0 && opts->normalize != 1) return BLOCKOA_ERR_INVALID;
    if (!std::isfinite(opts->normalize_min) || opts->normalize_min >= 1.0) return BLOCKOA_ERR_INVALID;
    epi.nz.seed = (unsigned long long)opts->noise_seed;
    epi.nz.amp = opts->noise_amp;
    epi.nz.kind = opts->noise_kind;
    normalize = opts->normalize == 1;
    if (opts->normalize_min > 0.0) min_rel = opts->normalize_min;
  }
  if (M == 0) return BLOCKOA_OK;
  if (!U || !C || !T) return BLOCKOA_ERR_INVALID;
  if (dtype == BLOCKOA_FP64 && (M + CT_FIELDS - 1) / CT_FIELDS > 65535) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (!normalize) return launch_combine(op, U, C, T, s, M, dtype, epi, st);
  // the weights' column sums first; a field whose sum is ~0 fails the call
  const long long np = (long long)op->n_chips * M;
  void *inv = nullptr, *bad = nullptr;
  int rc = pool_alloc(op, &inv, sizeof(double) * (size_t)np, st);
  if (!rc) rc = pool_alloc(op, &bad, 8, st);
  auto done = [&](int code) { pool_free(inv, st); pool_free(bad, st); return code; };
  if (rc) return done(rc);
  cudaError_t e = cudaMemsetAsync(bad, 0, 8, st);
  if (e == cudaSuccess) {
    g_launches += 1;
    comb_inv_sum_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(C, op->n_chips, s, M, min_rel,
                                                                      (double *)inv, (int *)bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    op->h_flag[0] = 0;
    e = read_small(op->h_flag, bad, 8, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return done(cuda_status(e, "combine: normalised weights"));
  if (op->h_flag[0]) {
    set_last_error(cudaErrorInvalidValue,
                   "blockoa_combine_ex: a field's coefficients sum to ~0 (normalize_min)");
    return done(BLOCKOA_ERR_INVALID);
  }
  epi.inv_sum = (const double *)inv;
  return done(launch_combine(op, U, C, T, s, M, dtype, epi, st));
}

extern "C" int blockoa_combine(blockoa_operator *op, const double *U, const double *C, void *T,
                               int s, int M, int dtype, blockoa_stream stream) {
  return blockoa_combine_ex(op, U, C, T, s, M, dtype, nullptr, stream);
}

extern "C" int blockoa_combine_apply(blockoa_operator *op, const double *U, const double *C, float *T,
                                     float *q, int s, int M, blockoa_stream stream) {
  if (!op || s < 1 || s > 64 || M < 0) return BLOCKOA_ERR_INVALID;
  if (M == 0) return BLOCKOA_OK;
  if (!U || !C || !T || !q || T == q) return BLOCKOA_ERR_INVALID;
  if ((M + 7) / 8 > 65535) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  if (fa_supported(op, s)) return launch_combine_apply(op, U, C, T, q, s, M, st);
  CombineEpi epi;   // rows wider than one window: the two calls in turn
  int rc = launch_combine(op, U, C, T, s, M, BLOCKOA_MIXED, epi, st);
  if (rc) return rc;
  return launch_apply_fields(op, T, q, M, BLOCKOA_MIXED, st);
}

extern "C" int blockoa_apply_basis(const blockoa_operator *op, const double *U, double *AU, int s,
                                   blockoa_stream stream) {
  if (!op || !U || !AU || s < 1 || s > 4096) return BLOCKOA_ERR_INVALID;
  return launch_apply_block64(op, U, AU, s, (cudaStream_t)stream);
}

extern "C" int blockoa_residual_ratio(const blockoa_operator *op, const double *B, const double *X, int s,
                                      double *ratio, blockoa_stream stream) {
  if (!op || s < 1 || s > 64 || !B || !X || !ratio) return BLOCKOA_ERR_INVALID;
  return launch_residual_ratio(op, B, X, s, ratio, (cudaStream_t)stream);
}

extern "C" int blockoa_apply_operator(const blockoa_operator *op, const void *T, void *q, int M,
                                      int dtype, blockoa_stream stream) {
  if (!op || M < 0 || !valid_dtype(dtype)) return BLOCKOA_ERR_INVALID;
  if (M == 0) return BLOCKOA_OK;
  if (!T || !q || T == q) return BLOCKOA_ERR_INVALID;
  if ((M + 7) / 8 > 65535) return BLOCKOA_ERR_INVALID;
  return launch_apply_fields(op, T, q, M, dtype, (cudaStream_t)stream);
}

extern "C" int blockoa_pair_check(const blockoa_operator *op, const void *T, const void *q, int M,
                                  int dtype, double *e_pair, blockoa_stream stream) {
  if (!op || M < 0 || !valid_dtype(dtype)) return BLOCKOA_ERR_INVALID;
  if (M == 0) return BLOCKOA_OK;
  if (!T || !q || !e_pair || M > 65535) return BLOCKOA_ERR_INVALID;
  return launch_pair_check(op, T, q, M, dtype, e_pair, (cudaStream_t)stream);
}
