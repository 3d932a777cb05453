// Block conjugate gradient for the basis solutions (Eq. 3-4, Sec. III-A).
//
// All s right-hand sides of a chip share its operator A and one Krylov
// space.  One iteration, per chip:
//   Q = A P,   Gamma = P^T Q,   rho = P^T R                 (spmm_gram)
//   deflating solve of the s x s system, alpha = Gamma^-1 rho
//   X += P alpha,  R -= Q alpha,  W = Q^T Z,  ||R_j||^2     (update_gram)
//   beta = -Gamma^-1 W, per-column convergence test
//   P = Z + P beta                                          (p_update)
// with Z = R, or Z = diag(A)^-1 R under Jacobi preconditioning.  Deflated
// columns get zero rows in alpha and beta.  The mixed form forms alpha and
// beta in the last CTA per chip of spmm_gram and update_gram by sweeping
// Gamma in double-float (smallsolve.cuh); the float64 form factors Gamma by
// pivoted Cholesky and substitutes in kernels of their own
// (smallsolve_chol.cuh).
//
// Precision.  FP64 runs the loop in float64.  MIXED runs it in float32 with
// the Gram products folded into compensated float32 sums and reduced in
// float64, the s x s solves in double-float, inside float64 iterative
// refinement on the true residual B - A X.
//
// Layout.  Block vectors are [n_total][S] with S in {8, 16, 32, 64} (the
// caller's s columns zero-padded).  A CTA processes one unit: a contiguous
// range of one chip's cells, in tiles of TC cells (TPC threads per cell, 16
// bytes of columns per thread).  Gram partials are reduced inside the CTA
// and added to per-chip float64 accumulators.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "smallsolve.cuh"
#include "smallsolve_chol.cuh"
#include "tc.cuh"

namespace blockoa {

// ---------------------------------------------------------------- geometry
// A thread owns CPT = 4 consecutive cells x V columns (16 bytes of each of
// the four rows).  TPR threads span the S columns and TCG thread groups span
// the TC = 4 * TCG cells of a tile.  Tiles are staged in shared memory
// transposed, [column][cell] with a padded row of LD cells, so every step of
// the s x s products reads 16-byte vectors of four cells: the updates read
// three vectors per 32 FMAs, the Gram blocks eight vectors per 64 FMAs.
template <typename T, int S>
struct BK {
  static constexpr int V = 16 / (int)sizeof(T);  // columns per thread
  static constexpr int CPT = 4;                  // cells per thread
  static constexpr int TPR = S / V;              // threads across the columns
  static constexpr int TCG = 256 / TPR;          // thread groups along the cells
  static constexpr int TC = TCG * CPT;           // cells per tile
  static constexpr int LD = TC;                  // row of a transposed tile (swizzled)
  static constexpr int NB = S / 4;               // 4x4 Gram blocks per side
  static constexpr int NT = NB * NB;             // threads per Gram group
  static constexpr int NG = 256 / NT;            // Gram groups (split the tile's cells)
  static constexpr int GC = TC / NG;             // cells per group and tile
  static_assert(TPR >= 1 && TC % 4 == 0 && NG >= 1 && GC % 4 == 0, "bad block geometry");
  static_assert((TC / V) % 8 == 0, "swizzle needs at least eight 16-byte units per row");
};

template <typename T>
__device__ __forceinline__ void vload(T *dst, const T *src);
template <>
__device__ __forceinline__ void vload<float>(float *d, const float *s) {
  float4 v = *reinterpret_cast<const float4 *>(s);
  d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
}
template <>
__device__ __forceinline__ void vload<double>(double *d, const double *s) {
  double2 v = *reinterpret_cast<const double2 *>(s);
  d[0] = v.x; d[1] = v.y;
}
template <typename T>
__device__ __forceinline__ void vstore(T *dst, const T *src);
template <>
__device__ __forceinline__ void vstore<float>(float *d, const float *s) {
  *reinterpret_cast<float4 *>(d) = make_float4(s[0], s[1], s[2], s[3]);
}
template <>
__device__ __forceinline__ void vstore<double>(double *d, const double *s) {
  *reinterpret_cast<double2 *>(d) = make_double2(s[0], s[1]);
}
// Transposed tiles are [column][cell] rows of LD = TC cells.  The 16-byte
// units of a row are XOR-swizzled with (row / 4) & 7 so that the transposed
// writes (rows four apart), the update reads (one row, four units) and the
// 4x4 Gram reads (four or eight rows, one unit) each spread over all eight
// 16-byte bank groups.
template <typename T>
__device__ __forceinline__ int swz(int row, int cell) {
  constexpr int V = 16 / sizeof(T);
  return (((cell / V) ^ ((row >> 2) & 7)) * V) + (cell % V);
}
// four consecutive cells (multiple of 4) of a tile row
template <typename T, int LD>
__device__ __forceinline__ void ld4(T *d, const T *tile, int row, int cell) {
  const T *r = tile + row * LD;
  vload<T>(d, r + swz<T>(row, cell));
  if (sizeof(T) == 8) vload<T>(d + 2, r + swz<T>(row, cell + 2));
}
template <typename T, int LD>
__device__ __forceinline__ void st4(T *tile, const T *s, int row, int cell) {
  T *r = tile + row * LD;
  vstore<T>(r + swz<T>(row, cell), s);
  if (sizeof(T) == 8) vstore<T>(r + swz<T>(row, cell + 2), s + 2);
}

__device__ __forceinline__ float4 coef_ld(const float *g, long long a) {
  return __ldg(reinterpret_cast<const float4 *>(g) + a);
}
__device__ __forceinline__ Coef64 coef_ld(const double *g, long long a) {
  const double2 lo = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a);
  const double2 hi = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a + 1);
  return Coef64{lo.x, lo.y, hi.x, hi.y};
}

// (A v)_a on the V columns at j0 of a [cell][S] block vector vb, given the
// cell's own values vc and its grid position.  All six neighbour rows and
// the three lower-face coefficients are requested before any is used; a
// neighbour outside the chip is read at the cell itself with a zero
// coefficient, so its term is exactly zero and the sum is the 7-point
// stencil in the order +x, -x, +y, -y, +z, -z.
template <typename T, int S>
__device__ __forceinline__ void stencil_row(const T *__restrict__ g, const T *__restrict__ vb, long long a,
                                            const T (&vc)[16 / sizeof(T)], int x, int y, int z, int nx, int ny,
                                            int nz, long long nxny, int j0, T (&out)[16 / sizeof(T)]) {
  constexpr int V = 16 / sizeof(T);
  const bool xp = x + 1 < nx, xm = x > 0, yp = y + 1 < ny, ym = y > 0, zp = z + 1 < nz, zm = z > 0;
  const long long b[6] = {xp ? a + 1 : a, xm ? a - 1 : a, yp ? a + nx : a,
                          ym ? a - nx : a, zp ? a + nxny : a, zm ? a - nxny : a};
  const auto c4 = coef_ld(g, a);
  const auto cxm = coef_ld(g, b[1]);
  const auto cym = coef_ld(g, b[3]);
  const auto czm = coef_ld(g, b[5]);
  T o[6][V];
#pragma unroll
  for (int i = 0; i < 6; ++i) vload<T>(o[i], vb + b[i] * S + j0);
  const T gg[6] = {xp ? c4.x : T(0), xm ? cxm.x : T(0), yp ? c4.y : T(0),
                   ym ? cym.y : T(0), zp ? c4.z : T(0), zm ? czm.z : T(0)};
#pragma unroll
  for (int v = 0; v < V; ++v) {
    T acc = c4.w * vc[v];
#pragma unroll
    for (int i = 0; i < 6; ++i) acc += gg[i] * (vc[v] - o[i][v]);
    out[v] = acc;
  }
}

// Load this thread's 4 cells x V columns of a [cell][S] block (zeros past `end`).
template <typename T, int S>
__device__ __forceinline__ void load_block(T (&x)[4][16 / sizeof(T)], const T *G, long long c0,
                                           long long end, int j0) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (c0 + k < end) vload<T>(x[k], G + (c0 + k) * S + j0);
    else {
#pragma unroll
      for (int v = 0; v < V; ++v) x[k][v] = T(0);
    }
  }
}
template <typename T, int S>
__device__ __forceinline__ void store_block(T *G, const T (&x)[4][16 / sizeof(T)], long long c0,
                                            long long end, int j0) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    if (c0 + k < end) vstore<T>(G + (c0 + k) * S + j0, x[k]);
}
// Write the block transposed into a [column][cell] tile at local cell cl0.
template <typename T, int LD>
__device__ __forceinline__ void put_tile(T *tile, const T (&x)[4][16 / sizeof(T)], int cl0, int j0) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    T col[4] = {x[0][v], x[1][v], x[2][v], x[3][v]};
    st4<T, LD>(tile, col, j0 + v, cl0);
  }
}

// acc[a*4+b] += sum over cells [cbeg, cbeg + nc) of A[i0+a][c] * B[j0+b][c]
// for transposed tiles A, B.
// float32: paired FMAs (fma.rn.f32x2) over adjacent cells, two partial sums
// per entry folded into acc at the end of the range -- half the FMA
// instructions of the scalar form for the same arithmetic.
template <typename T, int S>
__device__ __forceinline__ void gram_range(T *acc, const T *A, const T *B, int i0, int j0,
                                           int cbeg, int nc) {
  using G = BK<T, S>;
  if constexpr (sizeof(T) == 4 && S == 32 && G::LD % 32 == 0) {
    if ((cbeg & 31) == 0 && (nc & 31) == 0) {
      // Same products and order, addresses without per-load swizzle arithmetic:
      // rows i0..i0+3 (j0..j0+3) share the swizzle key (row / 4) & 7, and for
      // a range starting at a multiple of 32 cells the 16-byte unit of cell
      // step u is (u & ~7) + ((u & 7) ^ key).
      const int kA = (i0 >> 2) & 7, kB = (j0 >> 2) & 7;
      const float *a0 = A + i0 * G::LD + cbeg, *b0 = B + j0 * G::LD + cbeg;
      float2 pr[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) pr[e] = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int u8 = 0; u8 < nc / 4; u8 += 8)
#pragma unroll
      for (int uu = 0; uu < 8; ++uu) {
        const int oa = (u8 + (uu ^ kA)) * 4, ob = (u8 + (uu ^ kB)) * 4;
        float a[4][4], b[4][4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          vload<float>(a[q], a0 + q * G::LD + oa);
          vload<float>(b[q], b0 + q * G::LD + ob);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            pr[q * 4 + r] = __ffma2_rn(make_float2(a[q][0], a[q][1]), make_float2(b[r][0], b[r][1]), pr[q * 4 + r]);
            pr[q * 4 + r] = __ffma2_rn(make_float2(a[q][2], a[q][3]), make_float2(b[r][2], b[r][3]), pr[q * 4 + r]);
          }
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[e] += pr[e].x + pr[e].y;
      return;
    }
  }
  if constexpr (sizeof(T) == 4) {
    float2 pr[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) pr[e] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int c = cbeg; c < cbeg + nc; c += 4) {
      float a[4][4], b[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ld4<float, G::LD>(a[q], A, i0 + q, c);
        ld4<float, G::LD>(b[q], B, j0 + q, c);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          pr[q * 4 + r] = __ffma2_rn(make_float2(a[q][0], a[q][1]), make_float2(b[r][0], b[r][1]), pr[q * 4 + r]);
          pr[q * 4 + r] = __ffma2_rn(make_float2(a[q][2], a[q][3]), make_float2(b[r][2], b[r][3]), pr[q * 4 + r]);
        }
    }
#pragma unroll
    for (int e = 0; e < 16; ++e) acc[e] += pr[e].x + pr[e].y;
  } else {
#pragma unroll 2
    for (int c = cbeg; c < cbeg + nc; c += 4) {
      T a[4][4], b[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        ld4<T, G::LD>(a[q], A, i0 + q, c);
        ld4<T, G::LD>(b[q], B, j0 + q, c);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[q * 4 + r] += a[q][k] * b[r][k];
    }
  }
}

// Same over this group's share of the tile.
template <typename T, int S>
__device__ __forceinline__ void gram_tile(T *acc, const T *A, const T *B, int i0, int j0, int grp) {
  using G = BK<T, S>;
  gram_range<T, S>(acc, A, B, i0, j0, grp * G::GC, G::GC);
}

// float32 -> float64 by integer instructions (float64 instructions issue at
// 1/64 of the float32 rate on this part): exact for every float, subnormals
// and non-finite values included.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long m = u & 0x7fffffu;
  if (ex == 0xffu) return __longlong_as_double((long long)(sgn | 0x7ff0000000000000ull | (m << 29)));
  if (ex == 0u) {
    if (m == 0) return __longlong_as_double((long long)sgn);
    const int b = 63 - __clzll((long long)m);   // leading bit of a subnormal's m 2^-149
    return __longlong_as_double((long long)(sgn | ((unsigned long long)(b + 874) << 52) |
                                            ((m ^ (1ull << b)) << (52 - b))));
  }
  return __longlong_as_double((long long)(sgn | ((unsigned long long)(ex + 896) << 52) | (m << 29)));
}

// Where a flush puts its per-entry partial sums: added to the chip's
// float64 accumulator by atomics (entry e at acc[e * stride]), or, in a
// deterministic solve, stored in the CTA's slot (entry e at slot[e]) for a
// reduction in a fixed order (ordered_reduce_kernel).
struct Sink {
  double *acc;
  double *slot;
  int stride;
  __device__ __forceinline__ void put(int e, double v) const {
    if (slot) slot[e] = v;
    else atomicAdd(acc + (long long)e * stride, v);
  }
};
__device__ __forceinline__ Sink sink(double *acc, double *slot, int stride = 1) { return Sink{acc, slot, stride}; }

// Reduce the NG groups' 4x4 blocks in shared memory and add the S x S
// result to the chip's float64 accumulator.  float partial sums (each over
// at most a few hundred cells of one CTA) are combined across groups with
// error-free transformations, so an entry costs one float64 conversion and
// one float64 atomic per CTA; float64 arithmetic runs at 1/64 of the float32
// rate on this part.
template <typename T, int S>
__device__ void gram_flush(const T *acc, double *red, const Sink &dst, bool diag) {
  using G = BK<T, S>;
  const int t = threadIdx.x;
  const int g = t / G::NT, w = t % G::NT;
  const int i0 = (w / G::NB) * 4, j0 = (w % G::NB) * 4;
  T *rt = reinterpret_cast<T *>(red);
#pragma unroll
  for (int e = 0; e < 16; ++e) rt[g * S * S + (i0 + e / 4) * S + j0 + (e % 4)] = acc[e];
  __syncthreads();
  for (int e = t; e < S * S; e += 256) {
    if (diag && e / S != e % S) continue;   // independent columns: diagonal only
    if constexpr (sizeof(T) == 4) {
      float hi = 0.f, lo = 0.f;
      for (int gg = 0; gg < G::NG; ++gg) {
        const float v = rt[gg * S * S + e];
        const float sum = hi + v;
        const float bp = sum - hi;
        lo += (hi - (sum - bp)) + (v - bp);
        hi = sum;
      }
      dst.put(e, f2d_exact(hi) + f2d_exact(lo));
    } else {
      double sum = 0.0;
      for (int gg = 0; gg < G::NG; ++gg) sum += rt[gg * S * S + e];
      dst.put(e, sum);
    }
  }
  __syncthreads();
}

// Flush when the first NG/2 groups hold P^T Q partials and the rest P^T R.
template <typename T, int S>
__device__ void gram_flush_split(const T *acc, double *red, const Sink &dst_a, const Sink &dst_b, bool diag) {
  using G = BK<T, S>;
  const int t = threadIdx.x;
  const int g = t / G::NT, w = t % G::NT;
  const int i0 = (w / G::NB) * 4, j0 = (w % G::NB) * 4;
  T *rt = reinterpret_cast<T *>(red);
#pragma unroll
  for (int e = 0; e < 16; ++e) rt[g * S * S + (i0 + e / 4) * S + j0 + (e % 4)] = acc[e];
  __syncthreads();
  constexpr int H = G::NG / 2;
  for (int e = t; e < S * S; e += 256) {
    if (diag && e / S != e % S) continue;   // independent columns: diagonal only
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      T hi = T(0), lo = T(0);
      for (int gg = half * H; gg < (half + 1) * H; ++gg) {
        const T v = rt[gg * S * S + e];
        const T sum = hi + v;
        const T bp = sum - hi;
        lo += (hi - (sum - bp)) + (v - bp);
        hi = sum;
      }
      if constexpr (sizeof(T) == 4) (half ? dst_b : dst_a).put(e, f2d_exact(hi) + f2d_exact(lo));
      else (half ? dst_b : dst_a).put(e, (double)hi + (double)lo);
    }
  }
  __syncthreads();
}

template <typename T, int S>
constexpr size_t tile_bytes() { return (size_t)S * BK<T, S>::LD * sizeof(T); }
constexpr size_t kRedBytes = 256 * 16 * sizeof(double);

// ---------------------------------------------------------------- unit scheduling
// The loop kernels run persistent CTAs (about as many as fit on the GPU at
// once) that fetch units -- a few tiles of one chip -- from a counter, so
// SMs finish together whatever the chips' sizes, and units of chips that
// have converged are skipped in bulk (the chips' units are contiguous).
struct UnitSched {
  const Unit *units;
  int n_units;
  const int *chip_unit_end;   // [chip] index of the first unit past the chip
  int *work;                  // [0] next unit, [1] CTAs finished (zero between launches)
  int stat;                   // 1: static schedule (deterministic solves): CTA b takes units b, b + G, ...
  const int *chip_unit_count; // [chip] units of the chip (chips' units are contiguous, largest chip first)
};
// First unit of chip c.
__device__ __forceinline__ int unit0(const UnitSched &us, int c) {
  return us.chip_unit_end[c] - us.chip_unit_count[c];
}

// Thread 0's scheduling registers: the unit fetched ahead, and the last
// chip whose active flag it read, as 2 chip + flag (flags do not change
// while a loop kernel runs: a chip is switched off only after its last
// unit of the launch).
struct SchedLocal {
  int pend = -1, ck = -1;
};
// The unit handed to the CTA and its chip's geometry, published in shared
// memory by thread 0 (the geometry is read from global memory only when
// the chip changes; ch_id is the chip it belongs to).
struct UnitSlot {
  Unit u;
  ChipDev ch;
  int ui, ch_id;
};

// Next unit of the calling CTA (n_units when none is left).  Thread 0
// fetches one unit ahead: the atomic for the following unit is issued here
// and its value (kept in `sl.pend`) is used at the next call, so the round
// trip to the counter overlaps the current unit's work instead of stalling
// the CTA at every unit.  Thread 0 also publishes the unit's record (and,
// given `chips`, its chip's geometry) in shared memory and reads a chip's
// active flag once per chip, so the CTA's threads start on the unit
// without global round trips of their own.
__device__ __forceinline__ int next_unit(const UnitSched &us, const ChipSolveState *state, UnitSlot *slot,
                                         SchedLocal &sl, const ChipDev *chips = nullptr) {
  __syncthreads();   // every thread has read the previous value
  if (threadIdx.x == 0 && us.stat) {   // static: units b, b + G, ... of active chips, in order
    if (sl.pend < 0) slot->ch_id = -1;   // first call of the launch
    const int G = (int)gridDim.x, b = (int)blockIdx.x;
    int ui = sl.pend >= 0 ? sl.pend : b;
    Unit u{};
    while (ui < us.n_units) {
      u = us.units[ui];
      if ((sl.ck >> 1) != u.chip) sl.ck = 2 * u.chip + (state[u.chip].active ? 1 : 0);
      if (sl.ck & 1) break;
      const int e = us.chip_unit_end[u.chip];   // this CTA's first unit past the chip
      ui = e + (((b - e) % G) + G) % G;
    }
    if (ui > us.n_units) ui = us.n_units;
    slot->u = u;
    slot->ui = ui;
    if (chips && ui < us.n_units && u.chip != slot->ch_id) {
      slot->ch = chips[u.chip];
      slot->ch_id = u.chip;
    }
    sl.pend = ui < us.n_units ? ui + G : us.n_units;
  } else if (threadIdx.x == 0) {
    if (sl.pend < 0) slot->ch_id = -1;   // first call of the launch
    int ui = sl.pend >= 0 ? sl.pend : atomicAdd(&us.work[0], 1);
    Unit u{};
    for (;;) {
      if (ui >= us.n_units) break;
      u = us.units[ui];
      if ((sl.ck >> 1) != u.chip) sl.ck = 2 * u.chip + (state[u.chip].active ? 1 : 0);
      if (sl.ck & 1) break;
      atomicMax(&us.work[0], us.chip_unit_end[u.chip]);   // skip the rest of this chip
      ui = atomicAdd(&us.work[0], 1);
    }
    slot->u = u;
    slot->ui = ui;
    if (chips && ui < us.n_units && u.chip != slot->ch_id) {
      slot->ch = chips[u.chip];
      slot->ch_id = u.chip;
    }
    sl.pend = ui < us.n_units ? atomicAdd(&us.work[0], 1) : us.n_units;
  }
  __syncthreads();
  return slot->ui;
}

// Every CTA calls this once its loop is over; the last one resets the
// counters for the next launch (no CTA fetches after it has finished).
__device__ __forceinline__ void sched_finish(const UnitSched &us) {
  __syncthreads();
  if (threadIdx.x == 0 && !us.stat) {
    __threadfence();
    if (atomicAdd(&us.work[1], 1) == (int)gridDim.x - 1) {
      us.work[0] = 0;
      us.work[1] = 0;
    }
  }
}

// ---------------------------------------------------------------- staged tiles (float32)
// The staged loop kernels copy whole tiles (TC cells x S columns of a block
// vector, 16 KB) into shared memory with cp.async several tiles ahead of
// the one they compute on, so global latency overlaps arithmetic.  A staged
// tile keeps the global [cell][column] order; the 16-byte chunks of row r
// are XOR-swizzled with r & 7 (r & 3 for 64-byte rows) so that one chunk
// read from four consecutive rows hits four different bank groups.
template <int S>
struct Stage32 {
  static constexpr int NQ = S / 4;                   // 16-byte chunks per row
  static constexpr int TC = BK<float, S>::TC;        // cells per tile
  static constexpr int MASK = NQ < 8 ? NQ - 1 : 7;
  static constexpr int FLOATS = TC * S;              // floats per staged tile
  static_assert(TC * NQ % 256 == 0, "a tile is a whole number of chunks per thread");
  __device__ static __forceinline__ int off(int row, int q) { return row * S + ((q ^ (row & MASK)) << 2); }
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stage rows [base, base + TC) of a [cell][S] block vector (zeros past end).
template <int S>
__device__ __forceinline__ void stage_tile(float *dst, const float *src, long long base, long long end) {
  using SG = Stage32<S>;
#pragma unroll
  for (int m = 0; m < SG::TC * SG::NQ / 256; ++m) {
    const int c = threadIdx.x + 256 * m;
    const int row = c / SG::NQ, q = c % SG::NQ;
    const bool in = base + row < end;
    cp_async16(dst + SG::off(row, q), in ? src + (base + row) * S + q * 4 : src, in ? 16 : 0);
  }
}

// The tiles of the calling CTA, in order: units blockIdx.x, blockIdx.x +
// gridDim.x, ... of chips that are still active, each cut into tiles of TC
// cells.  Every thread walks the same sequence.
struct TileWalk {
  int ui = 0, chip = -1;
  long long base = 0, end = 0;
  __device__ void seek(const UnitSched &us, const ChipSolveState *state, int u) {
    const int G = (int)gridDim.x;
    while (u < us.n_units) {
      const Unit un = us.units[u];
      // the chip being walked is active (flags do not change while the kernel runs)
      if (un.chip == chip || state[un.chip].active) {
        ui = u; chip = un.chip; base = un.begin; end = un.end;
        return;
      }
      const int e = us.chip_unit_end[un.chip];   // skip the chip's other units
      u += ((e - u + G - 1) / G) * G;
    }
    ui = us.n_units;
    chip = -1;
  }
  template <int TC>
  __device__ void next(const UnitSched &us, const ChipSolveState *state) {
    base += TC;
    if (base >= end) seek(us, state, ui + (int)gridDim.x);
  }
  __device__ bool valid(const UnitSched &us) const { return ui < us.n_units; }
};

// ---------------------------------------------------------------- kernels
// Q = A P on the block layout; Gamma += P^T Q and rho += P^T R per chip.
template <typename T, int S>
__global__ void __launch_bounds__(256, 2)
spmm_gram_kernel(const UnitSched us, const ChipDev *__restrict__ chips, const T *__restrict__ g,
                 const T *__restrict__ P, const T *__restrict__ R, T *__restrict__ Q, const SmallArgs A) {
  using G = BK<T, S>;
  constexpr int V = G::V;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  T *sQ = sP + S * G::LD;
  T *sR = sQ + S * G::LD;
  double *red = reinterpret_cast<double *>(smem);   // reused between units
  __shared__ UnitSlot s_unit;
  grid_release_next();
  grid_wait_prior();
  const int t = threadIdx.x;
  const int j0 = (t % G::TPR) * V, cl0 = (t / G::TPR) * 4;
  const int grp = t / G::NT, w = t % G::NT;
  const int i0 = (w / G::NB) * 4, k0 = (w % G::NB) * 4;
  // With two or more Gram groups, the first half of the groups accumulates
  // P^T Q and the second half P^T R, each over twice the cells (one 4x4
  // block of accumulators per thread); with one group a thread holds both.
  constexpr bool SPLIT = G::NG >= 2;
  constexpr int NA = SPLIT ? 16 : 32;
  T acc[NA];
#pragma unroll
  for (int e = 0; e < NA; ++e) acc[e] = T(0);
  int cur = -1, run = 0, run_first = 0;   // chip of the running accumulation and its units
  SchedLocal sl;   // thread 0: the unit fetched ahead, the last chip checked
  for (;;) {
    const int ui = next_unit(us, A.state, &s_unit, sl, chips);
    const int chip = ui < us.n_units ? s_unit.u.chip : -1;
    if (run > 0 && chip != cur) {   // flush the running chip
      double *slot = A.det_spmm ? A.det_spmm + (long long)(A.det_base[cur] + run_first - unit0(us, cur)) * 2 * S * S
                                : nullptr;
      const Sink sg = sink(A.gram + (long long)cur * S * S, slot);
      const Sink sr = sink(A.rho + (long long)cur * S * S, slot ? slot + S * S : nullptr);
      if constexpr (SPLIT) {
        gram_flush_split<T, S>(acc, red, sg, sr, A.diag);
      } else {
        gram_flush<T, S>(acc, red, sg, A.diag);
        gram_flush<T, S>(acc + 16, red, sr, A.diag);
      }
      // mixed form: the flush that completes the chip sweeps Gamma and forms alpha
      if constexpr (sizeof(T) == 4) {
        if (A.tail && last_flush_of_chip(A.ticket + cur, run, A.unit_count[cur])) chip_alpha<T, S>(A, cur);
      }
#pragma unroll
      for (int e = 0; e < NA; ++e) acc[e] = T(0);
      run = 0;
    }
    if (ui >= us.n_units) break;
    const Unit u = s_unit.u;
    cur = u.chip;
    if (run == 0) run_first = ui;
    ++run;
    const ChipDev ch = s_unit.ch;
    const int nx = ch.nx, ny = ch.ny, nz = ch.nz, nxny = nx * ny;
    for (long long base = u.begin; base < u.end; base += G::TC) {
      T pc[4][V], qv[4][V], rv[4][V];
      load_block<T, S>(pc, P, base + cl0, u.end, j0);
      load_block<T, S>(rv, R, base + cl0, u.end, j0);
      // grid position of the first of this thread's four consecutive cells;
      // the others follow by increments (one division per tile, not per cell)
      const int loc0 = (int)(base + cl0 - ch.off);
      int x = loc0 % nx, y = (loc0 / nx) % ny, z = loc0 / nxny;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long long a = base + cl0 + k;
        if (k > 0) {
          ++x;
          while (x >= nx) {
            x -= nx;
            if (++y >= ny) { y = 0; ++z; }
          }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) qv[k][v] = T(0);
        if (a < u.end) stencil_row<T, S>(g, P, a, pc[k], x, y, z, nx, ny, nz, nxny, j0, qv[k]);
      }
      store_block<T, S>(Q, qv, base + cl0, u.end, j0);
      put_tile<T, G::LD>(sP, pc, cl0, j0);
      put_tile<T, G::LD>(sQ, qv, cl0, j0);
      put_tile<T, G::LD>(sR, rv, cl0, j0);
      __syncthreads();
      if constexpr (SPLIT) {
        constexpr int H = G::NG / 2;
        const bool second = grp >= H;
        gram_range<T, S>(acc, sP, second ? sR : sQ, i0, k0, (grp % H) * 2 * G::GC, 2 * G::GC);
      } else {
        gram_tile<T, S>(acc, sP, sQ, i0, k0, grp);
        gram_tile<T, S>(acc + 16, sP, sR, i0, k0, grp);
      }
      __syncthreads();
    }
  }
  sched_finish(us);
}

// Flush of the update kernel's running accumulation for chip c: W += Q^T Z
// (Gram blocks) and rn2 += ||R_new_j||^2 (threads with equal t % TPR own the
// same columns).
template <typename T, int S>
__device__ __forceinline__ void update_flush(const T *aw, const T *rn, double *red, const SmallArgs &A, int c,
                                             bool with_w, double *slot) {
  using G = BK<T, S>;
  constexpr int V = G::V;
  const int t = threadIdx.x;
  // slot layout of a deterministic solve: W (with_w), then ||R_j||^2
  const Sink rs = sink(A.rn2 + rn2_at(c, S, 0), slot ? slot + (with_w ? S * S : 0) : nullptr, kRn2Stride);
  if (with_w) gram_flush<T, S>(aw, red, sink(A.wg + (long long)c * S * S, slot), A.diag);
  T *rt = reinterpret_cast<T *>(red);
#pragma unroll
  for (int v = 0; v < V; ++v) rt[t * V + v] = rn[v];
  __syncthreads();
  if (t < G::TPR) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      T hi = T(0), lo = T(0);
      for (int tt = t; tt < 256; tt += G::TPR) {
        const T x = rt[tt * V + v];
        const T s2 = hi + x;
        const T bp = s2 - hi;
        lo += (hi - (s2 - bp)) + (x - bp);
        hi = s2;
      }
      if constexpr (sizeof(T) == 4) rs.put(t * V + v, f2d_exact(hi) + f2d_exact(lo));
      else rs.put(t * V + v, (double)hi + (double)lo);
    }
  }
  __syncthreads();
}

// X += P alpha, R -= Q alpha; W += Q^T Z_new and rn2 += ||R_new_j||^2, with
// Z = R (PCM 0) or D^-1 R (PCM 1).  Two CTAs per SM: the persistent loop
// keeps the Gram and norm partials of the running chip live across units,
// which does not fit 80 registers.
template <typename T, int S, int PCM>
__global__ void __launch_bounds__(256, 2)
update_gram_kernel(const UnitSched us, const T *__restrict__ P, const T *__restrict__ Q,
                   T *__restrict__ X, T *__restrict__ R, const T *__restrict__ dinv, const SmallArgs A) {
  using G = BK<T, S>;
  constexpr int V = G::V;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  T *sQ = sP + S * G::LD;
  T *sR = sQ + S * G::LD;
  T *sA = sR + S * G::LD;
  double *red = reinterpret_cast<double *>(smem);   // reused between units
  __shared__ UnitSlot s_unit;
  grid_release_next();
  grid_wait_prior();
  const int t = threadIdx.x;
  const int j0 = (t % G::TPR) * V, cl0 = (t / G::TPR) * 4;
  const int grp = t / G::NT, w = t % G::NT;
  const int i0 = (w / G::NB) * 4, k0 = (w % G::NB) * 4;
  T aw[16], rn[V];
#pragma unroll
  for (int e = 0; e < 16; ++e) aw[e] = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) rn[v] = T(0);
  int cur = -1, run = 0, run_first = 0;
  SchedLocal sl;   // thread 0: the unit fetched ahead, the last chip checked
  for (;;) {
    const int ui = next_unit(us, A.state, &s_unit, sl);
    const int chip = ui < us.n_units ? s_unit.u.chip : -1;
    if (run > 0 && chip != cur) {   // flush the running chip
      update_flush<T, S>(aw, rn, red, A, cur, true,
                         A.det_upd ? A.det_upd + (long long)(A.det_ubase[cur] + run_first - unit0(us, cur)) * (S * S + S)
                                   : nullptr);
      // mixed form: the flush that completes the chip forms beta and tests convergence
      if constexpr (sizeof(T) == 4) {
        if (A.tail && last_flush_of_chip(A.ticket + A.n_chips + cur, run, A.unit_count[cur]))
          chip_beta<T, S>(A, cur);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) aw[e] = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) rn[v] = T(0);
      run = 0;
    }
    if (ui >= us.n_units) break;
    const Unit u = s_unit.u;
    if (u.chip != cur) {   // alpha of the chip (the tiles below read sA after a barrier)
      const T *al = reinterpret_cast<const T *>(A.alpha) + (long long)u.chip * S * S;
      for (int e = t; e < S * S; e += 256) sA[e] = al[e];
    }
    cur = u.chip;
    if (run == 0) run_first = ui;
    ++run;
    for (long long base = u.begin; base < u.end; base += G::TC) {
      {
        T pv[4][V], qv[4][V];
        load_block<T, S>(pv, P, base + cl0, u.end, j0);
        load_block<T, S>(qv, Q, base + cl0, u.end, j0);
        put_tile<T, G::LD>(sP, pv, cl0, j0);
        put_tile<T, G::LD>(sQ, qv, cl0, j0);
      }
      T xv[4][V], rv[4][V];
      load_block<T, S>(xv, X, base + cl0, u.end, j0);
      load_block<T, S>(rv, R, base + cl0, u.end, j0);
      __syncthreads();
#pragma unroll 4
      for (int i = 0; i < S; ++i) {
        T p4[4], q4[4], av[V];
        ld4<T, G::LD>(p4, sP, i, cl0);
        ld4<T, G::LD>(q4, sQ, i, cl0);
        vload<T>(av, sA + i * S + j0);
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int v = 0; v < V; ++v) {
            xv[k][v] += p4[k] * av[v];
            rv[k][v] -= q4[k] * av[v];
          }
      }
      store_block<T, S>(X, xv, base + cl0, u.end, j0);
      store_block<T, S>(R, rv, base + cl0, u.end, j0);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) rn[v] += rv[k][v] * rv[k][v];  // zero past the end
      if constexpr (PCM == 1) {
        // Gram with Z = D^-1 R_new (R stays unscaled in memory)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T di = base + cl0 + k < u.end ? dinv[base + cl0 + k] : T(0);
#pragma unroll
          for (int v = 0; v < V; ++v) rv[k][v] *= di;
        }
      }
      put_tile<T, G::LD>(sR, rv, cl0, j0);
      __syncthreads();
      gram_tile<T, S>(aw, sQ, sR, i0, k0, grp);
      __syncthreads();
    }
  }
  sched_finish(us);
}

// P = Z + P beta, Z = R (PCM 0), D^-1 R (PCM 1) or the z-line Z stored by
// the update kernel (PCM 2, read from Zb).
template <typename T, int S, int PCM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 2)
p_update_kernel(const UnitSched us, const ChipSolveState *__restrict__ state, const T *__restrict__ beta,
                const T *__restrict__ R, T *__restrict__ P, const T *__restrict__ dinv, const T *__restrict__ Zb) {
  using G = BK<T, S>;
  constexpr int V = G::V;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  T *sB = sP + S * G::LD;
  __shared__ UnitSlot s_unit;
  grid_release_next();
  grid_wait_prior();
  const int t = threadIdx.x;
  const int j0 = (t % G::TPR) * V, cl0 = (t / G::TPR) * 4;
  int cur = -1;
  SchedLocal sl;   // thread 0: the unit fetched ahead, the last chip checked
  for (;;) {
    const int ui = next_unit(us, state, &s_unit, sl);
    if (ui >= us.n_units) break;
    const Unit u = s_unit.u;
    if (u.chip != cur) {   // beta of the chip (read after the tile barrier)
      const T *be = beta + (long long)u.chip * S * S;
      for (int e = t; e < S * S; e += 256) sB[e] = be[e];
      cur = u.chip;
    }
    for (long long base = u.begin; base < u.end; base += G::TC) {
      {
        T pv[4][V];
        load_block<T, S>(pv, P, base + cl0, u.end, j0);
        put_tile<T, G::LD>(sP, pv, cl0, j0);
      }
      T rv[4][V];
      load_block<T, S>(rv, PCM == 2 ? Zb : R, base + cl0, u.end, j0);
      if constexpr (PCM == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T di = base + cl0 + k < u.end ? dinv[base + cl0 + k] : T(0);
#pragma unroll
          for (int v = 0; v < V; ++v) rv[k][v] *= di;
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int i = 0; i < S; ++i) {
        T p4[4], bv[V];
        ld4<T, G::LD>(p4, sP, i, cl0);
        vload<T>(bv, sB + i * S + j0);
#pragma unroll
        for (int k = 0; k < 4; ++k)
#pragma unroll
          for (int v = 0; v < V; ++v) rv[k][v] += p4[k] * bv[v];
      }
      store_block<T, S>(P, rv, base + cl0, u.end, j0);
      __syncthreads();
    }
  }
  sched_finish(us);
}

// Staged float32 form of p_update_kernel: P = Z + P beta with the old P and
// Z tiles copied NST - 1 tiles ahead.  P is updated in place (every tile is
// read and written by one CTA only).
template <int S, int PCM, int NST>
__global__ void __launch_bounds__(256, 2)
p_update_staged_kernel(const UnitSched us, const ChipSolveState *__restrict__ state, const float *__restrict__ beta,
                       const float *__restrict__ R, float *__restrict__ P, const float *__restrict__ dinv,
                       const float *__restrict__ Zb) {
  using SG = Stage32<S>;
  constexpr int TC = SG::TC, TPR = S / 4;
  extern __shared__ __align__(128) unsigned char smem_staged[];
  float *sB = reinterpret_cast<float *>(smem_staged);
  float *sP = sB + S * S;                 // NST staged tiles of P
  float *sZ = sP + NST * SG::FLOATS;      // NST staged tiles of Z (R under PCM 0 and 1)
  grid_release_next();
  grid_wait_prior();
  const int t = threadIdx.x;
  const int jq = t % TPR, cl0 = (t / TPR) * 4;
  const float *zsrc = PCM == 2 ? Zb : R;
  TileWalk pre, cur;
  pre.seek(us, state, (int)blockIdx.x);
  cur = pre;
#pragma unroll
  for (int st = 0; st < NST - 1; ++st) {
    if (pre.valid(us)) {
      stage_tile<S>(sP + st * SG::FLOATS, P, pre.base, pre.end);
      stage_tile<S>(sZ + st * SG::FLOATS, zsrc, pre.base, pre.end);
      pre.next<TC>(us, state);
    }
    cp_async_commit();
  }
  int bchip = -1;
  for (int k = 0; cur.valid(us); ++k) {
    const int sn = (k + NST - 1) % NST, sc = k % NST;
    if (pre.valid(us)) {
      stage_tile<S>(sP + sn * SG::FLOATS, P, pre.base, pre.end);
      stage_tile<S>(sZ + sn * SG::FLOATS, zsrc, pre.base, pre.end);
      pre.next<TC>(us, state);
    }
    cp_async_commit();
    if (cur.chip != bchip) {   // the previous tile's readers of sB passed the trailing barrier
      const float *be = beta + (long long)cur.chip * S * S;
      for (int e = t; e < S * S; e += 256) sB[e] = be[e];
      bchip = cur.chip;
    }
    float di[4];
    if constexpr (PCM == 1) {
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) di[k4] = cur.base + cl0 + k4 < cur.end ? dinv[cur.base + cl0 + k4] : 0.f;
    }
    cp_async_wait<NST - 1>();
    __syncthreads();
    const float *tP = sP + sc * SG::FLOATS, *tZ = sZ + sc * SG::FLOATS;
    float rv[4][4];
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4) {
      vload<float>(rv[k4], tZ + SG::off(cl0 + k4, jq));
      if constexpr (PCM == 1) {
#pragma unroll
        for (int v = 0; v < 4; ++v) rv[k4][v] *= di[k4];
      }
    }
#pragma unroll 2
    for (int iq = 0; iq < TPR; ++iq) {
      float p[4][4], b[4][4];
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4) vload<float>(p[k4], tP + SG::off(cl0 + k4, iq));
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) vload<float>(b[ii], sB + (4 * iq + ii) * S + 4 * jq);
#pragma unroll
      for (int k4 = 0; k4 < 4; ++k4)
#pragma unroll
        for (int ii = 0; ii < 4; ++ii)
#pragma unroll
          for (int v = 0; v < 4; ++v) rv[k4][v] += p[k4][ii] * b[ii][v];
    }
#pragma unroll
    for (int k4 = 0; k4 < 4; ++k4)
      if (cur.base + cl0 + k4 < cur.end) vstore<float>(P + (cur.base + cl0 + k4) * S + 4 * jq, rv[k4]);
    __syncthreads();   // stage sc is refilled in the next iteration
    cur.next<TC>(us, state);
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------- tensor-core P update
// P = Z + P beta on the tensor cores (float32 form, S = 32).  Each CTA walks
// its 128-cell tiles with the next tile's P and Z rows in flight
// (cp.async, coalesced, two stages).  Per tile, thread t owns cell t: it
// splits its P row into tf32 pairs x = hi + lo (hi rounded to nearest,
// lo = x - hi exact in float32) written as K-major operand images without
// swizzle, one thread issues
//   D = P_lo beta_hi + P_hi beta_lo + P_hi beta_hi
// (tcgen05.mma kind::tf32, M = 128, N = 32, K = 8 per instruction, float32
// accumulator in TMEM), and thread t adds its TMEM row to its Z row.  The
// dropped P_lo beta_lo term and the tf32 rounding of the lo parts leave a
// relative error of order 2^-22 per product, the order of float32 rounding.
// Results go back through shared memory for coalesced stores.
constexpr int TCP_M = 128;

struct TcImg32 {
  static constexpr int S = 32;
  static constexpr int SBO = (S / 4) * 128;       // bytes between 8-row groups
  static constexpr int BYTES_A = TCP_M * S * 4;   // one plane of a 128 x 32 operand
  static constexpr int BYTES_B = S * S * 4;       // one plane of the 32 x 32 operand
  // byte offset of element (r, k): 8 x 16-byte core matrices, K-adjacent ones 128 bytes apart
  __device__ static __forceinline__ int off(int r, int k) {
    return (r >> 3) * SBO + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
  }
};

constexpr size_t ptc_smem() {
  // 2 stages x (P, Z) staged tiles, P hi / lo planes, beta^T hi / lo planes, barrier + TMEM slot
  return 4 * (size_t)Stage32<32>::FLOATS * 4 + 2 * (size_t)TcImg32::BYTES_A + 2 * (size_t)TcImg32::BYTES_B + 64;
}

template <int PCM>
__global__ void __launch_bounds__(128, 2)
p_update_tc_kernel(const UnitSched us, ChipSolveState *__restrict__ state, const float *__restrict__ beta,
                   const float *__restrict__ R, float *__restrict__ P, const float *__restrict__ dinv,
                   const float *__restrict__ Zb) {
  constexpr int S = 32, NQ = S / 4;
  using I = TcImg32;
  using SG = Stage32<S>;
  static_assert(SG::TC == TCP_M, "one staged tile per MMA tile");
  constexpr uint32_t TCOLS = 32;
  extern __shared__ __align__(1024) unsigned char smem_tc[];
  float *stP = reinterpret_cast<float *>(smem_tc);      // [2][TC * S] staged P rows
  float *stZ = stP + 2 * SG::FLOATS;                  // [2][TC * S] staged Z rows, then results
  unsigned char *aHi = reinterpret_cast<unsigned char *>(stZ + 2 * SG::FLOATS);
  unsigned char *aLo = aHi + I::BYTES_A;
  unsigned char *bHi = aLo + I::BYTES_A, *bLo = bHi + I::BYTES_B;
  uint64_t *bar = reinterpret_cast<uint64_t *>(bLo + I::BYTES_B);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
  __shared__ int s_fail;
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    mbar_init(bar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, TCOLS);   // before dependents may launch and allocate
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  grid_release_next();
  grid_wait_prior();
  const uint32_t idesc = idesc_tf32(TCP_M, S);
  const float *zsrc = PCM == 2 ? Zb : R;
  // rows [base, base + 128) of P and Z into stage st (128 threads, 8 chunks each per array)
  auto stage = [&](int st, long long base, long long end) {
#pragma unroll
    for (int m = 0; m < SG::TC * NQ / 128; ++m) {
      const int c = t + 128 * m, row = c / NQ, q = c % NQ;
      const bool in = base + row < end;
      const long long g = in ? (base + row) * S + q * 4 : 0;
      cp_async16(stP + st * SG::FLOATS + SG::off(row, q), P + g, in ? 16 : 0);
      cp_async16(stZ + st * SG::FLOATS + SG::off(row, q), zsrc + g, in ? 16 : 0);
    }
  };
  TileWalk pre, cur;
  pre.seek(us, state, (int)blockIdx.x);
  cur = pre;
  if (pre.valid(us)) {
    stage(0, pre.base, pre.end);
    pre.next<TCP_M>(us, state);
  }
  cp_async_commit();
  int bchip = -1, fail_chip = -1;
  uint32_t phase = 0;
  for (int k = 0; cur.valid(us); ++k) {
    const int sc = k & 1;
    const TileWalk after = pre;   // tile k + 1: the walker staged one tile ahead already found it
    if (pre.valid(us)) {
      stage(sc ^ 1, pre.base, pre.end);
      pre.next<TCP_M>(us, state);
    }
    cp_async_commit();
    if (cur.chip != bchip) {   // beta^T planes: B(n, k) = beta(k, n)
      const float *be = beta + (long long)cur.chip * S * S;
      for (int e = t; e < S * S; e += 128) {
        const int kk = e / S, n = e % S;
        const float v = be[e];
        const float hi = tf32_rna(v);
        *reinterpret_cast<float *>(bHi + I::off(n, kk)) = hi;
        *reinterpret_cast<float *>(bLo + I::off(n, kk)) = v - hi;
      }
      bchip = cur.chip;
    }
    float di = 1.f;
    if constexpr (PCM == 1) di = cur.base + t < cur.end ? dinv[cur.base + t] : 0.f;
    cp_async_wait<1>();
    __syncthreads();   // tile k staged by all threads
    const float *tP = stP + sc * SG::FLOATS;
    float *tZ = stZ + sc * SG::FLOATS;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {   // this thread's P row -> hi / lo planes
      const float4 v = *reinterpret_cast<const float4 *>(tP + SG::off(t, q));
      const float4 h = make_float4(tf32_rna(v.x), tf32_rna(v.y), tf32_rna(v.z), tf32_rna(v.w));
      *reinterpret_cast<float4 *>(aHi + I::off(t, 4 * q)) = h;
      *reinterpret_cast<float4 *>(aLo + I::off(t, 4 * q)) = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (t == 0) {
      tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < S / 8; ++ks)   // small terms first
        mma_tf32(tmem, smem_desc(aLo + ks * 256, 128, I::SBO), smem_desc(bHi + ks * 256, 128, I::SBO), idesc,
                 ks > 0 ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < S / 8; ++ks)
        mma_tf32(tmem, smem_desc(aHi + ks * 256, 128, I::SBO), smem_desc(bLo + ks * 256, 128, I::SBO), idesc, 1u);
#pragma unroll
      for (int ks = 0; ks < S / 8; ++ks)
        mma_tf32(tmem, smem_desc(aHi + ks * 256, 128, I::SBO), smem_desc(bHi + ks * 256, 128, I::SBO), idesc, 1u);
      mma_commit(bar);
    }
    float z[S];   // Z row while the MMAs run
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const float4 v = *reinterpret_cast<const float4 *>(tZ + SG::off(t, q));
      z[4 * q] = v.x * di; z[4 * q + 1] = v.y * di; z[4 * q + 2] = v.z * di; z[4 * q + 3] = v.w * di;
    }
    if (!mbar_wait(bar, phase)) s_fail = 1;
    __syncthreads();
    if (s_fail) {
      fail_chip = cur.chip;
      break;
    }
    phase ^= 1;
    tc_fence_after();
    uint32_t d[S];
    BLOCKOA_TMEM_LD32(tmem + ((uint32_t)(warp * 32) << 16), d);
    tmem_wait_ld();
#pragma unroll
    for (int q = 0; q < NQ; ++q)
      *reinterpret_cast<float4 *>(tZ + SG::off(t, q)) =
          make_float4(z[4 * q] + __uint_as_float(d[4 * q]), z[4 * q + 1] + __uint_as_float(d[4 * q + 1]),
                      z[4 * q + 2] + __uint_as_float(d[4 * q + 2]), z[4 * q + 3] + __uint_as_float(d[4 * q + 3]));
    tc_fence_before();
    __syncthreads();
#pragma unroll
    for (int m = 0; m < SG::TC * NQ / 128; ++m) {   // coalesced stores of the new P rows
      const int c = t + 128 * m, row = c / NQ, q = c % NQ;
      if (cur.base + row < cur.end)
        *reinterpret_cast<float4 *>(P + (cur.base + row) * S + q * 4) =
            *reinterpret_cast<const float4 *>(tZ + SG::off(row, q));
    }
    __syncthreads();   // stage sc, the planes and TMEM are reused
    cur = after;
  }
  cp_async_wait<0>();
  if (fail_chip >= 0 && t == 0) {   // MMA completion timed out: report, let it land, release TMEM
    state[fail_chip].status = BLOCKOA_ERR_TIMEOUT;
    state[fail_chip].active = 0;
    mbar_wait(bar, phase);
  }
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TCOLS);
}

// ---------------------------------------------------------------- z-line preconditioning
// Z = M^-1 R with M the part of A that couples the cells of one (x, y)
// column (tridiagonal in z), by the Thomas recurrences with the per-cell
// factors 1/den_z of the assembly:
//   w_z = (r_z + e_z w_{z-1}) / den_z,   z_z = w_z + f_z / den_z z_{z+1},
// e_z = conductance (z-1, z), f_z = conductance (z, z+1).

// Restart: Z = P = M^-1 R.  One thread per (chip column, 16 bytes of columns).
template <typename T, int S>
__global__ void zline_init_kernel(const ChipDev *__restrict__ chips, int n_chips, const int *__restrict__ outer_active,
                                  const T *__restrict__ g, const T *__restrict__ zinv, const T *__restrict__ R,
                                  T *__restrict__ P, T *__restrict__ Zb) {
  constexpr int V = 16 / sizeof(T), NQ = S / V;
  const int c = blockIdx.y;
  if (c >= n_chips || !outer_active[c]) return;
  const ChipDev ch = chips[c];
  const long long nxny = (long long)ch.nx * ch.ny;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < nxny * NQ;
       it += (long long)gridDim.x * blockDim.x) {
    const long long col = it / NQ;
    const int j0 = (int)(it % NQ) * V;
    T w[V], prev[V];
    for (int v = 0; v < V; ++v) prev[v] = T(0);
    T e = T(0);
    for (int z = 0; z < ch.nz; ++z) {   // forward: w_z -> Z (temporary)
      const long long a = ch.off + z * nxny + col;
      const T inv = zinv[a];
      T r[V];
      vload<T>(r, R + a * S + j0);
#pragma unroll
      for (int v = 0; v < V; ++v) w[v] = (r[v] + e * prev[v]) * inv;
      vstore<T>(Zb + a * S + j0, w);
#pragma unroll
      for (int v = 0; v < V; ++v) prev[v] = w[v];
      e = coef_ld(g, a).z;
    }
    for (int z = ch.nz - 2; z >= 0; --z) {   // backward, prev = z_{z+1}
      const long long a = ch.off + z * nxny + col;
      const T fz = coef_ld(g, a).z * zinv[a];
      T ww[V];
      vload<T>(ww, Zb + a * S + j0);
#pragma unroll
      for (int v = 0; v < V; ++v) prev[v] = ww[v] + fz * prev[v];
      vstore<T>(Zb + a * S + j0, prev);
    }
    for (int z = 0; z < ch.nz; ++z) {
      const long long a = ch.off + z * nxny + col;
      T ww[V];
      vload<T>(ww, Zb + a * S + j0);
      vstore<T>(P + a * S + j0, ww);
    }
  }
}

// Column tiles of the z-line update: XT = TC / nz x positions of one y row,
// all z; slot s = z XT + dx of a tile.
struct ColGeom {
  int xt, tiles_x;
  __device__ __forceinline__ ColGeom(const ChipDev &ch, int tc) {
    xt = tc / ch.nz;
    tiles_x = (ch.nx + xt - 1) / xt;
  }
  // global cell of slot s in column tile c (-1 when the slot is outside the chip)
  __device__ __forceinline__ long long cell(const ChipDev &ch, int c, int s) const {
    const int z = s / xt, dx = s % xt;
    const int y = c / tiles_x, x = (c % tiles_x) * xt + dx;
    if (z >= ch.nz || x >= ch.nx) return -1;
    return ch.off + (long long)z * ch.nx * ch.ny + (long long)y * ch.nx + x;
  }
  // the same split in two: per tile, its first cell (z = 0, dx = 0) and the
  // x positions it has inside the chip; per slot, (z, dx)
  __device__ __forceinline__ void tile(const ChipDev &ch, int c, long long &cell0, int &xin) const {
    int y, xb;
    tile(ch, c, cell0, xin, y, xb);
  }
  __device__ __forceinline__ void tile(const ChipDev &ch, int c, long long &cell0, int &xin, int &y, int &xb) const {
    y = c / tiles_x;
    xb = (c - y * tiles_x) * xt;
    cell0 = ch.off + (long long)y * ch.nx + xb;
    xin = ch.nx - xb;
  }
  __device__ __forceinline__ static long long slot_cell(const ChipDev &ch, long long cell0, int xin, int z, int dx) {
    return (z < ch.nz && dx < xin) ? cell0 + (long long)z * ch.nx * ch.ny + dx : -1;
  }
};

// Tridiagonal factors of a column tile's slots into shared memory: e (the
// conductance to z-1), f / den and 1 / den per slot.  fz, fdx: (z, dx) of
// slot t, the calling thread's first slot.
template <typename T, int TC>
__device__ __forceinline__ void zline_factors(const ChipDev &ch, const ColGeom &cg, long long cell0, int xin,
                                              int fz, int fdx, const T *__restrict__ g,
                                              const T *__restrict__ zinv, T *sE, T *sF, T *sI) {
  const int t = threadIdx.x;
  for (int sl = t; sl < TC; sl += 256) {
    const int z = sl == t ? fz : sl / cg.xt, dx = sl == t ? fdx : sl % cg.xt;
    const long long a = ColGeom::slot_cell(ch, cell0, xin, z, dx);
    T e = T(0), f = T(0), iv = T(0);
    if (a >= 0) {
      iv = zinv[a];
      f = coef_ld(g, a).z * iv;
      if (z > 0) e = coef_ld(g, a - (long long)ch.nx * ch.ny).z;
    }
    sE[sl] = e;
    sF[sl] = f;
    sI[sl] = iv;
  }
}

// In place on a transposed [column][slot] tile: every cell column of every
// block column is replaced by M^-1 of it (forward and back substitution of
// the Thomas recurrences), one thread per (block column j, x position dx).
template <typename T, int S, int LD>
__device__ __forceinline__ void zline_solve_tile(T *sV, const T *sE, const T *sF, const T *sI, int nz, int xt) {
  for (int pr = threadIdx.x; pr < S * xt; pr += 256) {
    const int j = pr / xt, dx = pr % xt;
    T *row = sV + j * LD;
    T prev = T(0);
    for (int z = 0; z < nz; ++z) {
      const int sl = z * xt + dx;
      T &val = row[swz<T>(j, sl)];
      prev = (val + sE[sl] * prev) * sI[sl];
      val = prev;
    }
    for (int z = nz - 2; z >= 0; --z) {
      const int sl = z * xt + dx;
      T &val = row[swz<T>(j, sl)];
      prev = val + sF[sl] * prev;
      val = prev;
    }
  }
}

// The update kernel with z-line preconditioning: as update_gram, over column
// tiles (units are ranges of column tiles of one chip).  After X and R are
// updated the tile holds whole cell columns of R_new: the tridiagonal
// solves run in shared memory (one thread per (column of the block, x
// position)), Z is stored for the P update, and W += Q^T Z.
// TWO (two-step z-line): Z1 = M^-1 R_new is stored and ||R_j||^2 flushed; the
// second step, W and the beta tail belong to zline2_kernel.  The float32
// two-step form at 32 columns runs three CTAs per SM (80 registers, ~100
// bytes of spills; measured 38.4 -> 37.5 us a launch on a 131K-cell chip);
// the one-step form spills ~0.5 KB at 80 and keeps two, as do the other
// widths (not measured at three).
template <typename T, int S, bool TWO>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && TWO && S == 32) ? 3 : 2)
update_zline_kernel(const UnitSched us, const ChipDev *__restrict__ chips, const T *__restrict__ g,
                    const T *__restrict__ zinv, const T *__restrict__ P, const T *__restrict__ Q,
                    T *__restrict__ X, T *__restrict__ R, T *__restrict__ Zb, const SmallArgs A) {
  using G = BK<T, S>;
  constexpr int V = G::V;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sP = reinterpret_cast<T *>(smem);
  T *sQ = sP + S * G::LD;
  T *sR = sQ + S * G::LD;
  T *sA = sR + S * G::LD;
  T *sE = sA + S * S;        // per slot: e (conductance to z-1), f / den, 1 / den
  T *sF = sE + G::TC;
  T *sI = sF + G::TC;
  double *red = reinterpret_cast<double *>(smem);   // reused between units
  __shared__ UnitSlot s_unit;
  grid_release_next();
  grid_wait_prior();
  const int t = threadIdx.x;
  const int j0 = (t % G::TPR) * V, cl0 = (t / G::TPR) * 4;
  const int grp = t / G::NT, w = t % G::NT;
  const int i0 = (w / G::NB) * 4, k0 = (w % G::NB) * 4;
  T aw[16], rn[V];
#pragma unroll
  for (int e = 0; e < 16; ++e) aw[e] = T(0);
#pragma unroll
  for (int v = 0; v < V; ++v) rn[v] = T(0);
  int cur = -1, run = 0, run_first = 0;
  SchedLocal sl;   // thread 0: the unit fetched ahead, the last chip checked
  for (;;) {
    const int ui = next_unit(us, A.state, &s_unit, sl, chips);
    const int chip = ui < us.n_units ? s_unit.u.chip : -1;
    if (run > 0 && chip != cur) {
      update_flush<T, S>(aw, rn, red, A, cur, !TWO,
                         A.det_upd ? A.det_upd + (long long)(A.det_ubase[cur] + run_first - unit0(us, cur)) *
                                                     ((TWO ? 0 : S * S) + S)
                                   : nullptr);
      if constexpr (sizeof(T) == 4 && !TWO) {
        if (A.tail && last_flush_of_chip(A.ticket + A.n_chips + cur, run, A.zunit_count[cur]))
          chip_beta<T, S>(A, cur);
      }
#pragma unroll
      for (int e = 0; e < 16; ++e) aw[e] = T(0);
#pragma unroll
      for (int v = 0; v < V; ++v) rn[v] = T(0);
      run = 0;
    }
    if (ui >= us.n_units) break;
    const Unit u = s_unit.u;
    if (u.chip != cur) {
      const T *al = reinterpret_cast<const T *>(A.alpha) + (long long)u.chip * S * S;
      for (int e = t; e < S * S; e += 256) sA[e] = al[e];
    }
    cur = u.chip;
    if (run == 0) run_first = ui;
    ++run;
    const ChipDev ch = s_unit.ch;
    const ColGeom cg(ch, G::TC);
    // (z, dx) of this thread's four slots and of its tridiagonal-factor slot
    int sz[4], sdx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sz[k] = (cl0 + k) / cg.xt;
      sdx[k] = (cl0 + k) - sz[k] * cg.xt;
    }
    const int fz = t / cg.xt, fdx = t - fz * cg.xt;
    for (long long ct = u.begin; ct < u.end; ++ct) {
      long long cell0;
      int xin;
      cg.tile(ch, (int)ct, cell0, xin);
      long long cell[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cell[k] = ColGeom::slot_cell(ch, cell0, xin, sz[k], sdx[k]);
      auto ld = [&](T (&x)[4][V], const T *src) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (cell[k] >= 0) vload<T>(x[k], src + cell[k] * S + j0);
          else {
#pragma unroll
            for (int v = 0; v < V; ++v) x[k][v] = T(0);
          }
        }
      };
      auto st = [&](T *dst, const T (&x)[4][V]) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cell[k] >= 0) vstore<T>(dst + cell[k] * S + j0, x[k]);
      };
      {
        T pv[4][V], qv[4][V];
        ld(pv, P);
        ld(qv, Q);
        put_tile<T, G::LD>(sP, pv, cl0, j0);
        put_tile<T, G::LD>(sQ, qv, cl0, j0);
      }
      zline_factors<T, G::TC>(ch, cg, cell0, xin, fz, fdx, g, zinv, sE, sF, sI);
      T xv[4][V], rv[4][V];
      ld(xv, X);
      ld(rv, R);
      __syncthreads();
#pragma unroll 4
      for (int i = 0; i < S; ++i) {
        T p4[4], q4[4], av[V];
        ld4<T, G::LD>(p4, sP, i, cl0);
        ld4<T, G::LD>(q4, sQ, i, cl0);
        vload<T>(av, sA + i * S + j0);
        if constexpr (sizeof(T) == 4) {   // paired FMAs over adjacent columns
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int v = 0; v < V; v += 2) {
              const float2 a2 = make_float2(av[v], av[v + 1]);
              float2 x2 = __ffma2_rn(make_float2(p4[k], p4[k]), a2, make_float2(xv[k][v], xv[k][v + 1]));
              float2 r2 = __ffma2_rn(make_float2(-q4[k], -q4[k]), a2, make_float2(rv[k][v], rv[k][v + 1]));
              xv[k][v] = x2.x; xv[k][v + 1] = x2.y;
              rv[k][v] = r2.x; rv[k][v + 1] = r2.y;
            }
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k)
#pragma unroll
            for (int v = 0; v < V; ++v) {
              xv[k][v] += p4[k] * av[v];
              rv[k][v] -= q4[k] * av[v];
            }
        }
      }
      st(X, xv);
      st(R, rv);
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int v = 0; v < V; ++v) rn[v] += rv[k][v] * rv[k][v];  // zero outside the chip
      put_tile<T, G::LD>(sR, rv, cl0, j0);
      __syncthreads();
      // Z = M^-1 R_new in place
      zline_solve_tile<T, S, G::LD>(sR, sE, sF, sI, ch.nz, cg.xt);
      __syncthreads();
      {   // store Z (this thread's slots, read back from the transposed tile)
        T zv[4][V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          T z4[4];
          ld4<T, G::LD>(z4, sR, j0 + v, cl0);
#pragma unroll
          for (int k = 0; k < 4; ++k) zv[k][v] = z4[k];
        }
        st(Zb, zv);
      }
      if constexpr (!TWO) gram_tile<T, S>(aw, sQ, sR, i0, k0, grp);
      __syncthreads();
    }
  }
  sched_finish(us);
}

// Second step of the two-step z-line preconditioner (PCM 3):
//   Z = M^-1 (2 R - A Z1),  Z1 = M^-1 R from update_zline_kernel<TWO>,
// i.e. the polynomial p(x) = 2 - x of M^-1 A applied to M^-1 R (symmetric
// positive definite since the z-line splitting puts the spectrum of M^-1 A
// in (0, 2)).  Over the same column tiles: the stencil reads Z1 of the
// neighbouring cells from global memory (complete: the update kernel has
// finished), the tridiagonal solves run in shared memory, Z goes to Zout,
// and W += Q^T Z with the beta tail in the chip's last CTA.  INIT (the
// restart of a refinement pass) writes Z to Zout (= P) and nothing else.
template <typename T, int S, bool INIT>
__global__ void __launch_bounds__(256, 2)
zline2_kernel(const UnitSched us, const ChipDev *__restrict__ chips, const T *__restrict__ g,
              const T *__restrict__ zinv, const T *__restrict__ Z1, const T *__restrict__ R,
              const T *__restrict__ Q, T *__restrict__ Zout, const SmallArgs A) {
  using G = BK<T, S>;
  constexpr int V = G::V;
  extern __shared__ __align__(16) unsigned char smem[];
  T *sQ = reinterpret_cast<T *>(smem);
  T *sR = sQ + S * G::LD;
  T *sE = sR + S * G::LD;
  T *sF = sE + G::TC;
  T *sI = sF + G::TC;
  double *red = reinterpret_cast<double *>(smem);   // reused between units
  __shared__ UnitSlot s_unit;
  grid_release_next();
  grid_wait_prior();
  const int t = threadIdx.x;
  const int j0 = (t % G::TPR) * V, cl0 = (t / G::TPR) * 4;
  const int grp = t / G::NT, w = t % G::NT;
  const int i0 = (w / G::NB) * 4, k0 = (w % G::NB) * 4;
  T aw[16];
#pragma unroll
  for (int e = 0; e < 16; ++e) aw[e] = T(0);
  int cur = -1, run = 0, run_first = 0;
  SchedLocal sl;   // thread 0: the unit fetched ahead, the last chip checked
  for (;;) {
    const int ui = next_unit(us, A.state, &s_unit, sl, chips);
    const int chip = ui < us.n_units ? s_unit.u.chip : -1;
    if constexpr (!INIT) {
      if (run > 0 && chip != cur) {
        gram_flush<T, S>(aw, red,
                         sink(A.wg + (long long)cur * S * S,
                              A.det_z2 ? A.det_z2 + (long long)(A.det_zbase[cur] + run_first - unit0(us, cur)) * S * S
                                       : nullptr),
                         A.diag);
        if constexpr (sizeof(T) == 4) {
          if (A.tail && last_flush_of_chip(A.ticket + A.n_chips + cur, run, A.zunit_count[cur]))
            chip_beta<T, S>(A, cur);
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) aw[e] = T(0);
        run = 0;
      }
    }
    if (ui >= us.n_units) break;
    const Unit u = s_unit.u;
    cur = u.chip;
    if (run == 0) run_first = ui;
    ++run;
    const ChipDev ch = s_unit.ch;
    const ColGeom cg(ch, G::TC);
    const long long nxny = (long long)ch.nx * ch.ny;
    int sz[4], sdx[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      sz[k] = (cl0 + k) / cg.xt;
      sdx[k] = (cl0 + k) - sz[k] * cg.xt;
    }
    const int fz = t / cg.xt, fdx = t - fz * cg.xt;
    for (long long ct = u.begin; ct < u.end; ++ct) {
      long long cell0;
      int xin, y, xb;
      cg.tile(ch, (int)ct, cell0, xin, y, xb);
      long long cell[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) cell[k] = ColGeom::slot_cell(ch, cell0, xin, sz[k], sdx[k]);
      {   // Y = 2 R - A Z1 on this thread's slots, into the transposed tile
        T yv[4][V];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
          for (int v = 0; v < V; ++v) yv[k][v] = T(0);
          const long long a = cell[k];
          if (a >= 0) {
            const int x = xb + sdx[k], z = sz[k];
            T zc[V], rr[V], az[V];
            vload<T>(zc, Z1 + a * S + j0);
            vload<T>(rr, R + a * S + j0);
            stencil_row<T, S>(g, Z1, a, zc, x, y, z, ch.nx, ch.ny, ch.nz, nxny, j0, az);
#pragma unroll
            for (int v = 0; v < V; ++v) yv[k][v] = T(2) * rr[v] - az[v];
          }
        }
        put_tile<T, G::LD>(sR, yv, cl0, j0);
      }
      if constexpr (!INIT) {
        T qv[4][V];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (cell[k] >= 0) vload<T>(qv[k], Q + cell[k] * S + j0);
          else {
#pragma unroll
            for (int v = 0; v < V; ++v) qv[k][v] = T(0);
          }
        }
        put_tile<T, G::LD>(sQ, qv, cl0, j0);
      }
      zline_factors<T, G::TC>(ch, cg, cell0, xin, fz, fdx, g, zinv, sE, sF, sI);
      __syncthreads();
      zline_solve_tile<T, S, G::LD>(sR, sE, sF, sI, ch.nz, cg.xt);
      __syncthreads();
      {   // store Z (this thread's slots, read back from the transposed tile)
        T zv[4][V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          T z4[4];
          ld4<T, G::LD>(z4, sR, j0 + v, cl0);
#pragma unroll
          for (int k = 0; k < 4; ++k) zv[k][v] = z4[k];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (cell[k] >= 0) vstore<T>(Zout + cell[k] * S + j0, zv[k]);
      }
      if constexpr (!INIT) gram_tile<T, S>(aw, sQ, sR, i0, k0, grp);
      __syncthreads();
    }
  }
  sched_finish(us);
}

// ---------------------------------------------------------------- ordered reduction
// Deterministic solves: for every chip c (active ones, given `state`) and
// entry e, the sum over k in [0, count[c]) of slots[(begin[c] + k) * n + e]
// in an order fixed by the sizes alone -- lane l of the entry's warp adds
// k = l, l + 32, ... in turn, then the 32 lane sums combine in a fixed
// butterfly -- written to the entry's accumulator (mode: 0 Gamma then rho,
// 1 ||R_j||^2, 2 W then ||R_j||^2, 3 W, 4 a plain [chip][S] vector).  In
// independent-column solves the off-diagonal Gram entries are zero.
__global__ void ordered_reduce_kernel(const double *__restrict__ slots, int n, const int *__restrict__ begin,
                                      const int *__restrict__ count, const ChipSolveState *__restrict__ state,
                                      int n_chips, int mode, int S, double *__restrict__ a, double *__restrict__ b,
                                      int diag) {
  const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (long long)n_chips * n) return;
  const int c = (int)(wid / n), e = (int)(wid % n);
  if (state && !state[c].active) return;
  const double *p = slots + (long long)begin[c] * n + e;
  double v = 0.0;
  for (int k = lane; k < count[c]; k += 32) v += p[(long long)k * n];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    // the partner's value, added in lane order so both partners hold the same sum
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (lane & o) ? w + v : v + w;
  }
  if (lane != 0) return;
  const int SS = S * S;
  const bool gram_entry = (mode == 0) || ((mode == 2 || mode == 3) && e < SS);
  if (diag && gram_entry) {
    const int k = e % SS;
    if (k / S != k % S) v = 0.0;
  }
  switch (mode) {
    case 0: (e < SS ? a : b)[(long long)c * SS + (e % SS)] = v; break;
    case 1: a[rn2_at(c, S, e)] = v; break;
    case 2: if (e < SS) a[(long long)c * SS + e] = v; else b[rn2_at(c, S, e - SS)] = v; break;
    case 3: a[(long long)c * SS + e] = v; break;
    default: a[(long long)c * S + e] = v; break;
  }
}

cudaError_t launch_ordered_reduce(const double *slots, int n, const int *begin, const int *count,
                                  const ChipSolveState *state, int n_chips, int mode, int S, double *a, double *b,
                                  int diag, cudaStream_t st) {
  const long long threads = (long long)n_chips * n * 32;
  const unsigned blocks = (unsigned)((threads + 255) / 256);
  ordered_reduce_kernel<<<blocks, 256, 0, st>>>(slots, n, begin, count, state, n_chips, mode, S, a, b, diag);
  g_launches += 1;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- glue kernels
// dst[a][j] = src[a][j] for j < s, 0 for s <= j < S (float64).
__global__ void pad_cols_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                long long n, int s, int S) {
  const long long total = n * S;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long a = i / S;
    const int j = (int)(i % S);
    dst[i] = (src && j < s) ? src[a * s + j] : 0.0;
  }
}

__global__ void unpad_cols_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                  long long n, int s, int S) {
  const long long total = n * s;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    dst[i] = src[(i / s) * S + (i % s)];
  }
}

// Squared column norms of a float64 block per chip: out[chip][j] += sum_a v^2.
template <int S>
__global__ void col_norms_kernel(const Unit *__restrict__ units, const double *__restrict__ V,
                                 double *__restrict__ out, double *__restrict__ slot) {
  const Unit u = units[blockIdx.x];
  const int j = threadIdx.x % S;
  const int r0 = threadIdx.x / S;
  constexpr int RPB = 256 / S;
  double s = 0.0;
  for (long long a = u.begin + r0; a < u.end; a += RPB) {
    const double v = V[a * S + j];
    s += v * v;
  }
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x < S) {
    double acc = 0.0;
    for (int k = threadIdx.x; k < 256; k += S) acc += red[k];
    if (slot) slot[(long long)blockIdx.x * S + threadIdx.x] = acc;   // deterministic: ordered reduction
    else atomicAdd(out + (long long)u.chip * S + threadIdx.x, acc);
  }
}

// Start an inner solve on A D = R64: R = R64 / sigma_j, P = R, D = 0.
template <typename T, int S, int PCM>
__global__ void inner_init_kernel(const Unit *__restrict__ units, const int *__restrict__ outer_active,
                                  const double *__restrict__ R64, const double *__restrict__ inv_sigma,
                                  T *__restrict__ R, T *__restrict__ P, T *__restrict__ D,
                                  const T *__restrict__ dinv) {
  const Unit u = units[blockIdx.x];
  if (!outer_active[u.chip]) return;
  const double *is = inv_sigma + (long long)u.chip * S;
  for (long long i = u.begin * S + threadIdx.x; i < u.end * S; i += blockDim.x) {
    const T v = (T)(R64[i] * is[i % S]);
    R[i] = v;
    P[i] = PCM == 1 ? v * dinv[i / S] : v;   // z-line: zline_init_kernel follows
    D[i] = T(0);
  }
}

// X64 += sigma_j D.
template <typename T, int S>
__global__ void accumulate_kernel(const Unit *__restrict__ units, const int *__restrict__ outer_active,
                                  const double *__restrict__ sigma, const T *__restrict__ D,
                                  double *__restrict__ X64) {
  const Unit u = units[blockIdx.x];
  if (!outer_active[u.chip]) return;
  const double *sg = sigma + (long long)u.chip * S;
  for (long long i = u.begin * S + threadIdx.x; i < u.end * S; i += blockDim.x)
    X64[i] += sg[i % S] * (double)D[i];
}

// ---------------------------------------------------------------- workspace
// Launches per block-CG iteration and their timing classes: with the small
// solves in the tails of the Gram kernels (CH = false) three, with the
// Cholesky kernels (CH = true) five.
constexpr int kMaxLoopKernels = 6;
// The two-step z-line form (pc 3) adds the second-step kernel after the update.
constexpr int loop_kernels(bool ch, int pc) { return (ch ? 5 : 3) + (pc == 3 ? 1 : 0); }
constexpr int loop_class(bool ch, int pc, int i) {
  return pc == 3 ? (!ch ? (i == 0 ? KC_SPMM_GRAM : i == 1 ? KC_UPDATE_GRAM : i == 2 ? KC_ZLINE2 : KC_P_UPDATE)
                        : (i == 0 ? KC_SPMM_GRAM : i == 1 ? KC_ALPHA_SOLVE : i == 2 ? KC_UPDATE_GRAM
                                  : i == 3 ? KC_ZLINE2 : i == 4 ? KC_BETA_SOLVE : KC_P_UPDATE))
                 : !ch ? (i == 0 ? KC_SPMM_GRAM : i == 1 ? KC_UPDATE_GRAM : KC_P_UPDATE)
                       : (i == 0 ? KC_SPMM_GRAM : i == 1 ? KC_ALPHA_SOLVE : i == 2 ? KC_UPDATE_GRAM
                                 : i == 3 ? KC_BETA_SOLVE : KC_P_UPDATE);
}

struct SolveWS {
  int S = 0, prec = -1;
  int tune_tpu = 0, tune_ztpu = 0;   // the operator's unit sizes this workspace was built with
  long long n = 0;
  int n_chips = 0;
  // float64 block vectors
  double *B64 = nullptr, *X64 = nullptr, *R64 = nullptr;
  // loop vectors in the loop's precision
  void *D = nullptr, *R = nullptr, *P = nullptr, *Q = nullptr;
  // per-chip small buffers
  double *gram = nullptr, *rho = nullptr, *wg = nullptr, *rn2 = nullptr, *rn64 = nullptr,
         *bn2 = nullptr, *target2 = nullptr, *sigma = nullptr, *inv_sigma = nullptr,
         *ginv = nullptr, *dsc = nullptr,   // small-solve arithmetic type (8 bytes)
         *rinv = nullptr;
  int *perm = nullptr, *rank = nullptr, *outer_active = nullptr;
  int *ticket = nullptr, *unit_count = nullptr, *chip_unit_end = nullptr, *work = nullptr;
  void *alpha = nullptr, *beta = nullptr;
  ChipSolveState *state = nullptr;
  Unit *units = nullptr;        // loop units (contiguous per chip)
  int n_units = 0;
  int grid_spmm = 0, grid_update = 0, grid_pupd = 0;   // persistent CTAs per loop kernel
  Unit *zunits = nullptr;       // column-tile units of the z-line update
  int n_zunits = 0, grid_zupdate = 0, grid_zupdate2 = 0;   // one-step, two-step z-line update
  int *zunit_count = nullptr, *zchip_unit_end = nullptr;
  bool zline_ok = false;        // every chip has nz <= TC
  void *Zb = nullptr;           // z-line Z = M^-1 R in the loop's precision
  void *Zb2 = nullptr;          // two-step z-line: the second step's Z (Zb holds M^-1 R)
  int grid_z2 = 0;              // persistent CTAs of the second-step kernel
  Unit *units_small = nullptr;  // elementwise units
  int n_units_small = 0;
  // host staging (pinned)
  ChipSolveState *h_state = nullptr;
  double *h_small = nullptr;    // [4][chip][S] staging
  int *h_active = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t tev[kMaxLoopKernels + 1] = {};   // recorded around the kernels of each chunk's first iteration
  int graph_iters = 0, graph_maxiter = -1, graph_s = -1, graph_pc = -1, graph_ch = -1, graph_diag = -1;
  double graph_tol = -1.0;
  int graph_det = -1;
  // deterministic solves (allocated by the first one): slot buffers and, per
  // kernel, each chip's [first slot | slot count] ranges
  std::vector<int> h_ucnt, h_zcnt, h_scnt;   // units per chip: loop, column-tile, elementwise
  double *det_spmm = nullptr, *det_upd = nullptr, *det_z2 = nullptr, *det_small = nullptr;
  int *det_rng_s = nullptr, *det_rng_u = nullptr, *det_rng_z = nullptr, *det_rng_small = nullptr;
  int det_pc = -1;              // preconditioner the update slots were laid out for
  std::vector<void *> allocs;
};

void free_solve_ws(void *p) {
  SolveWS *ws = (SolveWS *)p;
  if (!ws) return;
  if (ws->graph) cudaGraphExecDestroy(ws->graph);
  for (cudaEvent_t e : ws->tev)
    if (e) cudaEventDestroy(e);
  if (ws->cap) cudaStreamDestroy(ws->cap);
  for (void *a : ws->allocs) cudaFree(a);
  if (ws->h_state) cudaFreeHost(ws->h_state);
  if (ws->h_small) cudaFreeHost(ws->h_small);
  if (ws->h_active) cudaFreeHost(ws->h_active);
  cudaGetLastError();
  delete ws;
}

template <typename P>
static cudaError_t ws_alloc(SolveWS *ws, P **p, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    ws->allocs.push_back(q);
    *p = (P *)q;
  }
  return e;
}

constexpr size_t cmax(size_t a, size_t b) { return a > b ? a : b; }
template <typename T, int S>
constexpr size_t tail_smem() { return sizeof(T) == 4 ? small_smem_bytes<dfl, S>() : 0; }
template <typename T, int S>
constexpr size_t spmm_smem() {
  return cmax(cmax(3 * tile_bytes<T, S>(), kRedBytes), tail_smem<T, S>());
}
template <typename T, int S>
constexpr size_t update_smem() {
  return cmax(cmax(3 * tile_bytes<T, S>() + S * S * sizeof(T), kRedBytes), tail_smem<T, S>());
}
template <typename T, int S>
constexpr size_t pupdate_smem() { return tile_bytes<T, S>() + S * S * sizeof(T); }

// Resident CTAs per SM from the kernel's registers, threads and shared
// memory against the SM's limits (the largest shared-memory carveout).
template <typename K>
static int resident_ctas(K kernel, int threads, size_t dyn_smem, int device) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return 1;
  int smem_sm = 0, resv = 0, regs_sm = 0, thr_sm = 0;
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
  cudaDeviceGetAttribute(&resv, cudaDevAttrReservedSharedMemoryPerBlock, device);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, device);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, device);
  const long long per_block_smem = (long long)dyn_smem + (long long)fa.sharedSizeBytes + resv;
  const int warps = (threads + 31) / 32;
  const int warp_regs = (fa.numRegs * 32 + 255) / 256 * 256;   // allocation unit: 256 registers per warp
  int n = std::min(thr_sm / threads, 32);
  if (per_block_smem > 0) n = std::min<long long>(n, smem_sm / per_block_smem);
  if (warp_regs > 0) n = std::min(n, regs_sm / (warps * warp_regs));
  return std::max(n, 1);
}
// staged float32 P update: tiles in flight per CTA and its shared memory
constexpr int kPStages = 3;
template <int S>
constexpr size_t pstaged_smem() { return (size_t)S * S * 4 + 2 * (size_t)kPStages * Stage32<S>::FLOATS * 4; }
template <typename T, int S>
constexpr size_t zline2_smem() {
  return cmax(2 * tile_bytes<T, S>() + 3 * BK<T, S>::TC * sizeof(T), cmax(kRedBytes, tail_smem<T, S>()));
}

template <typename T, int S>
constexpr size_t zupdate_smem() {
  return cmax(update_smem<T, S>(), 3 * tile_bytes<T, S>() + S * S * sizeof(T) + 3 * BK<T, S>::TC * sizeof(T));
}

template <typename T, int S, int PCM>
static void set_smem_limits() {
  static bool done = false;
  if (done) return;
  done = true;
  cudaFuncSetAttribute(spmm_gram_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)spmm_smem<T, S>());
  if constexpr (PCM == 2 || PCM == 3) {
    cudaFuncSetAttribute(update_zline_kernel<T, S, PCM == 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)zupdate_smem<T, S>());
    cudaFuncSetAttribute(zline2_kernel<T, S, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)zline2_smem<T, S>());
    cudaFuncSetAttribute(zline2_kernel<T, S, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)zline2_smem<T, S>());
  }
  else
    cudaFuncSetAttribute(update_gram_kernel<T, S, PCM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)update_smem<T, S>());
  constexpr int PP = PCM == 3 ? 2 : PCM;   // the two-step form's P update reads Z like the z-line form
  cudaFuncSetAttribute(p_update_kernel<T, S, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)pupdate_smem<T, S>());
  if constexpr (sizeof(T) == 4 && S == 32) {
    cudaFuncSetAttribute(p_update_tc_kernel<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ptc_smem());
    // two CTAs of ~107 KB per SM need the largest shared-memory carveout
    cudaFuncSetAttribute(p_update_tc_kernel<PP>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
  }
  else if constexpr (sizeof(T) == 4)
    cudaFuncSetAttribute(p_update_staged_kernel<S, PP, kPStages>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)pstaged_smem<S>());
  cudaFuncSetAttribute(chol_alpha_kernel<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)chol_smem_bytes<S>());
}

// One block-CG iteration for every active chip; with `ev`, an event is
// recorded before each kernel and after the last (for live timing).
// `chain` says whether the previous node on the stream is a loop kernel:
// a kernel that follows one is launched chained (programmatic dependent
// launch), so its CTAs are scheduled while the previous kernel drains.
template <typename T, int S, int PCM, bool CH>
static void launch_iteration(const blockoa_operator *op, SolveWS *ws, const SmallArgs &sa,
                             cudaStream_t st, cudaEvent_t *ev, bool &chain) {
  const T *g = sizeof(T) == 4 ? (const T *)op->g32 : (const T *)op->g64;
  const T *dinv = sizeof(T) == 4 ? (const T *)op->dinv32 : (const T *)op->dinv64;
  // external record nodes: the events carry timestamps when the graph runs
  int m = 0;
  auto mark = [&]() {
    if (ev) {
      cudaEventRecordWithFlags(ev[m], st, cudaEventRecordExternal);
      chain = false;
    }
    ++m;
  };
  auto launched = [&]() { chain = true; };
  mark();
  // deterministic solves: static schedules, and each Gram kernel's slots
  // reduced in a fixed order right after it
  const int det = sa.det_spmm != nullptr;
  auto reduce = [&](const double *slots, int n, const int *rng, int mode, double *a, double *b) {
    if (!det) return;
    const long long threads = (long long)ws->n_chips * n * 32;
    ordered_reduce_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
        slots, n, rng, rng + ws->n_chips, ws->state, ws->n_chips, mode, S, a, b, sa.diag);
    chain = false;
  };
  const UnitSched us_s{ws->units, ws->n_units, ws->chip_unit_end, ws->work, det, ws->unit_count};
  const UnitSched us_u{ws->units, ws->n_units, ws->chip_unit_end, ws->work + 2, det, ws->unit_count};
  const UnitSched us_p{ws->units, ws->n_units, ws->chip_unit_end, ws->work + 4, 0, ws->unit_count};
  launch_chained(spmm_gram_kernel<T, S>, ws->grid_spmm, 256, spmm_smem<T, S>(), st, chain,
                 us_s, op->d_chips, g, (const T *)ws->P, (const T *)ws->R, (T *)ws->Q, sa);
  launched();
  reduce(ws->det_spmm, 2 * S * S, ws->det_rng_s, 0, ws->gram, ws->rho);
  if constexpr (CH) {
    mark();
    launch_chained(chol_alpha_kernel<T, S>, ws->n_chips * S, kCholThreads, chol_smem_bytes<S>(), st, chain, sa);
    launched();
  }
  mark();
  if constexpr (PCM == 2 || PCM == 3) {
    const UnitSched us_z{ws->zunits, ws->n_zunits, ws->zchip_unit_end, ws->work + 2, det, ws->zunit_count};
    const T *zinv = sizeof(T) == 4 ? (const T *)op->zinv32 : (const T *)op->zinv64;
    launch_chained(update_zline_kernel<T, S, PCM == 3>, PCM == 3 ? ws->grid_zupdate2 : ws->grid_zupdate, 256,
                   zupdate_smem<T, S>(), st, chain,
                   us_z, op->d_chips, g, zinv, (const T *)ws->P, (const T *)ws->Q, (T *)ws->D, (T *)ws->R,
                   (T *)ws->Zb, sa);
    if constexpr (PCM == 3) {   // second step: Zb2 = M^-1 (2 R - A Zb), W = Q^T Zb2, beta tail
      launched();
      reduce(ws->det_upd, S, ws->det_rng_u, 1, ws->rn2, nullptr);
      mark();
      const UnitSched us_z2{ws->zunits, ws->n_zunits, ws->zchip_unit_end, ws->work + 6, det, ws->zunit_count};
      launch_chained(zline2_kernel<T, S, false>, ws->grid_z2, 256, zline2_smem<T, S>(), st, chain,
                     us_z2, op->d_chips, g, zinv, (const T *)ws->Zb, (const T *)ws->R, (const T *)ws->Q,
                     (T *)ws->Zb2, sa);
      launched();
      reduce(ws->det_z2, S * S, ws->det_rng_z, 3, ws->wg, nullptr);
    } else {
      launched();
      reduce(ws->det_upd, S * S + S, ws->det_rng_u, 2, ws->wg, ws->rn2);
    }
  } else {
    launch_chained(update_gram_kernel<T, S, PCM>, ws->grid_update, 256, update_smem<T, S>(), st, chain,
                   us_u, (const T *)ws->P, (const T *)ws->Q, (T *)ws->D, (T *)ws->R, dinv, sa);
    launched();
    reduce(ws->det_upd, S * S + S, ws->det_rng_u, 2, ws->wg, ws->rn2);
  }
  if constexpr (CH) {
    mark();
    launch_chained(chol_beta_kernel<T, S>, ws->n_chips * S, kCholThreads, 0, st, chain, sa);
    launched();
  }
  mark();
  constexpr int PP = PCM == 3 ? 2 : PCM;   // the two-step form's P update reads its Z like the z-line form
  const void *zfin = PCM == 3 ? ws->Zb2 : ws->Zb;
  if constexpr (sizeof(T) == 4 && S == 32)
    launch_chained(p_update_tc_kernel<PP>, ws->grid_pupd, 128, ptc_smem(), st, chain,
                   us_p, ws->state, (const float *)ws->beta, (const float *)ws->R, (float *)ws->P,
                   (const float *)dinv, (const float *)zfin);
  else if constexpr (sizeof(T) == 4)
    launch_chained(p_update_staged_kernel<S, PP, kPStages>, ws->grid_pupd, 256, pstaged_smem<S>(), st, chain,
                   us_p, ws->state, (const float *)ws->beta, (const float *)ws->R, (float *)ws->P,
                   (const float *)dinv, (const float *)zfin);
  else
    launch_chained(p_update_kernel<T, S, PP>, ws->grid_pupd, 256, pupdate_smem<T, S>(), st, chain,
                   us_p, ws->state, (const T *)ws->beta, (const T *)ws->R, (T *)ws->P, dinv, (const T *)zfin);
  launched();
  mark();
}

// Slot ranges of a persistent loop kernel with a static schedule: CTA b of
// G takes units b, b + G, ..., so min(units, G) CTAs hold partial sums of a
// chip; a chip's slots follow the previous chip's.  rng = [first | count].
static std::vector<int> det_ranges(const std::vector<int> &cnt, int G, long long &total) {
  const int nc = (int)cnt.size();
  std::vector<int> r(2 * (size_t)nc);
  total = 0;
  for (int c = 0; c < nc; ++c) {
    const int k = G > 0 ? std::min(cnt[c], G) : cnt[c];
    r[c] = (int)total;
    r[nc + c] = k;
    total += k;
  }
  return r;
}

// Buffers of deterministic solves for preconditioner pc (allocated once per
// workspace and layout).
template <typename T, int S>
static int det_setup(SolveWS *ws, int pc) {
  if (ws->det_spmm && ws->det_pc == pc) return BLOCKOA_OK;
  const int nc = ws->n_chips;
  auto upload = [&](int **dst, const std::vector<int> &v) -> cudaError_t {
    cudaError_t e = ws_alloc(ws, dst, sizeof(int) * v.size());
    return e == cudaSuccess ? cudaMemcpy(*dst, v.data(), sizeof(int) * v.size(), cudaMemcpyHostToDevice) : e;
  };
  long long ns = 0, nu = 0, nz = 0, nsm = 0;
  const std::vector<int> rs = det_ranges(ws->h_ucnt, ws->grid_spmm, ns);
  const bool zl = pc == 2 || pc == 3;
  const std::vector<int> ru = zl ? det_ranges(ws->h_zcnt, pc == 3 ? ws->grid_zupdate2 : ws->grid_zupdate, nu)
                                 : det_ranges(ws->h_ucnt, ws->grid_update, nu);
  const std::vector<int> rz = det_ranges(ws->h_zcnt, ws->grid_z2, nz);
  std::vector<int> rsm(2 * (size_t)nc);   // elementwise units: one slot per unit, in unit order
  for (int c = 0; c < nc; ++c) {
    rsm[c] = (int)nsm;
    rsm[nc + c] = ws->h_scnt[c];
    nsm += ws->h_scnt[c];
  }
  const size_t upd_n = pc == 3 ? S : (size_t)S * S + S;
  BLOCKOA_CUDA(ws_alloc(ws, &ws->det_spmm, sizeof(double) * std::max<long long>(ns, 1) * 2 * S * S));
  BLOCKOA_CUDA(ws_alloc(ws, &ws->det_upd, sizeof(double) * std::max<long long>(nu, 1) * upd_n));
  BLOCKOA_CUDA(ws_alloc(ws, &ws->det_z2, sizeof(double) * std::max<long long>(nz, 1) * S * S));
  BLOCKOA_CUDA(ws_alloc(ws, &ws->det_small, sizeof(double) * std::max<long long>(nsm, 1) * S));
  BLOCKOA_CUDA(upload(&ws->det_rng_s, rs));
  BLOCKOA_CUDA(upload(&ws->det_rng_u, ru));
  BLOCKOA_CUDA(upload(&ws->det_rng_z, rz));
  BLOCKOA_CUDA(upload(&ws->det_rng_small, rsm));
  ws->det_pc = pc;
  return BLOCKOA_OK;
}

template <typename T, int S>
static int solve_impl(blockoa_operator *op, const double *B, double *X, int s,
                      const blockoa_solve_opts *o, blockoa_solve_stats *stats, cudaStream_t st) {
  const int prec = sizeof(T) == 4 ? BLOCKOA_MIXED : BLOCKOA_FP64;
  const int nc = op->n_chips;
  const long long n = op->n_total;
  SolveWS *ws = (SolveWS *)op->solve_ws;
  if (!ws || ws->S != S || ws->prec != prec || ws->n != n || ws->tune_tpu != op->tune_tpu ||
      ws->tune_ztpu != op->tune_ztpu) {
    free_solve_ws(ws);
    op->solve_ws = nullptr;
    ws = new SolveWS();
    op->solve_ws = ws;
    ws->S = S; ws->prec = prec; ws->n = n; ws->n_chips = nc;
    const size_t blk64 = sizeof(double) * (size_t)n * S, blkT = sizeof(T) * (size_t)n * S;
    const size_t sm = sizeof(double) * (size_t)nc * S * S, sv = sizeof(double) * (size_t)nc * S;
    BLOCKOA_CUDA(ws_alloc(ws, &ws->B64, blk64));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->X64, blk64));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->R64, blk64));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->D, blkT));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->R, blkT));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->P, blkT));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->Q, blkT));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->gram, sm));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->rho, sm));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->wg, sm));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->ginv, sm));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->rinv, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->perm, sizeof(int) * (size_t)nc * S));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->alpha, sizeof(T) * (size_t)nc * S * S));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->beta, sizeof(T) * (size_t)nc * S * S));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->rn2, sv * kRn2Stride));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->rn64, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->bn2, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->target2, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->sigma, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->inv_sigma, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->dsc, sv));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->rank, sizeof(int) * (size_t)nc));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->outer_active, sizeof(int) * (size_t)nc));
    BLOCKOA_CUDA(ws_alloc(ws, &ws->state, sizeof(ChipSolveState) * (size_t)nc));
    // loop units: 1-8 whole tiles of one chip, about 16 per persistent CTA
    using G = BK<T, S>;
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, op->device);
    set_smem_limits<T, S, 0>();
    set_smem_limits<T, S, 1>();
    set_smem_limits<T, S, 2>();
    set_smem_limits<T, S, 3>();
    int occ_s = 1, occ_u = 1, occ_p = 1, occ_z = 1;
    BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, spmm_gram_kernel<T, S>, 256,
                                                               spmm_smem<T, S>()));
    BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_u, update_gram_kernel<T, S, 1>, 256,
                                                               update_smem<T, S>()));
    if constexpr (sizeof(T) == 4 && S == 32)
      occ_p = resident_ctas(p_update_tc_kernel<1>, 128, ptc_smem(), op->device);
    else if constexpr (sizeof(T) == 4)
      BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, p_update_staged_kernel<S, 1, kPStages>,
                                                                 256, pstaged_smem<S>()));
    else
      BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, p_update_kernel<T, S, 1>, 256,
                                                                 pupdate_smem<T, S>()));
    BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_z, update_zline_kernel<T, S, false>, 256,
                                                               zupdate_smem<T, S>()));
    long long tiles = 0;
    for (const ChipDev &cd : op->chips) tiles += (cd.n + G::TC - 1) / G::TC;
    long long tpu = tiles / (16LL * std::max(occ_s, 1) * nsm);
    tpu = std::min<long long>(std::max<long long>(tpu, 1), 8);
    if (op->tune_tpu > 0) tpu = op->tune_tpu;   // chosen by blockoa_autotune or the caller
    ws->tune_tpu = op->tune_tpu;
    ws->tune_ztpu = op->tune_ztpu;
    // chips largest first (longest processing time first): a launch's last
    // units are small ones, so its CTAs finish together
    std::vector<int> order(nc);
    for (int c = 0; c < nc; ++c) order[c] = c;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return op->chips[a].n > op->chips[b].n; });
    std::vector<Unit> units;
    {
      const std::vector<Unit> by_chip = make_units(op, tpu * G::TC);
      std::vector<std::vector<Unit>> per(nc);
      for (const Unit &u : by_chip) per[u.chip].push_back(u);
      for (int c : order) units.insert(units.end(), per[c].begin(), per[c].end());
    }
    ws->n_units = (int)units.size();
    {
      std::vector<int> cnt(nc, 0), uend(nc, 0);
      for (size_t i = 0; i < units.size(); ++i) {
        cnt[units[i].chip] += 1;
        uend[units[i].chip] = (int)i + 1;
      }
      ws->h_ucnt = cnt;
      BLOCKOA_CUDA(ws_alloc(ws, &ws->unit_count, sizeof(int) * (size_t)nc));
      BLOCKOA_CUDA(cudaMemcpy(ws->unit_count, cnt.data(), sizeof(int) * (size_t)nc, cudaMemcpyHostToDevice));
      BLOCKOA_CUDA(ws_alloc(ws, &ws->chip_unit_end, sizeof(int) * (size_t)nc));
      BLOCKOA_CUDA(cudaMemcpy(ws->chip_unit_end, uend.data(), sizeof(int) * (size_t)nc, cudaMemcpyHostToDevice));
      BLOCKOA_CUDA(ws_alloc(ws, &ws->ticket, sizeof(int) * 2 * (size_t)nc));
      BLOCKOA_CUDA(cudaMemset(ws->ticket, 0, sizeof(int) * 2 * (size_t)nc));
      BLOCKOA_CUDA(ws_alloc(ws, &ws->work, sizeof(int) * 8));   // [spmm, update, P update, z-line second step] x 2
      BLOCKOA_CUDA(cudaMemset(ws->work, 0, sizeof(int) * 8));
    }
    BLOCKOA_CUDA(ws_alloc(ws, &ws->units, sizeof(Unit) * units.size()));
    BLOCKOA_CUDA(cudaMemcpy(ws->units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice));
    {   // column-tile units of the z-line update (chips with nz <= TC)
      std::vector<Unit> zu;
      std::vector<int> zcnt(nc, 0), zend(nc, 0);
      long long ztiles = 0;
      for (const ChipDev &cd : op->chips)
        if (cd.nz <= G::TC) ztiles += (long long)cd.ny * ((cd.nx + G::TC / cd.nz - 1) / (G::TC / cd.nz));
      long long ztpu = ztiles / (16LL * std::max(occ_z, 1) * nsm);
      ztpu = std::min<long long>(std::max<long long>(ztpu, 1), 8);
      if (op->tune_ztpu > 0) ztpu = op->tune_ztpu;
      for (int c : order) {
        const ChipDev &cd = op->chips[c];
        if (cd.nz > G::TC) continue;   // no z-line units: such chips cannot use PRECOND_ZLINE
        const int xt = G::TC / cd.nz;
        const long long nt = (long long)cd.ny * ((cd.nx + xt - 1) / xt);
        for (long long b = 0; b < nt; b += ztpu) {
          Unit zz;
          zz.chip = c;
          zz.pad = 0;
          zz.begin = b;
          zz.end = std::min(nt, b + ztpu);
          zu.push_back(zz);
          zcnt[c] += 1;
          zend[c] = (int)zu.size();
        }
      }
      ws->n_zunits = (int)zu.size();
      ws->zline_ok = true;
      for (const ChipDev &cd : op->chips) ws->zline_ok = ws->zline_ok && cd.nz <= G::TC;
      BLOCKOA_CUDA(ws_alloc(ws, &ws->zunits, sizeof(Unit) * std::max<size_t>(zu.size(), 1)));
      if (!zu.empty())
        BLOCKOA_CUDA(cudaMemcpy(ws->zunits, zu.data(), sizeof(Unit) * zu.size(), cudaMemcpyHostToDevice));
      BLOCKOA_CUDA(ws_alloc(ws, &ws->zunit_count, sizeof(int) * (size_t)nc));
      BLOCKOA_CUDA(cudaMemcpy(ws->zunit_count, zcnt.data(), sizeof(int) * (size_t)nc, cudaMemcpyHostToDevice));
      ws->h_zcnt = zcnt;
      BLOCKOA_CUDA(ws_alloc(ws, &ws->zchip_unit_end, sizeof(int) * (size_t)nc));
      BLOCKOA_CUDA(cudaMemcpy(ws->zchip_unit_end, zend.data(), sizeof(int) * (size_t)nc, cudaMemcpyHostToDevice));
      ws->grid_zupdate = (int)std::max<long long>(1, std::min<long long>(ws->n_zunits, (long long)std::max(occ_z, 1) * nsm));
      int occ_z2u = 1;
      BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_z2u, update_zline_kernel<T, S, true>, 256,
                                                                 zupdate_smem<T, S>()));
      ws->grid_zupdate2 = (int)std::max<long long>(1, std::min<long long>(ws->n_zunits, (long long)std::max(occ_z2u, 1) * nsm));
      BLOCKOA_CUDA(ws_alloc(ws, &ws->Zb, sizeof(T) * (size_t)n * S));
      BLOCKOA_CUDA(ws_alloc(ws, &ws->Zb2, sizeof(T) * (size_t)n * S));
      int occ_z2 = 1;
      BLOCKOA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_z2, zline2_kernel<T, S, false>, 256,
                                                                 zline2_smem<T, S>()));
      ws->grid_z2 = (int)std::max<long long>(1, std::min<long long>(ws->n_zunits, (long long)std::max(occ_z2, 1) * nsm));
    }
    ws->grid_spmm = (int)std::min<long long>(ws->n_units, (long long)std::max(occ_s, 1) * nsm);
    ws->grid_update = (int)std::min<long long>(ws->n_units, (long long)std::max(occ_u, 1) * nsm);
    ws->grid_pupd = (int)std::min<long long>(ws->n_units, (long long)std::max(occ_p, 1) * nsm);
    std::vector<Unit> us = make_units(op, 256);   // element-wise set-up kernels: ~512 CTAs on a 131K-cell chip
    ws->n_units_small = (int)us.size();
    ws->h_scnt.assign(nc, 0);
    for (const Unit &u : us) ws->h_scnt[u.chip] += 1;
    BLOCKOA_CUDA(ws_alloc(ws, &ws->units_small, sizeof(Unit) * us.size()));
    BLOCKOA_CUDA(cudaMemcpy(ws->units_small, us.data(), sizeof(Unit) * us.size(), cudaMemcpyHostToDevice));
    BLOCKOA_CUDA(cudaMallocHost((void **)&ws->h_state, sizeof(ChipSolveState) * nc));
    BLOCKOA_CUDA(cudaMallocHost((void **)&ws->h_small, sizeof(double) * 4 * (size_t)nc * S));
    BLOCKOA_CUDA(cudaMallocHost((void **)&ws->h_active, sizeof(int) * nc));
    BLOCKOA_CUDA(cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking));
    BLOCKOA_CUDA(cudaMemset(ws->gram, 0, sm));
    BLOCKOA_CUDA(cudaMemset(ws->rho, 0, sm));
    BLOCKOA_CUDA(cudaMemset(ws->wg, 0, sm));
    BLOCKOA_CUDA(cudaMemset(ws->rn2, 0, sv * kRn2Stride));
    BLOCKOA_CUDA(cudaMemset(ws->ginv, 0, sm));
    BLOCKOA_CUDA(cudaMemset(ws->rank, 0, sizeof(int) * (size_t)nc));
  }

  const double rtol = o->rtol;
  const int maxiter = o->maxiter;
  const double inner_rtol = prec == BLOCKOA_MIXED ? (o->inner_rtol > 0 ? o->inner_rtol : 1e-4) : 0.0;
  const int max_refine = o->max_refine > 0 ? o->max_refine : 12;
  const double tol = o->deflate_tol > 0 ? o->deflate_tol : (prec == BLOCKOA_MIXED ? 1e-6 : 1e-14);
  const int check_every = o->check_every > 0 ? o->check_every : 8;
  const int pc = o->precond == BLOCKOA_PRECOND_JACOBI ? 1 : o->precond == BLOCKOA_PRECOND_ZLINE ? 2
               : o->precond == BLOCKOA_PRECOND_ZLINE2 ? 3 : 0;
  if (pc >= 2 && !ws->zline_ok) {
    set_last_error(cudaErrorInvalidValue, "block_solve: PRECOND_ZLINE needs nz <= the tile cells of every chip");
    return BLOCKOA_ERR_INVALID;
  }
  // the float64 form always factors by Cholesky in kernels of their own
  // deterministic solves run the float64 Cholesky small solves (the tails
  // of the sweep form add to the accumulators while other CTAs flush)
  const bool det = o->deterministic != 0;
  const bool ch = prec == BLOCKOA_FP64 || o->small_solve == BLOCKOA_SMALL_FP64_CHOLESKY || det;
  if (det) {
    const int rc = det_setup<T, S>(ws, pc);
    if (rc) return rc;
  }

  SmallArgs sa;
  sa.det_spmm = det ? ws->det_spmm : nullptr;
  sa.det_upd = det ? ws->det_upd : nullptr;
  sa.det_z2 = det ? ws->det_z2 : nullptr;
  sa.det_base = ws->det_rng_s;
  sa.det_ubase = ws->det_rng_u;
  sa.det_zbase = ws->det_rng_z;
  sa.state = ws->state; sa.gram = ws->gram; sa.rho = ws->rho; sa.wg = ws->wg; sa.rn2 = ws->rn2;
  sa.target2 = ws->target2; sa.ginv = ws->ginv; sa.dsc = ws->dsc; sa.rank = ws->rank;
  sa.rinv = ws->rinv; sa.perm = ws->perm;
  sa.alpha = ws->alpha; sa.beta = ws->beta;
  sa.ticket = ws->ticket; sa.unit_count = ws->unit_count; sa.zunit_count = ws->zunit_count;
  sa.n_chips = nc; sa.tail = ch ? 0 : 1;
  sa.diag = o->independent ? 1 : 0;
  sa.s = s; sa.maxiter = maxiter; sa.tol = tol;

  // Build (or reuse) the graph of `check_every` iterations.
  if (!ws->graph || ws->graph_iters != check_every || ws->graph_maxiter != maxiter ||
      ws->graph_s != s || ws->graph_tol != tol || ws->graph_pc != pc || ws->graph_ch != (int)ch ||
      ws->graph_diag != sa.diag || ws->graph_det != (int)det) {
    if (ws->graph) { cudaGraphExecDestroy(ws->graph); ws->graph = nullptr; }
    cudaGraph_t graph = nullptr;
    for (int i = 0; i <= kMaxLoopKernels; ++i)
      if (!ws->tev[i]) BLOCKOA_CUDA(cudaEventCreate(&ws->tev[i]));
    BLOCKOA_CUDA(cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal));
    bool chain = false;   // the graph's first kernel waits for whatever precedes the launch
    for (int k = 0; k < check_every; ++k) {
      cudaEvent_t *ev = k == 0 ? ws->tev : nullptr;
      if (ch) {
        if (pc == 1) launch_iteration<T, S, 1, true>(op, ws, sa, ws->cap, ev, chain);
        else if (pc == 2) launch_iteration<T, S, 2, true>(op, ws, sa, ws->cap, ev, chain);
        else if (pc == 3) launch_iteration<T, S, 3, true>(op, ws, sa, ws->cap, ev, chain);
        else launch_iteration<T, S, 0, true>(op, ws, sa, ws->cap, ev, chain);
      } else if constexpr (sizeof(T) == 4) {
        if (pc == 1) launch_iteration<T, S, 1, false>(op, ws, sa, ws->cap, ev, chain);
        else if (pc == 2) launch_iteration<T, S, 2, false>(op, ws, sa, ws->cap, ev, chain);
        else if (pc == 3) launch_iteration<T, S, 3, false>(op, ws, sa, ws->cap, ev, chain);
        else launch_iteration<T, S, 0, false>(op, ws, sa, ws->cap, ev, chain);
      }
    }
    cudaError_t e = cudaStreamEndCapture(ws->cap, &graph);
    if (e != cudaSuccess) return cuda_status(e, "capture block-CG iterations");
    e = cudaGraphInstantiate(&ws->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status(e, "instantiate block-CG graph");
    ws->graph_iters = check_every;
    ws->graph_maxiter = maxiter;
    ws->graph_s = s;
    ws->graph_tol = tol;
    ws->graph_pc = pc;
    ws->graph_ch = (int)ch;
    ws->graph_diag = sa.diag;
    ws->graph_det = (int)det;
  }

  // Inputs: padded B and X0, ||B_j||^2.
  const unsigned eb = (unsigned)std::min<long long>((n * S + 255) / 256, 4096);
  g_launches += 3;
  pad_cols_kernel<<<eb, 256, 0, st>>>(B, ws->B64, n, s, S);
  pad_cols_kernel<<<eb, 256, 0, st>>>(o->x0, ws->X64, n, s, S);
  BLOCKOA_CUDA(cudaMemsetAsync(ws->bn2, 0, sizeof(double) * nc * S, st));
  col_norms_kernel<S><<<ws->n_units_small, 256, 0, st>>>(ws->units_small, ws->B64, ws->bn2,
                                                          det ? ws->det_small : nullptr);
  BLOCKOA_CUDA(cudaGetLastError());
  if (det) BLOCKOA_CUDA(launch_ordered_reduce(ws->det_small, S, ws->det_rng_small, ws->det_rng_small + nc, nullptr,
                                              nc, 4, S, ws->bn2, nullptr, 0, st));
  std::vector<double> bn2((size_t)nc * S);
  BLOCKOA_CUDA(read_small(ws->h_small, ws->bn2, sizeof(double) * nc * S, st));
  BLOCKOA_CUDA(cudaStreamSynchronize(st));
  memcpy(bn2.data(), ws->h_small, sizeof(double) * nc * S);

  std::vector<int> status(nc, BLOCKOA_OK), done(nc, 0), iters(nc, 0), refine(nc, 0), defl(nc, 0);
  std::vector<double> relres(nc, 0.0), prev_relres(nc, INFINITY);
  std::vector<double> sig((size_t)nc * S), isig((size_t)nc * S), tgt((size_t)nc * S);
  for (int step = 0;; ++step) {
    // True float64 residual R64 = B - A X64 and its column norms (from a
    // zero start the first one is B itself).
    if (step == 0 && !o->x0) {
      BLOCKOA_CUDA(cudaMemcpyAsync(ws->R64, ws->B64, sizeof(double) * (size_t)n * S, cudaMemcpyDeviceToDevice, st));
      BLOCKOA_CUDA(cudaMemcpyAsync(ws->rn64, ws->bn2, sizeof(double) * nc * S, cudaMemcpyDeviceToDevice, st));
    } else {
      BLOCKOA_CUDA(cudaMemsetAsync(ws->rn64, 0, sizeof(double) * nc * S, st));
      int rc = launch_residual64(op, ws->B64, ws->X64, ws->R64, S, ws->rn64, st, det);
      if (rc) return rc;
    }
    BLOCKOA_CUDA(read_small(ws->h_small, ws->rn64, sizeof(double) * nc * S, st));
    BLOCKOA_CUDA(cudaStreamSynchronize(st));
    int n_active = 0;
    for (int c = 0; c < nc; ++c) {
      double worst = 0.0;
      bool conv = true, finite = true;
      for (int j = 0; j < S; ++j) {
        const double r2 = ws->h_small[(size_t)c * S + j], b2 = bn2[(size_t)c * S + j];
        if (!std::isfinite(r2)) finite = false;
        const double rel = b2 > 0 ? std::sqrt(r2 / b2) : (r2 > 0 ? INFINITY : 0.0);
        worst = std::max(worst, rel);
        if (!(rel <= rtol)) conv = false;
        const double sg = std::sqrt(r2);
        sig[(size_t)c * S + j] = sg;
        isig[(size_t)c * S + j] = sg > 0 ? 1.0 / sg : 0.0;
        double t_in = sg > 0 ? rtol * std::sqrt(b2) / sg : 1.0;
        if (prec == BLOCKOA_MIXED) t_in = std::max(inner_rtol, 0.5 * t_in);
        tgt[(size_t)c * S + j] = t_in * t_in;
      }
      relres[c] = worst;
      if (done[c]) continue;
      if (!finite) { status[c] = BLOCKOA_ERR_BREAKDOWN; done[c] = 1; continue; }
      if (conv) { status[c] = BLOCKOA_OK; done[c] = 1; continue; }
      // Give up when the iteration budget is spent, or when a refinement
      // step failed to halve the true residual (float64 attainable accuracy).
      if (refine[c] >= max_refine || iters[c] >= maxiter || (refine[c] > 0 && worst > 0.5 * prev_relres[c])) {
        status[c] = BLOCKOA_ERR_NOT_CONVERGED;
        done[c] = 1;
        continue;
      }
      prev_relres[c] = worst;
      ++n_active;
    }
    if (n_active == 0) break;
    // Upload sigma, targets and chip states for the inner solve.
    for (int c = 0; c < nc; ++c) {
      ws->h_active[c] = !done[c];
      ChipSolveState &cs = ws->h_state[c];
      memset(&cs, 0, sizeof(cs));
      cs.active = !done[c];
      cs.status = BLOCKOA_OK;
      cs.iters = iters[c];
      cs.deflated = defl[c];
    }
    double *stage = ws->h_small + (size_t)nc * S;
    memcpy(stage, sig.data(), sizeof(double) * nc * S);
    memcpy(stage + (size_t)nc * S, isig.data(), sizeof(double) * nc * S);
    memcpy(stage + 2 * (size_t)nc * S, tgt.data(), sizeof(double) * nc * S);
    BLOCKOA_CUDA(cudaMemcpyAsync(ws->sigma, stage, sizeof(double) * nc * S, cudaMemcpyHostToDevice, st));
    BLOCKOA_CUDA(cudaMemcpyAsync(ws->inv_sigma, stage + (size_t)nc * S, sizeof(double) * nc * S, cudaMemcpyHostToDevice, st));
    BLOCKOA_CUDA(cudaMemcpyAsync(ws->target2, stage + 2 * (size_t)nc * S, sizeof(double) * nc * S, cudaMemcpyHostToDevice, st));
    BLOCKOA_CUDA(cudaMemcpyAsync(ws->outer_active, ws->h_active, sizeof(int) * nc, cudaMemcpyHostToDevice, st));
    BLOCKOA_CUDA(cudaMemcpyAsync(ws->state, ws->h_state, sizeof(ChipSolveState) * nc, cudaMemcpyHostToDevice, st));
    {
      const size_t sm = sizeof(double) * (size_t)nc * S * S, sv = sizeof(double) * (size_t)nc * S;
      BLOCKOA_CUDA(cudaMemsetAsync(ws->gram, 0, sm, st));
      BLOCKOA_CUDA(cudaMemsetAsync(ws->rho, 0, sm, st));
      BLOCKOA_CUDA(cudaMemsetAsync(ws->wg, 0, sm, st));
      BLOCKOA_CUDA(cudaMemsetAsync(ws->rn2, 0, sv * kRn2Stride, st));
      BLOCKOA_CUDA(cudaMemsetAsync(ws->ticket, 0, sizeof(int) * 2 * (size_t)nc, st));
      BLOCKOA_CUDA(cudaMemsetAsync(ws->work, 0, sizeof(int) * 8, st));
    }
    g_launches += 2;
    {
      const T *dinv = sizeof(T) == 4 ? (const T *)op->dinv32 : (const T *)op->dinv64;
      if (pc == 1)
        inner_init_kernel<T, S, 1><<<ws->n_units_small, 256, 0, st>>>(
            ws->units_small, ws->outer_active, ws->R64, ws->inv_sigma, (T *)ws->R, (T *)ws->P,
            (T *)ws->D, dinv);
      else
        inner_init_kernel<T, S, 0><<<ws->n_units_small, 256, 0, st>>>(
            ws->units_small, ws->outer_active, ws->R64, ws->inv_sigma, (T *)ws->R, (T *)ws->P,
            (T *)ws->D, dinv);
      if (pc >= 2) {   // P = Z = M^-1 R
        long long maxcols = 1;
        for (const ChipDev &cd : op->chips) maxcols = std::max<long long>(maxcols, (long long)cd.nx * cd.ny);
        const int nq = S / (16 / (int)sizeof(T));
        dim3 zg((unsigned)std::min<long long>((maxcols * nq + 255) / 256, 2048), (unsigned)nc);
        const T *gco = sizeof(T) == 4 ? (const T *)op->g32 : (const T *)op->g64;
        const T *zinv = sizeof(T) == 4 ? (const T *)op->zinv32 : (const T *)op->zinv64;
        zline_init_kernel<T, S><<<zg, 256, 0, st>>>(op->d_chips, nc, ws->outer_active, gco, zinv,
                                                   (const T *)ws->R, (T *)ws->P, (T *)ws->Zb);
        g_launches += 1;
        if (pc == 3) {   // two-step: P = Z = M^-1 (2 R - A M^-1 R)
          const UnitSched us_z2{ws->zunits, ws->n_zunits, ws->zchip_unit_end, ws->work + 6, 0, ws->zunit_count};
          zline2_kernel<T, S, true><<<ws->grid_z2, 256, zline2_smem<T, S>(), st>>>(
              us_z2, op->d_chips, gco, zinv, (const T *)ws->Zb, (const T *)ws->R, (const T *)ws->Q,
              (T *)ws->P, sa);
          g_launches += 1;
        }
      }
    }
    BLOCKOA_CUDA(cudaGetLastError());
    // Inner block-CG iterations, polled every `check_every` iterations.
    for (int poll = 0;; ++poll) {
      if (op->inject_chip >= 0 && op->inject_chip < nc && poll == op->inject_after) {
        // test support: the chip's device state as a device-side wait that
        // gave up would leave it (status set, chip inactive), between polls
        ChipSolveState &cs = ws->h_state[op->inject_chip];
        memset(&cs, 0, sizeof(cs));
        cs.status = op->inject_status;
        cs.active = 0;
        BLOCKOA_CUDA(cudaMemcpyAsync(ws->state + op->inject_chip, &cs, sizeof(cs), cudaMemcpyHostToDevice, st));
        BLOCKOA_CUDA(cudaStreamSynchronize(st));
        op->inject_chip = -1;
      }
      g_launches += (long long)(loop_kernels(ch, pc) + (det ? (pc == 3 ? 3 : 2) : 0)) * check_every;
      for (int i = 0; i < loop_kernels(ch, pc); ++i) add_launches(op, loop_class(ch, pc, i), check_every);
      BLOCKOA_CUDA(cudaGraphLaunch(ws->graph, st));
      BLOCKOA_CUDA(read_small(ws->h_state, ws->state, sizeof(ChipSolveState) * nc, st));
      BLOCKOA_CUDA(cudaStreamSynchronize(st));
      for (int i = 0; i < loop_kernels(ch, pc); ++i) {   // live timing of this chunk's first iteration
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ws->tev[i], ws->tev[i + 1]) == cudaSuccess)
          add_time(op, loop_class(ch, pc, i), ms);
        else
          cudaGetLastError();
      }
      bool any = false;
      for (int c = 0; c < nc; ++c) any = any || ws->h_state[c].active;
      if (!any) break;
    }
    accumulate_kernel<T, S><<<ws->n_units_small, 256, 0, st>>>(ws->units_small, ws->outer_active,
                                                               ws->sigma, (const T *)ws->D, ws->X64);
    BLOCKOA_CUDA(cudaGetLastError());
    for (int c = 0; c < nc; ++c) {
      if (done[c]) continue;
      const ChipSolveState &cs = ws->h_state[c];
      iters[c] = cs.iters;
      defl[c] = cs.deflated;
      refine[c] += 1;
      if (cs.status != BLOCKOA_OK) { status[c] = cs.status; done[c] = 1; }   // breakdown or a device wait timed out
    }
  }
  g_launches += 1;
  unpad_cols_kernel<<<eb, 256, 0, st>>>(ws->X64, X, n, s, S);
  BLOCKOA_CUDA(cudaGetLastError());
  BLOCKOA_CUDA(cudaStreamSynchronize(st));
  int worst = BLOCKOA_OK;
  for (int c = 0; c < nc; ++c) {
    stats[c].status = status[c];
    stats[c].iters = iters[c];
    stats[c].refine_steps = refine[c];
    stats[c].deflated_cols = defl[c];
    stats[c].relres_max = relres[c];
    if (status[c] != BLOCKOA_OK && (worst == BLOCKOA_OK || status[c] == BLOCKOA_ERR_BREAKDOWN))
      worst = status[c];
  }
  return worst;
}

}  // namespace blockoa

using namespace blockoa;

extern "C" int blockoa_block_solve(blockoa_operator *op, const double *B, double *X, int s,
                                   const blockoa_solve_opts *opts, blockoa_solve_stats *stats,
                                   blockoa_stream stream) {
  if (!op || !opts || !stats || s < 0 || s > 64) return BLOCKOA_ERR_INVALID;
  for (int c = 0; c < op->n_chips; ++c) {
    stats[c].status = BLOCKOA_ERR_INVALID;
    stats[c].iters = stats[c].refine_steps = stats[c].deflated_cols = 0;
    stats[c].relres_max = 0.0;
  }
  if (!(opts->rtol > 0.0) || opts->maxiter < 0) return BLOCKOA_ERR_INVALID;
  if (opts->precision != BLOCKOA_FP64 && opts->precision != BLOCKOA_MIXED) return BLOCKOA_ERR_INVALID;
  if (opts->precond != BLOCKOA_PRECOND_NONE && opts->precond != BLOCKOA_PRECOND_JACOBI &&
      opts->precond != BLOCKOA_PRECOND_ZLINE && opts->precond != BLOCKOA_PRECOND_ZLINE2)
    return BLOCKOA_ERR_INVALID;
  if (opts->small_solve != BLOCKOA_SMALL_AUTO && opts->small_solve != BLOCKOA_SMALL_FP64_CHOLESKY)
    return BLOCKOA_ERR_INVALID;
  if (opts->deterministic != 0 && opts->deterministic != 1) return BLOCKOA_ERR_INVALID;
  if (s == 0) {
    for (int c = 0; c < op->n_chips; ++c) stats[c].status = BLOCKOA_OK;
    return BLOCKOA_OK;
  }
  if (!B || !X) return BLOCKOA_ERR_INVALID;
  const int S = s <= 8 ? 8 : s <= 16 ? 16 : s <= 32 ? 32 : 64;
  cudaStream_t st = (cudaStream_t)stream;
  if (opts->precision == BLOCKOA_FP64) {
    switch (S) {
      case 8: return solve_impl<double, 8>(op, B, X, s, opts, stats, st);
      case 16: return solve_impl<double, 16>(op, B, X, s, opts, stats, st);
      case 32: return solve_impl<double, 32>(op, B, X, s, opts, stats, st);
      default: return solve_impl<double, 64>(op, B, X, s, opts, stats, st);
    }
  }
  switch (S) {
    case 8: return solve_impl<float, 8>(op, B, X, s, opts, stats, st);
    case 16: return solve_impl<float, 16>(op, B, X, s, opts, stats, st);
    case 32: return solve_impl<float, 32>(op, B, X, s, opts, stats, st);
    default: return solve_impl<float, 64>(op, B, X, s, opts, stats, st);
  }
}


extern "C" int blockoa_inject_chip_status(blockoa_operator *op, int chip, int status, int after_polls) {
  if (!op || chip < 0 || chip >= op->n_chips || after_polls < 0 || status <= BLOCKOA_OK ||
      status > BLOCKOA_ERR_OOM)
    return BLOCKOA_ERR_INVALID;
  op->inject_chip = chip;
  op->inject_status = status;
  op->inject_after = after_polls;
  return BLOCKOA_OK;
}

// ---------------------------------------------------------------- autotuning
namespace blockoa {
// Deterministic positive right-hand sides for timing runs.
__global__ void tune_rhs_kernel(double *B, long long total) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    B[i] = 1.0 + 0.25 * (double)((unsigned long long)(i * 2654435761LL) % 1024ull) / 1024.0;
}
}  // namespace blockoa

extern "C" int blockoa_set_tuning(blockoa_operator *op, const blockoa_tuning *t) {
  if (!op || !t || t->tiles_per_unit < 0 || t->tiles_per_unit > 64 || t->ztiles_per_unit < 0 ||
      t->ztiles_per_unit > 64)
    return BLOCKOA_ERR_INVALID;
  op->tune_tpu = t->tiles_per_unit;
  op->tune_ztpu = t->ztiles_per_unit;
  return BLOCKOA_OK;
}

extern "C" int blockoa_get_tuning(const blockoa_operator *op, blockoa_tuning *t) {
  if (!op || !t) return BLOCKOA_ERR_INVALID;
  t->tiles_per_unit = op->tune_tpu;
  t->ztiles_per_unit = op->tune_ztpu;
  t->ms_per_iter = 0.0;
  return BLOCKOA_OK;
}

extern "C" int blockoa_autotune(blockoa_operator *op, int s, int precision, int precond, blockoa_tuning *out,
                                blockoa_stream stream) {
  if (!op || !out || s < 1 || s > 64) return BLOCKOA_ERR_INVALID;
  if (precision != BLOCKOA_FP64 && precision != BLOCKOA_MIXED) return BLOCKOA_ERR_INVALID;
  if (precond < BLOCKOA_PRECOND_NONE || precond > BLOCKOA_PRECOND_ZLINE2) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const long long total = op->n_total * s;
  void *B = nullptr, *X = nullptr;
  int rc = pool_alloc(op, &B, sizeof(double) * total, st);
  if (!rc) rc = pool_alloc(op, &X, sizeof(double) * total, st);
  auto done = [&](int code) {
    pool_free(B, st);
    pool_free(X, st);
    cudaStreamSynchronize(st);
    return code;
  };
  if (rc) return done(rc);
  tune_rhs_kernel<<<1024, 256, 0, st>>>((double *)B, total);
  g_launches += 1;
  std::vector<blockoa_solve_stats> stats(op->n_chips);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    return done(BLOCKOA_ERR_CUDA);
  }
  // time of a solve that runs exactly `iters` block iterations (unreachable tolerance)
  auto run = [&](int iters, float &ms) -> int {
    blockoa_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.rtol = 1e-300;
    o.maxiter = iters;
    o.precision = precision;
    o.precond = precond;
    o.check_every = 8;
    int r = blockoa_block_solve(op, (const double *)B, (double *)X, s, &o, stats.data(), stream);   // warm: workspace, graph
    if (r != BLOCKOA_OK && r != BLOCKOA_ERR_NOT_CONVERGED) return r;
    cudaEventRecord(e0, st);
    r = blockoa_block_solve(op, (const double *)B, (double *)X, s, &o, stats.data(), stream);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    return (r == BLOCKOA_OK || r == BLOCKOA_ERR_NOT_CONVERGED) ? BLOCKOA_OK : r;
  };
  // per-iteration cost with the set-up and the refinement step cancelled
  auto per_iter = [&](double &ms_it) -> int {
    float a = 0.f, b = 0.f;
    int r = run(8, a);
    if (!r) r = run(24, b);
    ms_it = (b - a) / 16.0;
    return r;
  };
  const int saved_tpu = op->tune_tpu, saved_ztpu = op->tune_ztpu;
  int best_tpu = 0, best_ztpu = 0;
  double best = 1e30;
  static const int cands[] = {1, 2, 4, 8, 16, 32};
  for (int c : cands) {
    op->tune_tpu = c;
    op->tune_ztpu = saved_ztpu;
    double ms = 0.0;
    if ((rc = per_iter(ms))) break;
    if (ms < best) { best = ms; best_tpu = c; }
  }
  best_ztpu = saved_ztpu;   // the z-line unit size the first search ran with
  if (!rc && precond >= BLOCKOA_PRECOND_ZLINE) {
    for (int c : cands) {
      op->tune_tpu = best_tpu;
      op->tune_ztpu = c;
      double ms = 0.0;
      if ((rc = per_iter(ms))) break;
      if (ms < best) {
        best = ms;
        best_ztpu = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) {
    op->tune_tpu = saved_tpu;
    op->tune_ztpu = saved_ztpu;
    return done(rc);
  }
  op->tune_tpu = best_tpu;
  op->tune_ztpu = best_ztpu;
  out->tiles_per_unit = best_tpu;
  out->ztiles_per_unit = best_ztpu;
  out->ms_per_iter = best;
  return done(BLOCKOA_OK);
}

