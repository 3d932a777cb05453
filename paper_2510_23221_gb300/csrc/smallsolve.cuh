// Small s x s solves of the block-CG iteration (Eq. 4, Sec. III-A).
//
// Per chip and iteration, with D = diag(Gamma)^-1/2 (Jacobi scaling) and
// G = D Gamma D (unit diagonal):
//   the symmetric sweep operator (Gauss-Jordan elimination with diagonal
//   pivoting) is applied to G pivot by pivot, always on the largest
//   remaining Schur-complement diagonal, and stops at the first one <= tol
//   (deflation: the remaining directions are numerically dependent on the
//   kept set K).  The pivots and the deflation test are those of a
//   diagonal-pivoted Cholesky factorisation; after sweeping K the kept
//   block holds -(G_KK)^-1, so
//   alpha = D G_KK^-1 D rho  and  beta = -D G_KK^-1 D W
//   are plain s x s products (zero rows outside K), with no triangular
//   substitutions and their serial chains.
//
// Where they run.  Each loop kernel's CTAs add their Gram partials to the
// chip's float64 accumulators and then take a ticket; the CTA that takes a
// chip's last ticket has every partial of that chip and solves in place: at
// the end of the Q = A P kernel it sweeps Gamma and forms alpha
// (chip_alpha), at the end of the update kernel it forms beta and tests
// convergence (chip_beta).  No separate launches.  Each tail clears the
// accumulators it consumed.
//
// Arithmetic.  The float64 form runs this in float64.  The mixed form runs
// it in double-float: a value is the unevaluated sum hi + lo of two float32
// words (about 48 significant bits).  float64 instructions issue at 1/64 of
// the float32 rate on this part, and a sweep is a chain of s dependent
// steps whose latency, not its flops, sets the time.  Sums of products are
// carried as lazy compensated accumulators (s, c): the loop-carried
// dependency of one term is a single float32 add on s, while the rounding
// error (TwoSum) and the low-order product terms (TwoProd by fma) collect
// in c, as in the compensated dot product of Ogita, Rump and Oishi (SIAM J.
// Sci. Comput. 26(6), 2005); a value is normalised only where it is
// consumed.
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"

namespace blockoa {

// The ||R_j||^2 accumulators receive one float64 atomic per column from
// every CTA of the update pass; one cache line per entry spreads them over
// L2 slices (packed, a chip's S entries share one or two lines, and the
// few hundred CTAs' atomics queue at those lines' slices).
constexpr int kRn2Stride = 16;
__host__ __device__ __forceinline__ long long rn2_at(int c, int S, int j) {
  return ((long long)c * S + j) * kRn2Stride;
}

struct SmallArgs {
  ChipSolveState *state;
  double *gram;     // [chip][S][S] Gamma accumulator
  double *rho;      // [chip][S][S] rho = P^T R accumulator
  double *wg;       // [chip][S][S] W = Q^T Z accumulator
  double *rn2;      // [chip][S][kRn2Stride] ||R_j||^2 accumulator (entry (c, j) at rn2_at)
  const double *target2;  // [chip][S] squared per-column targets
  void *ginv;       // [chip][S][S] (G_KK)^-1, zero outside K (small-solve arithmetic type);
                    //   float64 form: substitution factors F
  void *dsc;        // [chip][S] scaling diagonal D (small-solve arithmetic type)
  int *rank;        // [chip] |K|
  double *rinv;     // [chip][S] float64 form: 1 / L[k][k] in pivot order
  int *perm;        // [chip][S] float64 form: kept columns in pivot order
  void *alpha;      // [chip][S][S] in the loop's precision
  void *beta;       // [chip][S][S]
  int *ticket;      // [2][chip] flushed-unit counters of the two Gram kernels (zero between launches)
  const int *unit_count;  // [chip] units per chip of the loop kernels
  const int *zunit_count; // [chip] column-tile units per chip of the z-line update
  int n_chips;
  int tail;         // 1: the Gram kernels' last CTAs solve (mixed form, sweep)
  int diag;         // 1: independent columns -- only the diagonals of Gamma, rho, W accumulate
  // deterministic solves: the loop kernels store each CTA's partial sums in
  // a slot (nullptr: atomics into the accumulators above); a chip's slots
  // start at det_base / det_ubase / det_zbase[chip] (the stencil pass, the
  // update, the second z-line step), one per CTA that takes a unit of it
  double *det_spmm;         // [slot][2 S^2]: P^T Q, then P^T R
  double *det_upd;          // [slot][S^2 + S] or [slot][S]: W (when the update forms it), then ||R_j||^2
  double *det_z2;           // [slot][S^2]: W of the second z-line step
  const int *det_base;
  const int *det_ubase;
  const int *det_zbase;
  int s;            // caller's columns (for deflation counts)
  int maxiter;      // limit on total iterations per chip
  double tol;       // deflation threshold on scaled pivots
};

// 2^e as a float64 for -1022 <= e <= 1023.
__device__ __forceinline__ double pow2(int e) {
  return __longlong_as_double((long long)(e + 1023) << 52);
}

// 1/sqrt(x) in float64 for normal x > 0: x = m 4^h with m in [1, 4) (exact
// power-of-two scaling), float32 seed for m (about 2^-23 relative error),
// one Newton step y <- y (3 - m y^2) / 2 (about 2^-45).
__device__ __forceinline__ double rsqrt_nr(double x) {
  const int ex = (int)((__double_as_longlong(x) >> 52) & 0x7ff) - 1023;
  const int h = ex >> 1;
  const double m = x * pow2(-2 * h);
  const double y = (double)rsqrtf((float)m);
  return (y * fma(-0.5 * m, y * y, 1.5)) * pow2(-h);
}

// ---------------------------------------------------------------- double-float
// A double-word value hi + lo with |lo| <= ulp(hi) / 2.  The product is the
// double-word product of Joldes, Muller and Popescu (ACM TOMS 44(2), 2017),
// relative error <= 5u^2, u = 2^-24.  Every operation uses the _rn
// intrinsics, so the compiler neither contracts nor reorders them.
struct dfl {
  float h, l;
};

// s + e = a + b exactly (Knuth's TwoSum, no ordering assumption).
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  return {s, __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv))};
}
// s + e = a + b exactly when exponent(a) >= exponent(b) or a = 0 (Dekker).
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl dw_mul(dfl x, dfl y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);   // exact error of ch
  const float cl2 = __fmaf_rn(x.l, y.h, __fmul_rn(x.h, y.l));
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

// Lazy compensated accumulator: the value is s + c.
struct acc2 {
  float s, c;
};

// The small-solve arithmetic: native float64, or double-float.
template <typename R>
struct SmallMath;

template <>
struct SmallMath<double> {
  using Acc = double;
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double from64(double x) { return x; }
  static __device__ __forceinline__ double to64(double x) { return x; }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double rsqrt(double x) { return rsqrt_nr(x); }
  static __device__ __forceinline__ double rcp(double x) { return __drcp_rn(x); }
  static __device__ __forceinline__ double neg(double x) { return -x; }
  static __device__ __forceinline__ bool greater(double x, double y) { return x > y; }
  // Order-preserving bits of a positive value (sign, exponent, 20 mantissa bits).
  static __device__ __forceinline__ unsigned order_bits(double x) { return (unsigned)__double2hiint(x); }
  static __device__ __forceinline__ double shfl(double x, int src) {
    return __shfl_sync(0xffffffffu, x, src);
  }
  static __device__ __forceinline__ Acc acc(double v) { return v; }
  static __device__ __forceinline__ double value(Acc x) { return x; }
  // x -= a b
  static __device__ __forceinline__ void fms(Acc &x, double a, double b) { x = __fma_rn(-a, b, x); }
  static constexpr bool kScaled = false;   // no range normalisation needed
};

template <>
struct SmallMath<dfl> {
  using Acc = acc2;
  static __device__ __forceinline__ dfl zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ dfl from64(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  static __device__ __forceinline__ double to64(dfl x) { return (double)x.h + (double)x.l; }
  static __device__ __forceinline__ dfl mul(dfl a, dfl b) { return dw_mul(a, b); }
  // Newton step on a float32 seed y0: y1 = y0 + y0 e / 2 with the residual
  // e = 1 - x y0^2 formed to double-word accuracy: x.h y0 = p + pe exactly
  // (TwoProd), so e = (1 - p y0) - (pe + x.l y0) y0, where the first fma is
  // exact up to its final rounding (p y0 is near 1).  The seed's ~2^-23
  // error becomes ~2^-44.
  static __device__ __forceinline__ dfl rsqrt(dfl x) {
    const float y0 = rsqrtf(x.h);
    const float p = __fmul_rn(x.h, y0);
    const float pe = __fmaf_rn(x.h, y0, -p);
    const float lo = __fmaf_rn(x.l, y0, pe);
    const float e = __fmaf_rn(-lo, y0, __fmaf_rn(-p, y0, 1.f));
    return fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e));
  }
  // Newton step on the float32 reciprocal y0: y1 = y0 + y0 e with
  // e = 1 - x y0 = (1 - p) - (pe + x.l y0), x.h y0 = p + pe exactly; 1 - p
  // is exact (p is near 1).  About 2^-46 relative error.
  static __device__ __forceinline__ dfl rcp(dfl x) {
    const float y0 = __frcp_rn(x.h);
    const float p = __fmul_rn(x.h, y0);
    const float pe = __fmaf_rn(x.h, y0, -p);
    const float e = __fsub_rn(__fsub_rn(1.f, p), __fmaf_rn(x.l, y0, pe));
    return fast_two_sum(y0, __fmul_rn(y0, e));
  }
  static __device__ __forceinline__ dfl neg(dfl x) { return {-x.h, -x.l}; }
  static __device__ __forceinline__ bool greater(dfl x, dfl y) {
    return x.h > y.h || (x.h == y.h && x.l > y.l);
  }
  static __device__ __forceinline__ unsigned order_bits(dfl x) { return __float_as_uint(x.h); }
  static __device__ __forceinline__ dfl shfl(dfl x, int src) {
    return {__shfl_sync(0xffffffffu, x.h, src), __shfl_sync(0xffffffffu, x.l, src)};
  }
  static __device__ __forceinline__ Acc acc(dfl v) { return {v.h, v.l}; }
  static __device__ __forceinline__ dfl value(Acc x) { return two_sum(x.s, x.c); }
  // x -= a b: the high product joins s through TwoSum, its exact error and
  // the cross terms join c.
  static __device__ __forceinline__ void fms(Acc &x, dfl a, dfl b) {
    const float ph = __fmul_rn(a.h, b.h);
    const float pe = __fmaf_rn(a.h, b.h, -ph);
    const float pl = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, pe));
    const dfl t = two_sum(x.s, -ph);
    x.s = t.h;
    x.c = __fadd_rn(x.c, __fsub_rn(t.l, pl));
  }
  static constexpr bool kScaled = true;    // float32 exponent range: normalise columns
};

// Small-solve arithmetic of a loop precision.
template <typename T>
using SmallT = typename std::conditional<sizeof(T) == 4, dfl, double>::type;

template <typename R, int S>
struct SweepSmem {
  R Gi[S][S + 1];   // (G_KK)^-1 on K x K, zero elsewhere
  R B[S][S + 1];    // right-hand sides, scaled: D rhs 2^-ex
  R C[2][S];        // published pivot column, by step parity
  R dR[S];          // D
  int ex[S];        // per-column exponent of the right-hand sides
  int sw[S];        // swept (kept) flags
  int bad;
  int rank;
};
template <typename R, int S>
constexpr size_t small_smem_bytes() { return sizeof(SweepSmem<R, S>); }

// True in the CTA whose flush completes a chip: each flush covers `done`
// of the chip's `count` units.  Every thread fences its own accumulator
// updates, then one thread adds the flush's units to the chip's ticket; the
// flush that reaches `count` resets the ticket for the next launch and
// fences again before its CTA reads the accumulators.
__device__ __forceinline__ bool last_flush_of_chip(int *ticket, int done, int count) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int prev = atomicAdd(ticket, done);
    s_last = prev + done == count;
    if (s_last) *ticket = 0;
  }
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// Unbiased exponent of a nonzero float64 (subnormals report -1023).
__device__ __forceinline__ int exponent64(double v) {
  return (int)((__double_as_longlong(v) >> 52) & 0x7ff) - 1023;
}

// x 2^ex in the loop's precision.
template <typename T, typename R>
__device__ __forceinline__ T scaled_out(R x, int ex);
template <>
__device__ __forceinline__ float scaled_out<float, dfl>(dfl x, int ex) {
  return ldexpf(__fadd_rn(x.h, x.l), ex);
}
template <>
__device__ __forceinline__ double scaled_out<double, double>(double x, int ex) {
  return ex == 0 ? x : x * pow2(ex);
}

// out = sign D (G_KK)^-1 D rhs for one chip (all S columns), with
// sh.Gi and sh.dR in place.  256 threads: thread t forms the entries
// (i, j = t % S) for rows i = t / S + (256 / S) m, each an S-term lazy
// compensated dot product.  The right-hand side (float64) is first
// normalised per column by an exact power of two, since double-float has
// float32's exponent range.
template <typename T, typename R, int S>
__device__ __forceinline__ void gram_apply(SweepSmem<R, S> &sh, const double *rhs, bool negate, T *out) {
  using M = SmallMath<R>;
  using Acc = typename M::Acc;
  constexpr int RS = 256 / S < S ? 256 / S : S;            // row stride
  constexpr int OPT = (S + RS - 1) / RS;                   // outputs per thread
  const int t = threadIdx.x;
  if (t < S) sh.ex[t] = M::kScaled ? INT_MIN : 0;
  __syncthreads();
  if (M::kScaled) {
    for (int e = t; e < S * S; e += 256) {
      const double v = __ldcg(rhs + e);
      if (v != 0.0) atomicMax(&sh.ex[e % S], exponent64(v));
    }
    __syncthreads();
    if (t < S) {
      const int x = sh.ex[t];
      sh.ex[t] = x == INT_MIN ? 0 : (x < -1000 ? -1000 : (x > 1000 ? 1000 : x));
    }
    __syncthreads();
  }
  for (int e = t; e < S * S; e += 256) {
    const int k = e / S, j = e % S;
    const double v = __ldcg(rhs + e) * (M::kScaled ? pow2(-sh.ex[j]) : 1.0);
    sh.B[k][j] = M::mul(sh.dR[k], M::from64(v));
  }
  __syncthreads();
  const int j = t % S, i0 = t / S;
  if (i0 >= RS) return;
  Acc acc[OPT];
#pragma unroll
  for (int m = 0; m < OPT; ++m) acc[m] = M::acc(M::zero());
  // i0 < RS and RS * OPT == S for S in {8, 16, 32, 64}: every row below is
  // in range, so the chains carry no guards and interleave freely
  static_assert(RS * OPT == S, "row split");
  for (int k = 0; k < S; ++k) {
    const R b = sh.B[k][j];
#pragma unroll
    for (int m = 0; m < OPT; ++m) M::fms(acc[m], sh.Gi[i0 + RS * m][k], b);   // accumulates -sum
  }
#pragma unroll
  for (int m = 0; m < OPT; ++m) {
    const int i = i0 + RS * m;
    R x = M::mul(sh.dR[i], M::value(acc[m]));
    if (!negate) x = M::neg(x);
    out[(long long)i * S + j] = scaled_out<T, R>(x, sh.ex[j]);
  }
}

// Pivot search over the Schur-complement diagonal (rows lane + 32 q of the
// calling warp).  Every lane first evaluates the reciprocal of its own
// candidates, off the serial path; then the largest candidate above tol
// wins a single 32-bit max-reduction over keys made of its
// order-preserving high bits with the low 6 bits replaced by 63 - index
// (exact up to a relative 2^-14 in float64, 2^-17 in double-float among
// near-equal pivots, lower index first -- any such choice keeps the
// pivoted elimination stable).  Returns the pivot (S: none), its value and
// its reciprocal in every lane.  Warps holding bitwise equal diagonals get
// bitwise equal results.
template <typename R, int S>
__device__ __forceinline__ int find_pivot(const typename SmallMath<R>::Acc *dg, const int *alive, R tol,
                                          R &a, R &inva) {
  using M = SmallMath<R>;
  constexpr int RL = (S + 31) / 32;
  const int lane = threadIdx.x & 31;
  unsigned key = 0;
  R cv[RL], ci[RL];
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    cv[q] = M::value(dg[q]);
    const bool ok = alive[q] && M::greater(cv[q], tol);
    const R rc = M::rcp(cv[q]);   // evaluated unconditionally: selects, not branches
    ci[q] = ok ? rc : M::zero();
    const unsigned kq = (M::order_bits(cv[q]) & ~63u) | (unsigned)(63 - i);
    key = (ok && kq > key) ? kq : key;
  }
  key = __reduce_max_sync(0xffffffffu, key);
  const int p = key ? 63 - (int)(key & 63u) : S;
  R mv = cv[0], mi = ci[0];
#pragma unroll
  for (int q = 1; q < RL; ++q)
    if ((p >> 5) == q) { mv = cv[q]; mi = ci[q]; }
  a = M::shfl(mv, p & 31);
  inva = M::shfl(mi, p & 31);
  return p;
}

// Sweep Gamma of chip c and form alpha.  256 threads; the kernel's dynamic
// shared memory holds SweepSmem.  Warp w keeps the column slab
// j in [w NC, w NC + NC) of G in registers (lane = row, lazy accumulators),
// and every warp keeps its own bitwise-identical copy of the diagonal, so
// all warps find the same pivot without communication.  Step k, pivot p,
// a = G[p][p], c = column p before the step:
//   G[i][j] -= c_i c_j / a (i, j != p),  G[i][p] = c_i / a,  G[p][j] = c_j / a,
//   G[p][p] = -1 / a.
// The warp owning column p publishes c; one barrier per step; then every
// warp updates its slab and diagonal copy and searches the next pivot.
template <typename T, int S>
__device__ __noinline__ void chip_alpha(const SmallArgs &A, int c) {
  using R = SmallT<T>;
  using M = SmallMath<R>;
  using Acc = typename M::Acc;
  constexpr int RL = (S + 31) / 32;            // rows per lane
  constexpr int NC = S / 8;                    // slab columns per warp
  extern __shared__ __align__(16) unsigned char small_smem[];
  SweepSmem<R, S> &sh = *reinterpret_cast<SweepSmem<R, S> *>(small_smem);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  ChipSolveState &st = A.state[c];
  double *g = A.gram + (long long)c * S * S;
  if (t == 0) sh.bad = 0;
  if (t < S) {
    const double w = __ldcg(g + t * S + t);
    sh.dR[t] = (w > 1e-290 && isfinite(w)) ? M::rsqrt(M::from64(w)) : M::zero();
    sh.sw[t] = 0;
  }
  __syncthreads();
  // the lower triangle defines the (exactly symmetric) matrix
  Acc W[RL][NC], dg[RL];
  int alive[RL];
  int bad = 0;
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    const int ic = i < S ? i : 0;
    const R di = sh.dR[ic];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      const int j = warp * NC + cc;
      double v = 0.0;
      if (i < S) {
        v = __ldcg(g + (i > j ? i : j) * S + (i > j ? j : i));
        bad |= !isfinite(v);
      }
      W[q][cc] = M::acc(M::mul(M::mul(M::from64(v), di), sh.dR[j]));
    }
    const double vd = i < S ? __ldcg(g + i * S + i) : 0.0;
    dg[q] = M::acc(M::mul(M::mul(M::from64(vd), di), di));   // bitwise equal to W[i][i]
    alive[q] = i < S && M::greater(di, M::zero());
  }
  if (bad) sh.bad = 1;
  __syncthreads();
  for (int e = t; e < S * S; e += 256) g[e] = 0.0;   // Gamma is consumed
  const R tolR = M::from64(A.tol);
  R a, inva;
  int p = sh.bad ? S : find_pivot<R, S>(dg, alive, tolR, a, inva);
  int k = 0;
  for (; k < S && p < S; ++k) {
    const int buf = k & 1;
    if (warp == p / NC) {   // owner of column p publishes it
      const int co = p % NC;
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int i = lane + 32 * q;
        if (S < 32 && i >= S) continue;
        Acc wv = W[q][0];
#pragma unroll
        for (int cc = 1; cc < NC; ++cc)
          if (cc == co) wv = W[q][cc];
        sh.C[buf][i] = M::value(wv);
      }
      if (lane == 0) sh.sw[p] = 1;
    }
    __syncthreads();
    R cjs[NC];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) cjs[cc] = M::mul(sh.C[buf][warp * NC + cc], inva);
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int i = lane + 32 * q;
      if (S < 32 && i >= S) continue;   // compile-time for S >= 32
      const R ci = sh.C[buf][i];
      const R cis = M::mul(ci, inva);
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const int j = warp * NC + cc;
        Acc u = W[q][cc];
        M::fms(u, ci, cjs[cc]);
        const R spec = j == p ? (i == p ? M::neg(inva) : cis) : cjs[cc];
        W[q][cc] = (i == p || j == p) ? M::acc(spec) : u;
      }
      Acc nd = dg[q];
      M::fms(nd, ci, cis);
      const bool keep = alive[q] && i != p;
      dg[q] = keep ? nd : dg[q];
      alive[q] = keep;
    }
    p = find_pivot<R, S>(dg, alive, tolR, a, inva);
  }
  __syncthreads();
  const int r = sh.bad ? 0 : k;
  // (G_KK)^-1 = -(swept block), zero outside K x K
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (S < 32 && i >= S) continue;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      const int j = warp * NC + cc;
      sh.Gi[i][j] = (r > 0 && sh.sw[i] && sh.sw[j]) ? M::neg(M::value(W[q][cc])) : M::zero();
    }
  }
  __syncthreads();
  // publish (G_KK)^-1 and D for the beta solve, update the chip state
  R *Gg = reinterpret_cast<R *>(A.ginv) + (long long)c * S * S;
  for (int e = t; e < S * S; e += 256) Gg[e] = sh.Gi[e / S][e % S];
  if (t < S) reinterpret_cast<R *>(A.dsc)[(long long)c * S + t] = sh.dR[t];
  if (t == 0) {
    A.rank[c] = r;
    st.rank = r;
    st.deflated += (A.s - r) > 0 ? (A.s - r) : 0;
    if (r == 0) {
      st.status = BLOCKOA_ERR_BREAKDOWN;
      st.active = 0;
    }
  }
  double *rho = A.rho + (long long)c * S * S;
  if (r > 0) gram_apply<T, R, S>(sh, rho, false, reinterpret_cast<T *>(A.alpha) + (long long)c * S * S);
  __syncthreads();
  for (int e = t; e < S * S; e += 256) rho[e] = 0.0;   // rho is consumed
}

// Form beta = -D (G_KK)^-1 D W for chip c from the published inverse, test
// per-column convergence of the updated residual, and clear W and ||R||^2.
// 256 threads; the kernel's dynamic shared memory holds SweepSmem.
template <typename T, int S>
__device__ __noinline__ void chip_beta(const SmallArgs &A, int c) {
  using R = SmallT<T>;
  extern __shared__ __align__(16) unsigned char small_smem[];
  SweepSmem<R, S> &sh = *reinterpret_cast<SweepSmem<R, S> *>(small_smem);
  const int t = threadIdx.x, warp = t >> 5;
  ChipSolveState &st = A.state[c];
  const R *Gg = reinterpret_cast<const R *>(A.ginv) + (long long)c * S * S;
  for (int e = t; e < S * S; e += 256) sh.Gi[e / S][e % S] = Gg[e];
  if (t < S) sh.dR[t] = reinterpret_cast<const R *>(A.dsc)[(long long)c * S + t];
  if (t == 0) sh.rank = A.rank[c];
  __syncthreads();
  double *wg = A.wg + (long long)c * S * S;
  if (sh.rank > 0) gram_apply<T, R, S>(sh, wg, true, reinterpret_cast<T *>(A.beta) + (long long)c * S * S);
  __syncthreads();
  for (int e = t; e < S * S; e += 256) wg[e] = 0.0;   // W is consumed
  if (warp == 0) {
    int conv = 1, bad = 0;
    for (int i = t; i < S; i += 32) {
      const double v = __ldcg(A.rn2 + rn2_at(c, S, i));
      if (!isfinite(v)) bad = 1;
      if (!(v <= A.target2[(long long)c * S + i])) conv = 0;
    }
    conv = __all_sync(0xffffffffu, conv);
    bad = __any_sync(0xffffffffu, bad);
    for (int i = t; i < S; i += 32) A.rn2[rn2_at(c, S, i)] = 0.0;   // consumed
    if (t == 0) {
      st.iters += 1;
      if (bad) {
        st.status = BLOCKOA_ERR_BREAKDOWN;
        st.active = 0;
      } else if (conv) {
        st.status = BLOCKOA_OK;
        st.active = 0;
      } else if (st.iters >= A.maxiter) {
        st.status = BLOCKOA_ERR_NOT_CONVERGED;
        st.active = 0;
      }
    }
  }
}

}  // namespace blockoa
