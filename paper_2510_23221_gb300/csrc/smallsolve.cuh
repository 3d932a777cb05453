// Small s x s solves of the block-CG iteration (Eq. 4, Sec. III-A).
//
// Per chip and iteration, with D = diag(Gamma)^-1/2 (Jacobi scaling):
//   D Gamma D = L L^T by diagonal-pivoted Cholesky, stopping at the first
//   pivot <= tol (deflation: the remaining directions are numerically
//   dependent on the kept ones);
//   alpha = Gamma^+ rho and beta = -Gamma^+ W on the kept columns, by
//   forward and backward substitution; deflated rows are zero.
//
// Arithmetic.  The float64 form runs this in float64.  The mixed form runs
// it in double-float: a value is the unevaluated sum hi + lo of two float32
// words (about 48 significant bits), built on the error-free transforms
// TwoSum and TwoProd.  float64 instructions issue at 1/64 of the float32
// rate on this part, and the factorisation and substitutions are long
// chains of dependent scalar steps, so double-float shortens them several
// times while staying about 2^-44 accurate, far below what the float32 loop
// resolves.
//
// Structure.  alpha_solve_kernel runs one CTA per (chip, column j): every
// CTA of a chip factors the same matrix with the same instruction sequence
// (bitwise the same factor), then solves its column of alpha.  CTA j = 0
// publishes the substitution factors for beta_solve_kernel, which solves
// one column of beta per single-warp CTA.
//
// Accumulators are cleared by the kernel that runs after their last reader:
// alpha_solve (CTA 0) clears W and ||R||^2, read by the previous beta solve;
// beta_solve (CTA 0) clears Gamma and rho, read by the alpha solve.
#pragma once

#include <climits>
#include <type_traits>

#include "common.cuh"

namespace blockoa {

struct SmallArgs {
  ChipSolveState *state;
  double *gram;     // [chip][S][S] Gamma accumulator
  double *rho;      // [chip][S][S] rho = P^T R accumulator
  double *wg;       // [chip][S][S] W = Q^T R accumulator
  double *rn2;      // [chip][S] ||R_j||^2 accumulator
  const double *target2;  // [chip][S] squared per-column targets
  void *lfac;       // [chip][S][S] substitution factors F (small-solve arithmetic type)
  void *rinv;       // [chip][S] 1 / L[k][k] (small-solve arithmetic type)
  int *perm;        // [chip][S] kept columns in pivot order
  double *dsc;      // [chip][S] scaling diagonal D
  int *rank;        // [chip]
  void *alpha;      // [chip][S][S] in the loop's precision
  void *beta;       // [chip][S][S]
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
// A double-word value hi + lo with |lo| <= ulp(hi) / 2.  The sum and
// product are the double-word algorithms of Joldes, Muller and Popescu
// (ACM TOMS 44(2), 2017): the sum has relative error <= 3u^2 and the
// product <= 5u^2, u = 2^-24.  Every operation uses the _rn intrinsics, so
// the compiler neither contracts nor reorders them.
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
__device__ __forceinline__ dfl dw_add(dfl x, dfl y) {
  const dfl s = two_sum(x.h, y.h);
  const dfl t = two_sum(x.l, y.l);
  const dfl v = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
  return fast_two_sum(v.h, __fadd_rn(t.l, v.l));
}
__device__ __forceinline__ dfl dw_mul(dfl x, dfl y) {
  const float ch = __fmul_rn(x.h, y.h);
  const float cl1 = __fmaf_rn(x.h, y.h, -ch);   // exact error of ch
  const float cl2 = __fmaf_rn(x.l, y.h, __fmul_rn(x.h, y.l));
  return fast_two_sum(ch, __fadd_rn(cl1, cl2));
}

// The small-solve arithmetic: native float64, or double-float.
template <typename R>
struct SmallMath;

template <>
struct SmallMath<double> {
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double from64(double x) { return x; }
  static __device__ __forceinline__ double to64(double x) { return x; }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  // acc - a b
  static __device__ __forceinline__ double fms(double acc, double a, double b) {
    return __fma_rn(-a, b, acc);
  }
  static __device__ __forceinline__ double rsqrt(double x) { return rsqrt_nr(x); }
  static __device__ __forceinline__ bool positive(double x) { return x > 0.0; }
  static __device__ __forceinline__ bool greater(double x, double y) { return x > y; }
  // Order-preserving bits of a positive value (sign, exponent, 20 mantissa bits).
  static __device__ __forceinline__ unsigned order_bits(double x) { return (unsigned)__double2hiint(x); }
  static __device__ __forceinline__ double shfl(double x, int src) {
    return __shfl_sync(0xffffffffu, x, src);
  }
  static constexpr bool kScaled = false;   // no range normalisation needed
};

template <>
struct SmallMath<dfl> {
  static __device__ __forceinline__ dfl zero() { return {0.f, 0.f}; }
  static __device__ __forceinline__ dfl from64(double x) {
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
  }
  static __device__ __forceinline__ double to64(dfl x) { return (double)x.h + (double)x.l; }
  static __device__ __forceinline__ dfl mul(dfl a, dfl b) { return dw_mul(a, b); }
  static __device__ __forceinline__ dfl fms(dfl acc, dfl a, dfl b) {
    const dfl p = dw_mul(a, b);
    return dw_add(acc, dfl{-p.h, -p.l});
  }
  // Newton step on a float32 seed: y1 = y0 + y0 (1 - x y0^2) / 2 with the
  // residual 1 - x y0^2 in double-word (y0^2 is exact as a TwoProd), so the
  // seed's ~2^-23 error becomes ~2^-44.
  static __device__ __forceinline__ dfl rsqrt(dfl x) {
    const float y0 = rsqrtf(x.h);
    const float q = __fmul_rn(y0, y0);
    const dfl xq = dw_mul(x, dfl{q, __fmaf_rn(y0, y0, -q)});
    const dfl e = dw_add(dfl{1.f, 0.f}, dfl{-xq.h, -xq.l});
    return fast_two_sum(y0, __fmul_rn(__fmul_rn(0.5f, y0), e.h));
  }
  static __device__ __forceinline__ bool positive(dfl x) { return x.h > 0.f; }
  static __device__ __forceinline__ bool greater(dfl x, dfl y) {
    return x.h > y.h || (x.h == y.h && x.l > y.l);
  }
  static __device__ __forceinline__ unsigned order_bits(dfl x) { return __float_as_uint(x.h); }
  static __device__ __forceinline__ dfl shfl(dfl x, int src) {
    return {__shfl_sync(0xffffffffu, x.h, src), __shfl_sync(0xffffffffu, x.l, src)};
  }
  static constexpr bool kScaled = true;    // float32 exponent range: normalise columns
};

// Small-solve arithmetic of a loop precision.
template <typename T>
using SmallT = typename std::conditional<sizeof(T) == 4, dfl, double>::type;

template <typename R, int S>
struct FactorSmem {
  R W[S][S + 1];   // scaled Gram (strict lower part); then F in pivot order
  R Lc[S][S];      // Lc[k][a]: column k of L, rows in the original order
  R rv[S];         // 1 / L[k][k], pivot order
  R sq[2], inv[2]; // published pivot: square root and reciprocal square root
  double d[S];     // D
  int perm[S];     // pivot order
  int removed[S];
  int piv[2];
  int bad;
};
template <typename R, int S>
constexpr size_t factor_smem_bytes() { return sizeof(FactorSmem<R, S>); }

// Pivot search over the Schur diagonal held by warp 0 (rows lane + 32 q):
// the largest value, as a 32-bit key of its order-preserving high bits with
// the low 6 bits replaced by 63 - index, reduced in one instruction.  The
// choice is exact up to a relative 2^-14 (float64) or 2^-17 (double-float)
// among near-equal pivots, lower index first; any such choice keeps the
// pivoted factorisation stable.  Lane 0 publishes the pivot or S when the
// largest value is <= tol.
template <typename R, int S>
__device__ __forceinline__ void find_pivot(const R *dg, const int *gone, R tol, FactorSmem<R, S> &sh,
                                           int slot) {
  using M = SmallMath<R>;
  constexpr int RL = (S + 31) / 32;
  const int lane = threadIdx.x & 31;
  unsigned key = 0;
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int a = lane + 32 * q;
    if (a < S && !gone[q] && M::positive(dg[q])) {
      const unsigned kq = (M::order_bits(dg[q]) & ~63u) | (unsigned)(63 - a);
      key = kq > key ? kq : key;
    }
  }
  key = __reduce_max_sync(0xffffffffu, key);
  const int p = key ? 63 - (int)(key & 63u) : S;
  R v = M::zero();
  if (p < S) {
    R mine = dg[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((p >> 5) == q) mine = dg[q];
    v = M::shfl(mine, p & 31);
  }
  if (lane == 0) {
    const bool ok = p < S && M::greater(v, tol);
    const R y = ok ? M::rsqrt(v) : M::zero();
    sh.piv[slot] = ok ? p : S;
    sh.inv[slot] = y;
    sh.sq[slot] = ok ? M::mul(v, y) : M::zero();
  }
}

// Solve column j of Gamma_KK x = rhs_K (kept set K) with the pivot-order
// substitution factors F (F[i][k] = L[i][k] / L[k][k] below the diagonal,
// L[k][i] / L[k][k] above, zero on it) and write sign * D x into column j of
// out (zero rows for deflated columns).  One warp; lane i holds rows i + 32 q.
template <typename T, typename R, int S, int LDF>
__device__ __forceinline__ void solve_column(const R *F, const R *rv, const double *d, const int *perm,
                                             int r, const double *rhs, int j, double sign, T *out) {
  using M = SmallMath<R>;
  constexpr int RL = (S + 31) / 32;
  const int lane = threadIdx.x & 31;
  double y64[RL];
  int pr[RL];
  int ex = INT_MIN;
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    pr[q] = i < r ? perm[i] : -1;
    y64[q] = i < r ? d[pr[q]] * rhs[(long long)pr[q] * S + j] : 0.0;
    if (y64[q] != 0.0) {
      const int e = (int)((__double_as_longlong(y64[q]) >> 52) & 0x7ff) - 1023;
      ex = e > ex ? e : ex;
    }
  }
  // double-float has float32's exponent range: bring the column's largest
  // entry to [1, 2) by an exact power of two, undone at the end
  if (M::kScaled) {
    ex = __reduce_max_sync(0xffffffffu, ex);
    ex = ex == INT_MIN ? 0 : (ex < -1000 ? -1000 : (ex > 1000 ? 1000 : ex));
  } else {
    ex = 0;
  }
  const double up = pow2(ex), down = pow2(-ex);
  R y[RL];
#pragma unroll
  for (int q = 0; q < RL; ++q) y[q] = M::from64(y64[q] * down);
  // L z = y: y_i -= F[i][k] y_k (i > k), then z_i = y_i / L[i][i]
  for (int k = 0; k < r; ++k) {
    R mine = y[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((k >> 5) == q) mine = y[q];
    const R yk = M::shfl(mine, k & 31);
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int i = lane + 32 * q;
      if (i > k && i < r) y[q] = M::fms(y[q], F[i * LDF + k], yk);
    }
  }
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (i < r) y[q] = M::mul(y[q], rv[i]);
  }
  // L^T x = z: z_i -= F[i][k] z_k (i < k), then x_i = z_i / L[i][i]
  for (int k = r - 1; k >= 0; --k) {
    R mine = y[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((k >> 5) == q) mine = y[q];
    const R yk = M::shfl(mine, k & 31);
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int i = lane + 32 * q;
      if (i < k) y[q] = M::fms(y[q], F[i * LDF + k], yk);
    }
  }
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (i < r) y[q] = M::mul(y[q], rv[i]);
  }
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (i < S) out[(long long)i * S + j] = T(0);
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (i < r) out[(long long)pr[q] * S + j] = (T)(sign * d[pr[q]] * (M::to64(y[q]) * up));
  }
}

// alpha = Gamma^+ rho, column j = blockIdx.x % S of chip blockIdx.x / S.
// Step k of the factorisation: threads a < S form column k of L from the
// published pivot; then warp 0 updates the Schur diagonal and searches the
// next pivot while warps 1-7 apply the rank-1 update to the strict lower
// part (fixed entries per thread; rows and columns already pivoted receive
// zero updates, the pivot's own row is never read again).  Two barriers
// per step.
template <typename T, int S>
__global__ void __launch_bounds__(256) alpha_solve_kernel(SmallArgs A) {
  using R = SmallT<T>;
  using M = SmallMath<R>;
  constexpr int RL = (S + 31) / 32;
  constexpr int NE = S * (S - 1) / 2;          // strict lower entries
  constexpr int NEPT = (NE + 223) / 224;       // per thread of warps 1-7
  extern __shared__ __align__(16) unsigned char smem_raw[];
  FactorSmem<R, S> &sh = *reinterpret_cast<FactorSmem<R, S> *>(smem_raw);
  const int c = blockIdx.x / S, j = blockIdx.x % S;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  ChipSolveState &st = A.state[c];
  if (!st.active) return;
  const double *g = A.gram + (long long)c * S * S;
  if (t == 0) sh.bad = 0;
  if (t < S) {
    const double w = g[t * S + t];
    const double dd = (w > 1e-290 && isfinite(w)) ? rsqrt_nr(w) : 0.0;
    sh.d[t] = dd;
    sh.removed[t] = dd == 0.0;
  }
  if (j == 0) {   // W and ||R||^2 of the previous iteration were read by its beta solve
    for (int e = t; e < S * S; e += 256) A.wg[(long long)c * S * S + e] = 0.0;
    if (t < S) A.rn2[(long long)c * S + t] = 0.0;
  }
  __syncthreads();
  for (int e = t; e < S * S; e += 256) {
    const int a = e / S, b = e % S;
    if (b <= a) {
      const double v = 0.5 * (g[a * S + b] + g[b * S + a]);
      if (!isfinite(v)) sh.bad = 1;
      if (b < a) sh.W[a][b] = M::from64(v * sh.d[a] * sh.d[b]);
    }
  }
  // warp 0: the Schur diagonal; warps 1-7: their fixed strict-lower entries
  R dg[RL];
  int gone[RL];
  const R tolR = M::from64(A.tol);
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int a = lane + 32 * q;
      gone[q] = a >= S || sh.removed[a];
      const double da = a < S ? sh.d[a] : 0.0;
      dg[q] = gone[q] ? M::zero() : M::from64(g[a * S + a] * da * da);
    }
  }
  int ea[NEPT], eb[NEPT];
#pragma unroll
  for (int m = 0; m < NEPT; ++m) {
    const int e = (t - 32) + 224 * m;
    int a = 0, b = 0;
    if (warp > 0 && e < NE) {
      a = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
      while (a * (a - 1) / 2 > e) --a;
      while ((a + 1) * a / 2 <= e) ++a;
      b = e - a * (a - 1) / 2;
    }
    ea[m] = (warp > 0 && e < NE) ? a : -1;
    eb[m] = b;
  }
  __syncthreads();
  if (warp == 0) find_pivot<R, S>(dg, gone, tolR, sh, 0);
  __syncthreads();
  int k = 0;
  for (; k < S; ++k) {
    const int p = sh.piv[k & 1];
    if (p >= S || sh.bad) break;
    if (t < S) {
      R l = M::zero();
      if (t == p) l = sh.sq[k & 1];
      else if (!sh.removed[t]) l = M::mul(t > p ? sh.W[t][p] : sh.W[p][t], sh.inv[k & 1]);
      sh.Lc[k][t] = l;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int a = lane + 32 * q;
        if (a == p) gone[q] = 1;
        else if (!gone[q]) dg[q] = M::fms(dg[q], sh.Lc[k][a], sh.Lc[k][a]);
      }
      if (lane == 0) {
        sh.removed[p] = 1;
        sh.perm[k] = p;
        sh.rv[k] = sh.inv[k & 1];
      }
      find_pivot<R, S>(dg, gone, tolR, sh, (k + 1) & 1);
    } else {
#pragma unroll
      for (int m = 0; m < NEPT; ++m)
        if (ea[m] >= 0) sh.W[ea[m]][eb[m]] = M::fms(sh.W[ea[m]][eb[m]], sh.Lc[k][ea[m]], sh.Lc[k][eb[m]]);
    }
    __syncthreads();
  }
  const int r = sh.bad ? 0 : k;
  // substitution factors in pivot order, over W (dead after the loop)
  for (int e = t; e < S * S; e += 256) {
    const int i = e / S, kk = e % S;
    R v = M::zero();
    if (i < r && kk < r) {
      if (i > kk) v = M::mul(sh.Lc[kk][sh.perm[i]], sh.rv[kk]);
      else if (i < kk) v = M::mul(sh.Lc[i][sh.perm[kk]], sh.rv[kk]);
    }
    sh.W[i][kk] = v;
  }
  __syncthreads();
  if (j == 0) {   // publish the factor for the beta solve, update the chip state
    R *F = reinterpret_cast<R *>(A.lfac) + (long long)c * S * S;
    for (int e = t; e < S * S; e += 256) F[e] = sh.W[e / S][e % S];
    if (t < S) {
      reinterpret_cast<R *>(A.rinv)[(long long)c * S + t] = t < r ? sh.rv[t] : M::zero();
      A.dsc[(long long)c * S + t] = sh.d[t];
      A.perm[(long long)c * S + t] = t < r ? sh.perm[t] : -1;
    }
    if (t == 0) {
      A.rank[c] = r;
      st.rank = r;
      st.deflated += (A.s - r) > 0 ? (A.s - r) : 0;
      if (r == 0) {
        st.status = BLOCKOA_ERR_BREAKDOWN;
        st.active = 0;
      }
    }
  }
  if (r == 0 || warp != 0) return;
  solve_column<T, R, S, S + 1>(&sh.W[0][0], sh.rv, sh.d, sh.perm, r, A.rho + (long long)c * S * S, j, 1.0,
                               reinterpret_cast<T *>(A.alpha) + (long long)c * S * S);
}

// beta = -Gamma^+ W, column j; CTA 0 of each chip also clears Gamma and rho
// and runs the per-column convergence test of the updated residual.
template <typename T, int S>
__global__ void __launch_bounds__(32) beta_solve_kernel(SmallArgs A) {
  using R = SmallT<T>;
  __shared__ R F[S][S + 1];
  __shared__ R rv[S];
  __shared__ double d[S];
  __shared__ int perm[S];
  const int c = blockIdx.x / S, j = blockIdx.x % S;
  const int t = threadIdx.x;
  ChipSolveState &st = A.state[c];
  if (!st.active) return;
  const int r = A.rank[c];
  const R *Fg = reinterpret_cast<const R *>(A.lfac) + (long long)c * S * S;
  for (int e = t; e < S * S; e += 32) F[e / S][e % S] = Fg[e];
  for (int i = t; i < S; i += 32) {
    rv[i] = reinterpret_cast<const R *>(A.rinv)[(long long)c * S + i];
    d[i] = A.dsc[(long long)c * S + i];
    perm[i] = A.perm[(long long)c * S + i];
  }
  __syncwarp();
  solve_column<T, R, S, S + 1>(&F[0][0], rv, d, perm, r, A.wg + (long long)c * S * S, j, -1.0,
                               reinterpret_cast<T *>(A.beta) + (long long)c * S * S);
  if (j != 0) return;
  for (int e = t; e < S * S; e += 32) {
    A.gram[(long long)c * S * S + e] = 0.0;
    A.rho[(long long)c * S * S + e] = 0.0;
  }
  int conv = 1, bad = 0;
  for (int i = t; i < S; i += 32) {
    const double v = A.rn2[(long long)c * S + i];
    if (!isfinite(v)) bad = 1;
    if (!(v <= A.target2[(long long)c * S + i])) conv = 0;
  }
  conv = __all_sync(0xffffffffu, conv);
  bad = __any_sync(0xffffffffu, bad);
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

}  // namespace blockoa
