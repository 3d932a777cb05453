// Small s x s solves by float64 diagonal-pivoted Cholesky and substitution
// (Eq. 4, Sec. III-A), as the float64 reference computes them: always for
// the float64 form, and for the mixed form on request
// (BLOCKOA_SMALL_FP64_CHOLESKY); alpha and beta are written in the loop's
// precision.
//
// Per chip and iteration, with D = diag(Gamma)^-1/2:
//   D Gamma D = L L^T by diagonal-pivoted Cholesky, stopping at the first
//   pivot <= tol (deflation), then
//   alpha = Gamma^+ rho and beta = -Gamma^+ W on the kept columns by
//   forward and backward substitution; deflated rows are zero.  In the
//   float32 loop beta is the product -Gamma^+ W instead, with Gamma^+
//   formed column by column by the same substitution (the float32 P update
//   cannot resolve the difference; the Galerkin conditions rest on alpha).
// A substitution leaves a small-system residual of the order of the
// rounding of Gamma itself, so the Galerkin conditions P^T R = 0 hold to
// float64 accuracy and the iteration tracks the exact-arithmetic one down to
// the float64 attainable accuracy.  (The mixed form instead forms an
// explicit inverse by sweeping, smallsolve.cuh: its float32 loop cannot
// resolve the difference.)
//
// chol_alpha_kernel runs one CTA per (chip, column j): every CTA of a chip
// factors the same matrix with the same instruction sequence (bitwise the
// same factor), then solves its column of alpha (and, in the float32
// loop, its column of Gamma^+); CTA j = 0 publishes the substitution
// factors (float64 loop) and clears W and ||R||^2 (read by the previous
// beta solve).  chol_beta_kernel forms one column of beta per CTA; CTA 0
// also clears Gamma and rho and tests convergence.
#pragma once

#include "smallsolve.cuh"

namespace blockoa {

template <int S>
struct CholSmem {
  double W[S][S + 1];   // scaled Gram, strict lower part (row > column); then F in pivot order
  double Lc[S][S];      // Lc[k][a]: column k of L, rows in the original order
  double rv[S];         // 1 / L[k][k], pivot order
  double d[S];          // D
  int perm[S];          // pivot order
  int rem[2][S];        // rows not yet pivoted, excluding the current pivot (by step parity)
  unsigned char tri[S * (S - 1) / 2][2];   // strict-lower pairs (row, column) in row order
  double y[2];          // 1 / sqrt(pivot) of the step (by parity)
  int piv[2], nrem[2];  // pivot row (S: none) and length of rem (by parity)
  int bad;
};
template <int S>
constexpr size_t chol_smem_bytes() { return sizeof(CholSmem<S>); }
constexpr int kCholThreads = 128;   // warp 0: the pivot chain; warps 1-3: rank-1 updates

// Pivot search over the Schur diagonal held by warp 0 (rows lane + 32 q):
// the largest value above tol, by one 32-bit max-reduction over keys made
// of the value's order-preserving high word with the low 6 bits replaced by
// 63 - index (exact up to a relative 2^-14 among near-equal pivots, lower
// index first).  Returns the pivot row (S: none) and its value in v.
// Comparisons of float64 values by their bits (integer instructions; float64
// instructions issue at 1/64 of the float32 rate here): x is positive and
// finite, and x > y for finite y >= 0.
__device__ __forceinline__ bool pos_finite(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b < 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool above(double x, double y) {
  return pos_finite(x) && __double_as_longlong(x) > __double_as_longlong(y);
}

template <int S>
__device__ __forceinline__ int chol_select(const double *dg, const int *gone, double tol, double &v) {
  constexpr int RL = (S + 31) / 32;
  const int lane = threadIdx.x & 31;
  unsigned key = 0;
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int a = lane + 32 * q;
    if (a < S && !gone[q] && pos_finite(dg[q])) {
      const unsigned kq = ((unsigned)__double2hiint(dg[q]) & ~63u) | (unsigned)(63 - a);
      key = kq > key ? kq : key;
    }
  }
  key = __reduce_max_sync(0xffffffffu, key);
  const int p = key ? 63 - (int)(key & 63u) : S;
  v = 0.0;
  if (p < S) {
    double mine = dg[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((p >> 5) == q) mine = dg[q];
    v = __shfl_sync(0xffffffffu, mine, p & 31);
  }
  return (p < S && above(v, tol)) ? p : S;
}

// Solve column j of Gamma_KK x = rhs_K with the pivot-order substitution
// factors F (F[i][k] = L[i][k] / L[k][k] below the diagonal, L[k][i] / L[k][k]
// above, zero on it) and write sign * D x into column j of out (zero rows
// for deflated columns).  rhs == nullptr stands for the unit vector e_j, so
// that out receives column j of Gamma^+.  One warp; lane i holds rows
// i + 32 q.
template <typename T, int S, int LDF>
__device__ __forceinline__ void chol_solve_column(const double *F, const double *rv, const double *d,
                                                  const int *perm, int r, const double *rhs, int j,
                                                  double sign, T *out) {
  constexpr int RL = (S + 31) / 32;
  const int lane = threadIdx.x & 31;
  double y[RL];
  int pr[RL];
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    pr[q] = i < r ? perm[i] : -1;
    y[q] = i < r ? d[pr[q]] * (rhs ? rhs[(long long)pr[q] * S + j] : (pr[q] == j ? 1.0 : 0.0)) : 0.0;
  }
  // L z = y: y_i -= F[i][k] y_k (i > k), then z_i = y_i / L[i][i]
  for (int k = 0; k < r; ++k) {
    double mine = y[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((k >> 5) == q) mine = y[q];
    const double yk = __shfl_sync(0xffffffffu, mine, k & 31);
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int i = lane + 32 * q;
      if (i > k && i < r) y[q] = __fma_rn(-F[i * LDF + k], yk, y[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (i < r) y[q] *= rv[i];
  }
  // L^T x = z: z_i -= F[i][k] z_k (i < k), then x_i = z_i / L[i][i]
  for (int k = r - 1; k >= 0; --k) {
    double mine = y[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((k >> 5) == q) mine = y[q];
    const double yk = __shfl_sync(0xffffffffu, mine, k & 31);
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int i = lane + 32 * q;
      if (i < k) y[q] = __fma_rn(-F[i * LDF + k], yk, y[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int i = lane + 32 * q;
    if (i < r) y[q] *= rv[i];
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
    if (i < r) out[(long long)pr[q] * S + j] = (T)(sign * d[pr[q]] * y[q]);
  }
}

// alpha = Gamma^+ rho, column j = blockIdx.x % S of chip blockIdx.x / S.
//
// float64 issues one warp instruction per 64 cycles on this part whatever
// the active lanes, so the factorisation is laid out as one dependent
// chain in warp 0 with the bulk work beside it.  Step k: warp 0 forms
// column k of L from the pivot column -- which the bulk warps have updated
// through step k-2; warp 0 applies step k-1's rank-1 term to it itself --
// updates the Schur diagonal, selects the next pivot and takes its
// reciprocal square root; meanwhile warps 1-3 apply step k-1's rank-1 term
// to every remaining strict-lower entry that is in neither the current nor
// an earlier pivot's row or column (a packed list of pairs, so the float64
// instructions shrink with the Schur complement).  One barrier per step.
template <typename T, int S>
__global__ void __launch_bounds__(kCholThreads) chol_alpha_kernel(SmallArgs A) {
  constexpr int RL = (S + 31) / 32;
  constexpr int NBULK = kCholThreads - 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CholSmem<S> &sh = *reinterpret_cast<CholSmem<S> *>(smem_raw);
  const int c = blockIdx.x / S, j = blockIdx.x % S;
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  grid_release_next();
  grid_wait_prior();
  ChipSolveState &st = A.state[c];
  if (!st.active) return;
  const double *g = A.gram + (long long)c * S * S;
  if (t == 0) sh.bad = 0;
  for (int e = t; e < S * (S - 1) / 2; e += kCholThreads) {   // row a holds the pairs (a, b < a)
    int a = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)e)) * 0.5f);
    while (a * (a - 1) / 2 > e) --a;
    while ((a + 1) * a / 2 <= e) ++a;
    sh.tri[e][0] = (unsigned char)a;
    sh.tri[e][1] = (unsigned char)(e - a * (a - 1) / 2);
  }
  double dg[RL];   // warp 0: Schur diagonal of its rows (lane + 32 q)
  int gone[RL];    // warp 0: row pivoted, deflated away or padding
  double lp[RL];   // warp 0: the previous step's column of L at its rows
  double lpp = 0.0;   // warp 0: the previous step's column of L at the current pivot's row
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int a = lane + 32 * q;
      const double w = a < S ? g[a * S + a] : 0.0;
      const bool use = a < S && above(w, 1e-290);
      const double dd = use ? rsqrt(w) : 0.0;
      if (a < S) sh.d[a] = dd;
      gone[q] = !use;
      dg[q] = use ? w * dd * dd : 0.0;
      lp[q] = 0.0;
    }
  }
  // the Gram into shared memory (Lc serves as staging): every load of a
  // thread in flight at once
  {
    constexpr int PER = (S * S + kCholThreads - 1) / kCholThreads;
    double v[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = t + u * kCholThreads;
      v[u] = e < S * S ? g[e] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int e = t + u * kCholThreads;
      if (e < S * S) sh.Lc[e / S][e % S] = v[u];
    }
  }
  if (j == 0) {   // W and ||R||^2 of the previous iteration were read by its beta solve
    for (int e = t; e < S * S; e += kCholThreads) A.wg[(long long)c * S * S + e] = 0.0;
    if (t < S) A.rn2[rn2_at(c, S, t)] = 0.0;
  }
  __syncthreads();
  {   // strict lower part of D (Gamma + Gamma^T) / 2 D; non-finite entries fail the chip
    int bad = 0;
    for (int e = t; e < S * (S - 1) / 2; e += kCholThreads) {
      const int a = sh.tri[e][0], b = sh.tri[e][1];
      const double x = sh.Lc[a][b], y = sh.Lc[b][a];
      const long long bx = __double_as_longlong(x) & 0x7fffffffffffffffll;
      const long long by = __double_as_longlong(y) & 0x7fffffffffffffffll;
      bad |= bx >= 0x7ff0000000000000ll || by >= 0x7ff0000000000000ll;
      sh.W[a][b] = (x + y) * (0.5 * sh.d[a] * sh.d[b]);
    }
    if (t < S) {
      const long long bd = __double_as_longlong(sh.Lc[t][t]) & 0x7fffffffffffffffll;
      bad |= bd >= 0x7ff0000000000000ll;
    }
    if (__syncthreads_or(bad) && t == 0) sh.bad = 1;
  }
  __syncthreads();   // Lc is rewritten by the factorisation
  // warp 0: the first pivot, its reciprocal square root, the rows left
  auto publish = [&](int pn, double y, int nxt, int nold, const int *old) {
    int n = 0;
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int i = lane + 32 * q;
      const int a = old ? (i < nold ? old[i] : -1) : (i < S && !gone[q] ? i : -1);
      const bool keep = a >= 0 && a != pn;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) sh.rem[nxt][n + __popc(m & ((1u << lane) - 1u))] = a;
      n += __popc(m);
    }
    if (lane == 0) {
      sh.piv[nxt] = pn;
      sh.nrem[nxt] = n;
      sh.y[nxt] = y;
    }
  };
  if (warp == 0) {
    double v;
    const int p0 = chol_select<S>(dg, gone, A.tol, v);
    publish(p0, p0 < S ? rsqrt(v) : 0.0, 0, 0, nullptr);
  }
  __syncthreads();
  int k = 0;
  for (; k < S; ++k) {
    const int par = k & 1;
    const int p = sh.piv[par];
    if (p >= S || sh.bad) break;
    if (warp == 0) {
      const double y = sh.y[par];
      double l[RL];
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int a = lane + 32 * q;
        l[q] = 0.0;
        if (!gone[q] && a != p) {   // pivot column with the previous step's term applied here
          const double w = a > p ? sh.W[a][p] : sh.W[p][a];
          l[q] = __fma_rn(-lp[q], lpp, w) * y;
        }
        if (a == p) gone[q] = 1;
        if (a < S) sh.Lc[k][a] = l[q];
        if (!gone[q]) dg[q] = __fma_rn(-l[q], l[q], dg[q]);
      }
      // reciprocal square roots of every candidate, under way while the
      // pivot is selected (the selected lane's value is the one kept)
      double ys[RL];
#pragma unroll
      for (int q = 0; q < RL; ++q) ys[q] = rsqrt(pos_finite(dg[q]) ? dg[q] : 1.0);
      double v;
      const int pn = chol_select<S>(dg, gone, A.tol, v);
      lpp = 0.0;
      double ynext = 0.0;
      if (pn < S) {
        double mine = l[0], myy = ys[0];
#pragma unroll
        for (int q = 1; q < RL; ++q)
          if ((pn >> 5) == q) { mine = l[q]; myy = ys[q]; }
        lpp = __shfl_sync(0xffffffffu, mine, pn & 31);
        ynext = __shfl_sync(0xffffffffu, myy, pn & 31);
      }
#pragma unroll
      for (int q = 0; q < RL; ++q) lp[q] = l[q];
      if (lane == 0) {
        sh.perm[k] = p;
        sh.rv[k] = y;
      }
      publish(pn, ynext, par ^ 1, sh.nrem[par], sh.rem[par]);
    } else if (k > 0) {
      // the previous step's rank-1 term on the pairs of the rows left
      // (rem[par] excludes p_0 .. p_k; the pivot column is warp 0's)
      // four entries per pass, all their loads before their float64 FMAs
      const int m = sh.nrem[par];
      const double *lc = sh.Lc[k - 1];
      const int *rem = sh.rem[par];
      const int ne = m * (m - 1) / 2;
      for (int e0 = t - 32; e0 < ne; e0 += 4 * NBULK) {
        int rr[4], cc[4];
        double w[4], la[4], lb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int e = e0 + u * NBULK;
          rr[u] = -1;
          if (e < ne) {
            const int a = rem[sh.tri[e][0]], b = rem[sh.tri[e][1]];
            rr[u] = a > b ? a : b;
            cc[u] = a > b ? b : a;
            w[u] = sh.W[rr[u]][cc[u]];
            la[u] = lc[rr[u]];
            lb[u] = lc[cc[u]];
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (rr[u] >= 0) sh.W[rr[u]][cc[u]] = __fma_rn(-la[u], lb[u], w[u]);
      }
    }
    __syncthreads();
  }
  const int r = sh.bad ? 0 : k;
  // substitution factors in pivot order, over W (dead after the loop)
  for (int e = t; e < S * S; e += kCholThreads) {
    const int i = e / S, kk = e % S;
    double v = 0.0;
    if (i < r && kk < r) {
      if (i > kk) v = sh.Lc[kk][sh.perm[i]] * sh.rv[kk];
      else if (i < kk) v = sh.Lc[i][sh.perm[kk]] * sh.rv[kk];
    }
    sh.W[i][kk] = v;
  }
  __syncthreads();
  if (j == 0) {   // publish the factor for the beta solve, update the chip state
    if constexpr (sizeof(T) != 4) {   // the float32 loop's beta solve reads Gamma^+ instead
      double *F = reinterpret_cast<double *>(A.ginv) + (long long)c * S * S;
      for (int e = t; e < S * S; e += kCholThreads) F[e] = sh.W[e / S][e % S];
    }
    if (t < S) {
      A.rinv[(long long)c * S + t] = t < r ? sh.rv[t] : 0.0;
      reinterpret_cast<double *>(A.dsc)[(long long)c * S + t] = sh.d[t];
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
  if (r == 0) return;
  if (warp == 0) {
    chol_solve_column<T, S, S + 1>(&sh.W[0][0], sh.rv, sh.d, sh.perm, r, A.rho + (long long)c * S * S, j, 1.0,
                                   reinterpret_cast<T *>(A.alpha) + (long long)c * S * S);
  } else if (sizeof(T) == 4 && warp == 1) {
    // float32 loop: column j of Gamma^+ by the same substitution, beside
    // the alpha column (warp 1 issues on its own scheduler), for the beta
    // product of chol_beta_kernel
    chol_solve_column<double, S, S + 1>(&sh.W[0][0], sh.rv, sh.d, sh.perm, r, nullptr, j, 1.0,
                                        reinterpret_cast<double *>(A.ginv) + (long long)c * S * S);
  }
}

// beta = -Gamma^+ W, column j; CTA 0 of each chip also clears Gamma and rho
// and runs the per-column convergence test of the updated residual.  Four
// warps load the factor (independent loads in flight together), warp 0
// substitutes.  In the float32 loop the factor is replaced by Gamma^+
// itself, formed column by column by substitution in chol_alpha_kernel
// (zero outside the kept rows and columns), and warp 0 takes the product
// -Gamma^+ W_j: independent float64 FMAs instead of the two dependent
// substitution chains (float64 instructions issue at 1/64 of the float32
// rate here).
template <typename T, int S>
__global__ void __launch_bounds__(kCholThreads) chol_beta_kernel(SmallArgs A) {
  constexpr int RL = (S + 31) / 32;
  static_assert(S % 4 == 0, "the product takes four columns per step");
  __shared__ double F[S][S + 1];
  __shared__ double rv[S], d[S], wj[S];
  __shared__ int perm[S];
  const int c = blockIdx.x / S, j = blockIdx.x % S;
  const int t = threadIdx.x;
  grid_release_next();
  grid_wait_prior();
  ChipSolveState &st = A.state[c];
  if (!st.active) return;
  const double *Fg = reinterpret_cast<const double *>(A.ginv) + (long long)c * S * S;
#pragma unroll 8
  for (int e = t; e < S * S; e += kCholThreads) F[e / S][e % S] = Fg[e];
  if constexpr (sizeof(T) == 4) {
    for (int i = t; i < S; i += kCholThreads) wj[i] = A.wg[(long long)c * S * S + (long long)i * S + j];
    __syncthreads();
    if (t < 32) {
      T *out = reinterpret_cast<T *>(A.beta) + (long long)c * S * S;
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int i = t + 32 * q;
        if (i < S) {
          double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll 2
          for (int k = 0; k < S; k += 4) {
            a0 = __fma_rn(F[i][k], wj[k], a0);
            a1 = __fma_rn(F[i][k + 1], wj[k + 1], a1);
            a2 = __fma_rn(F[i][k + 2], wj[k + 2], a2);
            a3 = __fma_rn(F[i][k + 3], wj[k + 3], a3);
          }
          out[(long long)i * S + j] = (T)(0.0 - ((a0 + a1) + (a2 + a3)));
        }
      }
    }
  } else {
    for (int i = t; i < S; i += kCholThreads) {
      rv[i] = A.rinv[(long long)c * S + i];
      d[i] = reinterpret_cast<const double *>(A.dsc)[(long long)c * S + i];
      perm[i] = A.perm[(long long)c * S + i];
    }
    __syncthreads();
    if (t < 32)
      chol_solve_column<T, S, S + 1>(&F[0][0], rv, d, perm, A.rank[c], A.wg + (long long)c * S * S, j, -1.0,
                                     reinterpret_cast<T *>(A.beta) + (long long)c * S * S);
  }
  if (j != 0) return;
  for (int e = t; e < S * S; e += kCholThreads) {
    A.gram[(long long)c * S * S + e] = 0.0;
    A.rho[(long long)c * S * S + e] = 0.0;
  }
  if (t >= 32) return;
  int conv = 1, bad = 0;
  for (int i = t; i < S; i += 32) {
    const double v = A.rn2[rn2_at(c, S, i)];
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
