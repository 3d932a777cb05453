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
//   forward and backward substitution; deflated rows are zero.
// A substitution leaves a small-system residual of the order of the
// rounding of Gamma itself, so the Galerkin conditions P^T R = 0 hold to
// float64 accuracy and the iteration tracks the exact-arithmetic one down to
// the float64 attainable accuracy.  (The mixed form instead forms an
// explicit inverse by sweeping, smallsolve.cuh: its float32 loop cannot
// resolve the difference.)
//
// chol_alpha_kernel runs one CTA per (chip, column j): every CTA of a chip
// factors the same matrix with the same instruction sequence (bitwise the
// same factor), then solves its column of alpha; CTA j = 0 publishes the
// substitution factors and clears W and ||R||^2 (read by the previous beta
// solve).  chol_beta_kernel solves one column of beta per single-warp CTA;
// CTA 0 also clears Gamma and rho and tests convergence.
#pragma once

#include "smallsolve.cuh"

namespace blockoa {

template <int S>
struct CholSmem {
  double W[S][S + 1];   // scaled Gram (strict lower part); then F in pivot order
  double Lc[S][S];      // Lc[k][a]: column k of L, rows in the original order
  double rv[S];         // 1 / L[k][k], pivot order
  double sq[2], inv[2]; // published pivot: square root and reciprocal square root
  double d[S];          // D
  int perm[S];          // pivot order
  int removed[S];
  int piv[2];
  int bad;
};
template <int S>
constexpr size_t chol_smem_bytes() { return sizeof(CholSmem<S>); }

// Pivot search over the Schur diagonal held by warp 0 (rows lane + 32 q):
// the largest value above tol, by one 32-bit max-reduction over keys made
// of the value's order-preserving high word with the low 6 bits replaced by
// 63 - index (exact up to a relative 2^-14 among near-equal pivots, lower
// index first).  Lane 0 publishes the pivot (S: none), its square root and
// its reciprocal square root.
template <int S>
__device__ __forceinline__ void chol_find_pivot(const double *dg, const int *gone, double tol,
                                                CholSmem<S> &sh, int slot) {
  constexpr int RL = (S + 31) / 32;
  const int lane = threadIdx.x & 31;
  unsigned key = 0;
#pragma unroll
  for (int q = 0; q < RL; ++q) {
    const int a = lane + 32 * q;
    if (a < S && !gone[q] && dg[q] > 0.0) {
      const unsigned kq = ((unsigned)__double2hiint(dg[q]) & ~63u) | (unsigned)(63 - a);
      key = kq > key ? kq : key;
    }
  }
  key = __reduce_max_sync(0xffffffffu, key);
  const int p = key ? 63 - (int)(key & 63u) : S;
  double v = 0.0;
  if (p < S) {
    double mine = dg[0];
#pragma unroll
    for (int q = 1; q < RL; ++q)
      if ((p >> 5) == q) mine = dg[q];
    v = __shfl_sync(0xffffffffu, mine, p & 31);
  }
  if (lane == 0) {
    const bool ok = p < S && v > tol;
    const double y = ok ? rsqrt_nr(v) : 0.0;
    sh.piv[slot] = ok ? p : S;
    sh.inv[slot] = y;
    sh.sq[slot] = ok ? v * y : 0.0;
  }
}

// Solve column j of Gamma_KK x = rhs_K with the pivot-order substitution
// factors F (F[i][k] = L[i][k] / L[k][k] below the diagonal, L[k][i] / L[k][k]
// above, zero on it) and write sign * D x into column j of out (zero rows
// for deflated columns).  One warp; lane i holds rows i + 32 q.
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
    y[q] = i < r ? d[pr[q]] * rhs[(long long)pr[q] * S + j] : 0.0;
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
// Step k: threads a < S form column k of L from the published pivot; then
// warp 0 updates the Schur diagonal and searches the next pivot while warps
// 1-7 apply the rank-1 update to the strict lower part (fixed entries per
// thread; rows and columns already pivoted receive zero updates, the
// pivot's own row is never read again).  Two barriers per step.
template <typename T, int S>
__global__ void __launch_bounds__(256) chol_alpha_kernel(SmallArgs A) {
  constexpr int RL = (S + 31) / 32;
  constexpr int NE = S * (S - 1) / 2;          // strict lower entries
  constexpr int NEPT = (NE + 223) / 224;       // per thread of warps 1-7
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
      if (b < a) sh.W[a][b] = v * sh.d[a] * sh.d[b];
    }
  }
  double dg[RL];
  int gone[RL];
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < RL; ++q) {
      const int a = lane + 32 * q;
      gone[q] = a >= S || sh.removed[a];
      const double da = a < S ? sh.d[a] : 0.0;
      dg[q] = gone[q] ? 0.0 : g[a * S + a] * da * da;
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
  if (warp == 0) chol_find_pivot<S>(dg, gone, A.tol, sh, 0);
  __syncthreads();
  int k = 0;
  for (; k < S; ++k) {
    const int p = sh.piv[k & 1];
    if (p >= S || sh.bad) break;
    if (t < S) {
      double l = 0.0;
      if (t == p) l = sh.sq[k & 1];
      else if (!sh.removed[t]) l = (t > p ? sh.W[t][p] : sh.W[p][t]) * sh.inv[k & 1];
      sh.Lc[k][t] = l;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
      for (int q = 0; q < RL; ++q) {
        const int a = lane + 32 * q;
        if (a == p) gone[q] = 1;
        else if (!gone[q]) dg[q] = __fma_rn(-sh.Lc[k][a], sh.Lc[k][a], dg[q]);
      }
      if (lane == 0) {
        sh.removed[p] = 1;
        sh.perm[k] = p;
        sh.rv[k] = sh.inv[k & 1];
      }
      chol_find_pivot<S>(dg, gone, A.tol, sh, (k + 1) & 1);
    } else {
#pragma unroll
      for (int m = 0; m < NEPT; ++m)
        if (ea[m] >= 0)
          sh.W[ea[m]][eb[m]] = __fma_rn(-sh.Lc[k][ea[m]], sh.Lc[k][eb[m]], sh.W[ea[m]][eb[m]]);
    }
    __syncthreads();
  }
  const int r = sh.bad ? 0 : k;
  // substitution factors in pivot order, over W (dead after the loop)
  for (int e = t; e < S * S; e += 256) {
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
    double *F = reinterpret_cast<double *>(A.ginv) + (long long)c * S * S;
    for (int e = t; e < S * S; e += 256) F[e] = sh.W[e / S][e % S];
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
  if (r == 0 || warp != 0) return;
  chol_solve_column<T, S, S + 1>(&sh.W[0][0], sh.rv, sh.d, sh.perm, r, A.rho + (long long)c * S * S, j, 1.0,
                                 reinterpret_cast<T *>(A.alpha) + (long long)c * S * S);
}

// beta = -Gamma^+ W, column j; CTA 0 of each chip also clears Gamma and rho
// and runs the per-column convergence test of the updated residual.
template <typename T, int S>
__global__ void __launch_bounds__(32) chol_beta_kernel(SmallArgs A) {
  __shared__ double F[S][S + 1];
  __shared__ double rv[S], d[S];
  __shared__ int perm[S];
  const int c = blockIdx.x / S, j = blockIdx.x % S;
  const int t = threadIdx.x;
  grid_release_next();
  grid_wait_prior();
  ChipSolveState &st = A.state[c];
  if (!st.active) return;
  const int r = A.rank[c];
  const double *Fg = reinterpret_cast<const double *>(A.ginv) + (long long)c * S * S;
  for (int e = t; e < S * S; e += 32) F[e / S][e % S] = Fg[e];
  for (int i = t; i < S; i += 32) {
    rv[i] = A.rinv[(long long)c * S + i];
    d[i] = reinterpret_cast<const double *>(A.dsc)[(long long)c * S + i];
    perm[i] = A.perm[(long long)c * S + i];
  }
  __syncwarp();
  chol_solve_column<T, S, S + 1>(&F[0][0], rv, d, perm, r, A.wg + (long long)c * S * S, j, -1.0,
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
