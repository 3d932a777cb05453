// Noise of the combination (the epsilon term of Eq. 5, Sec. III-B): a
// uniform perturbation in [-amp, amp) K per cell and field, drawn from the
// counter-based generator Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC 2011) so that any
// kernel can produce the value of any (cell, field) without state.
//
// Definition used here: counter (a, m / 4, 0, 0) with a the cell's global
// index and m the field, key (seed, 0); word m % 4 of the output, w, gives
// u = (w >> 11) 2^-53 in [0, 1) and epsilon = amp (2 u - 1) (float64
// fields; float32 fields use the top 24 bits, noise4f).
//
// Gaussian variant (the zero-mean Gaussian noise of the noise study, Sec.
// V-D): counter (a, m / 2, 1, 0), key (seed, 0); words 2 (m % 2) and
// 2 (m % 2) + 1, w1 and w2, give u1 = ((w1 >> 11) + 1/2) 2^-53 in (0, 1) and
// u2 = (w2 >> 11) 2^-53, and epsilon = sigma sqrt(-2 ln u1) cos(2 pi u2)
// (Box and Muller, 1958).  The third counter word keeps the stream apart
// from the uniform one.
#pragma once

#include <stdint.h>

namespace blockoa {

enum { NOISE_UNIFORM = 0, NOISE_GAUSSIAN = 1 };

struct NoiseSpec {
  unsigned long long seed = 0;
  double amp = 0.0;   // uniform: half-width; Gaussian: standard deviation; 0: no noise
  int kind = NOISE_UNIFORM;
};

// Epilogue options of the combination: noise and the normalised weights of
// Eq. 5 (inv_sum[chip * M + m] = 1 / sum_j C[chip][j][m], or NULL).
struct CombineEpi {
  NoiseSpec nz;
  const double *inv_sum = nullptr;
};

// One Philox4x64-10 block: ten rounds, the key bumped by the Weyl constants
// before every round after the first.  Round: with (hi, lo) the 128-bit
// products M0 c0 and M1 c2,
//   c <- (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)).
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += W0;
      k1 += W1;
    }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// float32 fields: the same words with u from their top 24 bits, exact in
// float32 (u = (w >> 40) 2^-24; differs from the float64 value by less than
// amp 2^-23, below the float32 storage of the field), so the epilogue needs
// no float64 arithmetic
__device__ __forceinline__ void noise4f(const NoiseSpec &nz, long long a, long long g, float eps[4]) {
  uint64_t c[4] = {(uint64_t)a, (uint64_t)g, 0ull, 0ull};
  philox4x64_10(c, (uint64_t)nz.seed, 0ull);
  const float amp = (float)nz.amp;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float u = (float)(unsigned)(c[i] >> 40) * 0x1.0p-24f;
    eps[i] = amp * (2.0f * u - 1.0f);
  }
}

// epsilon of fields 4 g .. 4 g + 3 at global cell a
__device__ __forceinline__ void noise4(const NoiseSpec &nz, long long a, long long g, double eps[4]) {
  uint64_t c[4] = {(uint64_t)a, (uint64_t)g, 0ull, 0ull};
  philox4x64_10(c, (uint64_t)nz.seed, 0ull);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const double u = (double)(c[i] >> 11) * 0x1.0p-53;
    eps[i] = nz.amp * (2.0 * u - 1.0);
  }
}

// Gaussian epsilon of fields 2 g and 2 g + 1 at global cell a, float64.
// cospi(2 u2) is cos(2 pi u2) with an exact argument reduction.
__device__ __forceinline__ void gauss2(const NoiseSpec &nz, long long a, long long g, double eps[2]) {
  uint64_t c[4] = {(uint64_t)a, (uint64_t)g, 1ull, 0ull};
  philox4x64_10(c, (uint64_t)nz.seed, 0ull);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const double u1 = ((double)(c[2 * i] >> 11) + 0.5) * 0x1.0p-53;
    const double u2 = (double)(c[2 * i + 1] >> 11) * 0x1.0p-53;
    eps[i] = nz.amp * sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
  }
}

// The same in float32 for float32 fields: u1 is the float32 rounding of the
// float64 value (the 54-bit odd integer 2 (w1 >> 11) + 1 rounded once, then
// scaled by 2^-54 exactly), so it keeps 2^-24 relative accuracy down to the
// smallest u1 and the tails of the distribution; u2 likewise.  The result
// differs from the float64 value by a few float32 roundings of sigma-sized
// numbers.
__device__ __forceinline__ void gauss2f(const NoiseSpec &nz, long long a, long long g, float eps[2]) {
  uint64_t c[4] = {(uint64_t)a, (uint64_t)g, 1ull, 0ull};
  philox4x64_10(c, (uint64_t)nz.seed, 0ull);
  const float sigma = (float)nz.amp;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float u1 = __ull2float_rn(((c[2 * i] >> 11) << 1) | 1ull) * 0x1.0p-54f;
    const float u2 = __ull2float_rn(c[2 * i + 1] >> 11) * 0x1.0p-53f;
    eps[i] = sigma * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
  }
}

}  // namespace blockoa
