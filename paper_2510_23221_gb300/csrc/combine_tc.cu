// T = U C on the tensor cores (Eq. 5, Sec. III-B), bfloat16x3 with float32
// accumulation in tensor memory (tcgen05, sm_103a).
//
// The float64 basis U is rounded to float32 and split into three bfloat16
// planes  hi = bf16(u),  mid = bf16(u - hi),  lo = bf16(u - hi - mid)
// (relative residual below 2^-23 |u|), C is bfloat16-exact, and
//   T = [lo | mid | hi] [C; C; C]
// is one GEMM with K = 3 S' (S' = s rounded up to 16), the small planes first
// so that they enter the float32 accumulator before the large ones.
//
// Data path: split kernels write U and C directly as shared-memory images
// of the tcgen05 canonical K-major layout without swizzle (8 x 16-byte core
// matrices; element (r, k) of a tile at (r/8)*SBO + (k/8)*128 + (r%8)*16 +
// (k%8)*2 with SBO = (K/8)*128), 128 cells per A tile and 256 fields per B
// chunk.  The GEMM kernel moves each image with one bulk copy
// (cp.async.bulk, completion on an mbarrier), one thread issues
// tcgen05.mma kind::f16 (M = 128, N = 256, K = 16 per instruction) into a
// 256-column TMEM accumulator, and four warps drain it with tcgen05.ld into
// coalesced streaming stores of T (each warp owns 32 cells, i.e. 128 bytes
// of one field per store).  Every mbarrier wait is bounded.
#include <cuda_bf16.h>

#include <vector>

#include "common.cuh"
#include "tc.cuh"
#include "noise.cuh"

namespace blockoa {

constexpr int TC_M = 128;       // cells per tile (MMA M, TMEM lanes)
constexpr int TC_N = 256;       // fields per chunk (MMA N, TMEM columns)
constexpr int TC_THREADS = 128;
static_assert(TC_N % 64 == 0, "the drain takes 64 tensor-memory columns per wait");

__host__ __device__ inline int tc_kpad(int s) { return (s + 15) / 16 * 16; }

// byte offset of element (r, k) in a K-major no-swizzle tcgen05 operand image
__host__ __device__ inline long long tc_img_off(int r, int k, int K) {
  return (long long)(r >> 3) * (K / 8) * 128 + (long long)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

struct TcTile {
  int chip;
  int ncells;       // valid cells in this tile (<= 128)
  long long cell0;  // first cell (global numbering)
  long long img;    // index of the tile's image in the U buffer
};

// ---------------------------------------------------------------- split kernels
// One thread writes one 16-byte row segment (8 consecutive k) of a tile image.
__global__ void split_u_kernel(const TcTile *__restrict__ tiles, int n_tiles,
                               const double *__restrict__ U, int s, int Sp,
                               __nv_bfloat16 *__restrict__ img) {
  const int K = 3 * Sp;
  const long long per_tile = (long long)TC_M * (K / 8);
  const long long total = per_tile * n_tiles;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(i / per_tile);
    const int rem = (int)(i % per_tile);
    const int r = rem / (K / 8), k0 = (rem % (K / 8)) * 8;
    const TcTile tile = tiles[t];
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + q;
      const int plane = k / Sp, j = k % Sp;   // 0 = lo, 1 = mid, 2 = hi
      double u = 0.0;
      if (r < tile.ncells && j < s) u = U[(tile.cell0 + r) * s + j];
      // one rounding to float32 (2^-24 relative), then an exact split in
      // float32: each residual is representable, so hi + mid + lo carries
      // the float value to its last bits without float64 arithmetic
      const float uf = (float)u;
      const __nv_bfloat16 hi = __float2bfloat16(uf);
      const float r1 = uf - __bfloat162float(hi);
      const __nv_bfloat16 mid = __float2bfloat16(r1);
      const float r2 = r1 - __bfloat162float(mid);
      const __nv_bfloat16 lo = __float2bfloat16(r2);
      v[q] = plane == 2 ? hi : (plane == 1 ? mid : lo);
    }
    char *dst = reinterpret_cast<char *>(img) + tile.img * (long long)TC_M * K * 2 + tc_img_off(r, k0, K);
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(v);
  }
}

// B images: chunk q of chip c holds fields [256 q, 256 q + 256) as rows and
// [C; C; C] as K.
__global__ void split_c_kernel(const double *__restrict__ C, int n_chips, int s, int Sp, int M,
                               int n_chunks, __nv_bfloat16 *__restrict__ img) {
  const int K = 3 * Sp;
  const long long per_chunk = (long long)TC_N * (K / 8);
  const long long total = per_chunk * n_chunks * n_chips;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long cq = i / per_chunk;   // chip * n_chunks + chunk
    const int rem = (int)(i % per_chunk);
    const int chip = (int)(cq / n_chunks), q = (int)(cq % n_chunks);
    const int r = rem / (K / 8), k0 = (rem % (K / 8)) * 8;
    const int field = q * TC_N + r;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = (k0 + e) % Sp;
      double c = 0.0;
      if (field < M && j < s) c = C[((long long)chip * s + j) * M + field];
      v[e] = __double2bfloat16(c);
    }
    char *dst = reinterpret_cast<char *>(img) + cq * (long long)TC_N * K * 2 + tc_img_off(r, k0, K);
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(v);
  }
}

// ---------------------------------------------------------------- GEMM kernel
// One CTA: one 128-cell tile of one chip, all fields in chunks of 256.
__global__ void __launch_bounds__(TC_THREADS)
combine_tc_kernel(const TcTile *__restrict__ tiles, const ChipDev *__restrict__ chips,
                  const __nv_bfloat16 *__restrict__ uimg, const __nv_bfloat16 *__restrict__ cimg,
                  float *__restrict__ Tout, int M, int Kdim, int n_chunks, int *__restrict__ err,
                  const CombineEpi epi) {
  const NoiseSpec &nz = epi.nz;
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t a_bytes = TC_M * Kdim * 2, b_bytes = TC_N * Kdim * 2;
  unsigned char *sA = smem;
  unsigned char *sB = smem + a_bytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + b_bytes);  // [0] loads, [1] mma
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const TcTile tile = tiles[blockIdx.x];
  const ChipDev ch = chips[tile.chip];
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(TC_N));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t sbo = (uint32_t)(Kdim / 8) * 128;
  const uint32_t idesc = idesc_bf16(TC_M, TC_N);
  const char *cbase = reinterpret_cast<const char *>(cimg) + (long long)tile.chip * n_chunks * b_bytes;
  uint32_t ld_phase = 0, mma_phase = 0;
  if (tid == 0) {
    mbar_expect_tx(&bars[0], a_bytes + b_bytes);
    bulk_g2s(sA, reinterpret_cast<const char *>(uimg) + tile.img * (long long)a_bytes, a_bytes, &bars[0]);
    bulk_g2s(sB, cbase, b_bytes, &bars[0]);
  }
  float *tbase = Tout + ch.off * (long long)M + (tile.cell0 - ch.off);
  for (int q = 0; q < n_chunks; ++q) {
    if (tid == 0) {
      bool ok = mbar_wait(&bars[0], ld_phase);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        for (int ks = 0; ks < Kdim / 16; ++ks) {
          const uint64_t ad = smem_desc(sA + ks * 256, 128, sbo);
          const uint64_t bd = smem_desc(sB + ks * 256, 128, sbo);
          mma_bf16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
        mma_commit(&bars[1]);
      } else {
        s_fail = 1;
      }
    }
    ld_phase ^= 1;
    __syncthreads();
    if (s_fail) break;
    if (!mbar_wait(&bars[1], mma_phase)) {
      s_fail = 1;
    }
    mma_phase ^= 1;
    __syncthreads();
    if (s_fail) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // the MMAs are done with sB: prefetch the next chunk while draining TMEM
    if (tid == 0 && q + 1 < n_chunks) {
      mbar_expect_tx(&bars[0], b_bytes);
      bulk_g2s(sB, cbase + (long long)(q + 1) * b_bytes, b_bytes, &bars[0]);
    }
    const int cell = warp * 32 + lane;
    const bool valid = cell < tile.ncells;
    const int f0 = q * TC_N;
    float *out = tbase + cell;
    // 64 columns per wait: two tensor-memory loads in flight together
#pragma unroll 1
    for (int c2 = 0; c2 < TC_N / 32; c2 += 2) {
      uint32_t rr[2][32];
      BLOCKOA_TMEM_LD32(tmem + ((uint32_t)(warp * 32) << 16) + c2 * 32, rr[0]);
      BLOCKOA_TMEM_LD32(tmem + ((uint32_t)(warp * 32) << 16) + (c2 + 1) * 32, rr[1]);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        uint32_t (&r)[32] = rr[hh];
        const int fb = f0 + (c2 + hh) * 32;
        if (valid) {
          if (epi.inv_sum) {   // normalised weights of Eq. 5: (U C)_m / sum_j C_jm
            const double *inv = epi.inv_sum + (long long)tile.chip * M + fb;
#pragma unroll
            for (int i = 0; i < 32; ++i)
              if (fb + i < M) r[i] = __float_as_uint(__uint_as_float(r[i]) * (float)__ldg(inv + i));
          }
          if (nz.amp > 0.0 && nz.kind == NOISE_UNIFORM) {   // epsilon of Eq. 5, 4 fields per block (fb % 32 == 0)
#pragma unroll   // constant indices keep r[] in registers
            for (int g = 0; g < 8; ++g) {
              float eps[4];
              noise4f(nz, tile.cell0 + cell, (fb + 4 * g) / 4, eps);
#pragma unroll
              for (int i = 0; i < 4; ++i) r[4 * g + i] = __float_as_uint(__uint_as_float(r[4 * g + i]) + eps[i]);
            }
          } else if (nz.amp > 0.0) {   // Gaussian epsilon, 2 fields per generator block
#pragma unroll
            for (int g = 0; g < 16; ++g) {
              float eps[2];
              gauss2f(nz, tile.cell0 + cell, (fb + 2 * g) / 2, eps);
#pragma unroll
              for (int i = 0; i < 2; ++i) r[2 * g + i] = __float_as_uint(__uint_as_float(r[2 * g + i]) + eps[i]);
            }
          }
#pragma unroll
          for (int i = 0; i < 32; ++i)
            if (fb + i < M) __stcs(out + (long long)(fb + i) * ch.n, __uint_as_float(r[i]));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (s_fail && tid == 0) {
    atomicExch(err, 1);
    // let copies and MMAs still in flight land before the memory is released
    mbar_wait(&bars[0], ld_phase);
    mbar_wait(&bars[1], mma_phase);
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_N));
}

int launch_combine_tc(blockoa_operator *op, const double *U, const double *C, float *Tout, int s,
                      int M, const CombineEpi &epi, cudaStream_t st) {
  const int Sp = tc_kpad(s), K = 3 * Sp;
  const int n_chunks = (M + TC_N - 1) / TC_N;
  std::vector<TcTile> tiles;
  for (int c = 0; c < op->n_chips; ++c)
    for (long long b = 0; b < op->chips[c].n; b += TC_M) {
      TcTile t;
      t.chip = c;
      t.ncells = (int)(op->chips[c].n - b < TC_M ? op->chips[c].n - b : TC_M);
      t.cell0 = op->chips[c].off + b;
      t.img = (long long)tiles.size();
      tiles.push_back(t);
    }
  const size_t a_bytes = (size_t)TC_M * K * 2, b_bytes = (size_t)TC_N * K * 2;
  const size_t smem = a_bytes + b_bytes + 2 * sizeof(uint64_t) + 16;
  void *d_tiles = nullptr, *uimg = nullptr, *cimg = nullptr, *err = nullptr;
  int rc = pool_alloc(op, &d_tiles, sizeof(TcTile) * tiles.size(), st);
  if (!rc) rc = pool_alloc(op, &uimg, a_bytes * tiles.size(), st);
  if (!rc) rc = pool_alloc(op, &cimg, b_bytes * n_chunks * op->n_chips, st);
  if (!rc) rc = pool_alloc(op, &err, 8, st);   // one int flag, read back as one 8-byte word
  auto done = [&](int code) {
    pool_free(d_tiles, st); pool_free(uimg, st); pool_free(cimg, st); pool_free(err, st);
    return code;
  };
  if (rc) return done(rc);
  static size_t attr_smem = 0;
  if (smem > attr_smem) {
    cudaError_t ea = cudaFuncSetAttribute(combine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ea != cudaSuccess) return done(cuda_status(ea, "combine_tc shared memory"));
    attr_smem = smem;
  }
  cudaError_t e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(TcTile) * tiles.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 8, st);
  if (e == cudaSuccess) {
    cudaEvent_t ev0, ev1;
    time_begin(op, st, &ev0);
    g_launches += 3;
    split_u_kernel<<<2048, 256, 0, st>>>((const TcTile *)d_tiles, (int)tiles.size(), U, s, Sp,
                                         (__nv_bfloat16 *)uimg);
    split_c_kernel<<<512, 256, 0, st>>>(C, op->n_chips, s, Sp, M, n_chunks, (__nv_bfloat16 *)cimg);
    time_end(op, st, KC_SPLIT, ev0);
    time_begin(op, st, &ev1);
    combine_tc_kernel<<<(unsigned)tiles.size(), TC_THREADS, smem, st>>>(
        (const TcTile *)d_tiles, op->d_chips, (const __nv_bfloat16 *)uimg,
        (const __nv_bfloat16 *)cimg, Tout, M, K, n_chunks, (int *)err, epi);
    e = cudaGetLastError();
    time_end(op, st, KC_COMBINE_TC, ev1);
  }
  if (e != cudaSuccess) return done(cuda_status(e, "combine_tc"));
  op->h_flag[0] = 0;
  e = read_small(op->h_flag, err, 8, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return done(cuda_status(e, "combine_tc"));
  return done(op->h_flag[0] ? BLOCKOA_ERR_TIMEOUT : BLOCKOA_OK);
}

}  // namespace blockoa
