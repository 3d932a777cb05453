// Fused combination and operator action (Eq. 5 then Eq. 6, Sec. III-B/C):
// for every field m, T_m = U C_m on the tensor cores and q_m = A T_m from
// the same tile's values, so the fields are written once and never read
// back from HBM (the unfused pair of calls writes T, reads it again and
// writes q).
//
// Work unit: one x-row of a chip (cells (z, y, 0 .. nx-1), nx <= 128).  Its
// T values and those of the four rows the 7-point stencil reaches outside
// the row -- (z, y -+ 1) and (z -+ 1, y) -- are five bfloat16x3 GEMMs of the
// same field chunk (M = 128 cells, N = 32 fields, K = 3 S' as in
// combine_tc.cu: planes lo | mid | hi of U against [C; C; C]) into five
// 32-column windows of tensor memory.  The x-neighbours come from the own
// window through shared memory.  A row's stencil rows are recomputed by
// the rows around it: a tensor-core product is cheap here, a second pass
// over T is not.  Each window's T values are bitwise the ones the owning
// row stores (same operands, same MMA sequence), so q = A T holds for the
// stored T exactly as in the unfused path, with float32 stencil arithmetic.
//
// Data path: split kernels write row images of U (128 cell rows, zero past
// nx, K-major no-swizzle core-matrix layout) and 32-field chunk images of
// C; one bulk copy per image, completion on mbarriers.  Warp-specialised
// CTA: one producer thread issues the copies (chunk images two ahead) and
// the tcgen05.mma kind::f16 of chunk g into tensor-memory half g & 1; two
// warpgroups drain the other half meanwhile (thread t owns cell x = t mod
// 128, warpgroup w fields 16 w .. 16 w + 15 of the chunk) and store T and q
// with coalesced streaming stores.  Every mbarrier wait is bounded; a
// timeout is reported as ERR_TIMEOUT after the CTA has let its copies and
// MMAs land and released its tensor memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace blockoa {

constexpr int FA_M = 128;        // cells per row window (MMA M, TMEM lanes)
constexpr int FA_N = 32;         // fields per chunk (MMA N)
constexpr int FA_W = 5;          // windows: own row, y - 1, y + 1, z - 1, z + 1
constexpr int FA_SLICE = 16;     // fields of a chunk drained by one warpgroup
constexpr int FA_DRAIN = 256;    // two drain warpgroups
constexpr int FA_THREADS = FA_DRAIN + 32;   // and one producer warp
constexpr int FA_NB = 4;         // chunk image buffers (two chunks loaded ahead)
constexpr uint32_t FA_HALF = FA_W * FA_N;   // tensor-memory columns of one chunk (5 windows)
constexpr uint32_t FA_TCOLS = 512;            // allocated: two chunks in flight (2 x 160 used)

struct FaRow {
  int chip, z, y, pad;
  int img[FA_W];   // row-image index of each window, -1 where the row lies outside the chip
  int pad2[3];
};

__host__ __device__ inline long long fa_img_off(int r, int k, int K) {
  return (long long)(r >> 3) * (K / 8) * 128 + (long long)(k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Row image i (chip c, row (z, y)): element (x, k) for x < nx, zero above.
// One thread writes one 16-byte segment (8 consecutive k) of one cell row.
__global__ void fa_split_rows_kernel(const FaRow *__restrict__ rows, int n_rows, const ChipDev *__restrict__ chips,
                                     const double *__restrict__ U, int s, int Sp, __nv_bfloat16 *__restrict__ img) {
  const int K = 3 * Sp;
  const long long per_row = (long long)FA_M * (K / 8);
  const long long total = per_row * n_rows;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int ri = (int)(i / per_row);
    const int rem = (int)(i % per_row);
    const int x = rem / (K / 8), k0 = (rem % (K / 8)) * 8;
    const FaRow row = rows[ri];
    const ChipDev ch = chips[row.chip];
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = k0 + q;
      const int plane = k / Sp, j = k % Sp;   // 0 = lo, 1 = mid, 2 = hi
      double u = 0.0;
      if (x < ch.nx && j < s) u = U[(ch.off + ((long long)row.z * ch.ny + row.y) * ch.nx + x) * s + j];
      const float uf = (float)u;
      const __nv_bfloat16 hi = __float2bfloat16(uf);
      const float r1 = uf - __bfloat162float(hi);
      const __nv_bfloat16 mid = __float2bfloat16(r1);
      const float r2 = r1 - __bfloat162float(mid);
      const __nv_bfloat16 lo = __float2bfloat16(r2);
      v[q] = plane == 2 ? hi : (plane == 1 ? mid : lo);
    }
    char *dst = reinterpret_cast<char *>(img) + (long long)ri * FA_M * K * 2 + fa_img_off(x, k0, K);
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(v);
  }
}

// Chunk q of chip c: fields [32 q, 32 q + 32) as rows, [C; C; C] as K.
__global__ void fa_split_c_kernel(const double *__restrict__ C, int n_chips, int s, int Sp, int M, int n_chunks,
                                  __nv_bfloat16 *__restrict__ img) {
  const int K = 3 * Sp;
  const long long per_chunk = (long long)FA_N * (K / 8);
  const long long total = per_chunk * n_chunks * n_chips;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long cq = i / per_chunk;
    const int rem = (int)(i % per_chunk);
    const int chip = (int)(cq / n_chunks), q = (int)(cq % n_chunks);
    const int r = rem / (K / 8), k0 = (rem % (K / 8)) * 8;
    const int field = q * FA_N + r;
    __align__(16) __nv_bfloat16 v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int j = (k0 + e) % Sp;
      double c = 0.0;
      if (field < M && j < s) c = C[((long long)chip * s + j) * M + field];
      v[e] = __double2bfloat16(c);
    }
    char *dst = reinterpret_cast<char *>(img) + cq * (long long)FA_N * K * 2 + fa_img_off(r, k0, K);
    *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(v);
  }
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Named barrier `id` over `n` threads; true on every thread if `pred` held
// on any of them.
__device__ __forceinline__ bool bar_or(int id, int n, bool pred) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.b32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
      " selp.b32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((int)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

struct FaSmem {
  unsigned char *sA, *sB;   // FA_W row images; FA_NB chunk images
  float *sX;                // [2 warpgroups][2][FA_SLICE][FA_M] own-row values
  uint64_t *barA, *barB, *barFull, *barEmpty;
};

// Producer (one thread): the rows' windows, chunk images two ahead, and the
// MMAs of chunk gq into tensor-memory half gq & 1 once the drain warps have
// released it.  Chunks are numbered gq = 0, 1, ... over this CTA's rows.
__device__ void fa_produce(const FaSmem &sm, const FaRow *__restrict__ rows, int my_rows, uint32_t tmem,
                           const __nv_bfloat16 *__restrict__ uimg, const __nv_bfloat16 *__restrict__ cimg,
                           int Kdim, int n_chunks, int *__restrict__ err) {
  const uint32_t a_bytes = FA_M * Kdim * 2, b_bytes = FA_N * Kdim * 2;
  const uint32_t sbo = (uint32_t)(Kdim / 8) * 128;
  const uint32_t idesc = idesc_bf16(FA_M, FA_N);
  const long long total = (long long)my_rows * n_chunks;
  const char *cb = reinterpret_cast<const char *>(cimg);
  long long loaded = 0, bwaited = 0, committed = 0;
  bool a_pending = false, ok = true;
  uint32_t ph_a = 0;
  auto load_chunk = [&](long long c) {
    const int ri = blockIdx.x + (int)(c / n_chunks) * gridDim.x;
    const int b = (int)(c % FA_NB);
    mbar_expect_tx(&sm.barB[b], b_bytes);
    bulk_g2s(sm.sB + b * b_bytes, cb + ((long long)rows[ri].chip * n_chunks + c % n_chunks) * b_bytes, b_bytes,
             &sm.barB[b]);
    loaded = c + 1;
  };
  for (long long c = 0; c < 2 && c < total; ++c) load_chunk(c);
  long long gq = 0;
  for (int k = 0; k < my_rows && ok; ++k) {
    const FaRow row = rows[blockIdx.x + k * gridDim.x];
    // the windows are overwritten once the previous row's last MMA is done
    if (committed > 0) ok = mbar_wait(&sm.barFull[(committed - 1) & 1], (uint32_t)((committed - 1) >> 1) & 1);
    if (!ok) break;
    uint32_t bytes = 0;
    for (int w = 0; w < FA_W; ++w) bytes += row.img[w] >= 0 ? a_bytes : 0;
    mbar_expect_tx(sm.barA, bytes);
    for (int w = 0; w < FA_W; ++w)
      if (row.img[w] >= 0)
        bulk_g2s(sm.sA + w * a_bytes, reinterpret_cast<const char *>(uimg) + (long long)row.img[w] * a_bytes,
                 a_bytes, sm.barA);
    a_pending = true;
    ok = mbar_wait(sm.barA, ph_a);
    if (!ok) break;
    a_pending = false;
    ph_a ^= 1;
    for (int qc = 0; qc < n_chunks; ++qc, ++gq) {
      const int h = (int)(gq & 1);
      // half h is free once chunk gq - 2 is drained; its MMAs are then done,
      // so chunk gq + 2 may go into the buffer they read
      if (gq >= 2) ok = mbar_wait(&sm.barEmpty[h], (uint32_t)((gq >> 1) - 1) & 1);
      if (!ok) break;
      if (gq + 2 < total) load_chunk(gq + 2);
      ok = mbar_wait(&sm.barB[gq % FA_NB], (uint32_t)(gq / FA_NB) & 1);
      if (!ok) break;
      bwaited = gq + 1;
      tc_fence_after();
      const unsigned char *bsrc = sm.sB + (gq % FA_NB) * b_bytes;
      for (int w = 0; w < FA_W; ++w) {
        if (row.img[w] < 0) continue;
        for (int ks = 0; ks < Kdim / 16; ++ks) {
          const uint64_t ad = smem_desc(sm.sA + w * a_bytes + ks * 256, 128, sbo);
          const uint64_t bd = smem_desc(bsrc + ks * 256, 128, sbo);
          mma_bf16(tmem + (uint32_t)(h * FA_HALF + w * FA_N), ad, bd, idesc, ks > 0 ? 1u : 0u);
        }
      }
      mma_commit(&sm.barFull[h]);
      committed = gq + 1;
    }
  }
  if (!ok) {
    atomicExch(err, 1);
    // let the copies and MMAs in flight land before the memory is released
    if (a_pending) mbar_wait(sm.barA, ph_a);
    for (long long c = bwaited; c < loaded; ++c) mbar_wait(&sm.barB[c % FA_NB], (uint32_t)(c / FA_NB) & 1);
    if (committed > 0) mbar_wait(&sm.barFull[(committed - 1) & 1], (uint32_t)((committed - 1) >> 1) & 1);
  }
}

// Drain (256 threads): warpgroup wg takes fields [16 wg, 16 wg + 16) of each
// chunk; thread tl owns cell x = tl of the row (tensor-memory lane tl).
__device__ void fa_drain(const FaSmem &sm, const FaRow *__restrict__ rows, int my_rows,
                         const ChipDev *__restrict__ chips, const float4 *__restrict__ g, uint32_t tmem,
                         float *__restrict__ Tout, float *__restrict__ qout, int M, int n_chunks,
                         int *__restrict__ err) {
  const int t = threadIdx.x, wg = t >> 7, tl = t & 127;
  const uint32_t lane_base = tmem + ((uint32_t)((tl >> 5) * 32) << 16) + (uint32_t)(wg * FA_SLICE);
  long long gq = 0;
  bool fail = false;
  for (int k = 0; k < my_rows && !fail; ++k) {
    const FaRow row = rows[blockIdx.x + k * gridDim.x];
    const ChipDev ch = chips[row.chip];
    // this thread's cell and its seven coefficients (zero for absent neighbours)
    const int x = tl;
    const bool valid = x < ch.nx;
    const long long nxny = (long long)ch.nx * ch.ny;
    const long long loc = ((long long)row.z * ch.ny + row.y) * ch.nx + (valid ? x : 0);
    const long long a = ch.off + loc;
    const bool xp = valid && x + 1 < ch.nx, xm = valid && x > 0;
    const bool yp = valid && row.y + 1 < ch.ny, ym = valid && row.y > 0;
    const bool zp = valid && row.z + 1 < ch.nz, zm = valid && row.z > 0;
    float gb = 0.f, gxp = 0.f, gxm = 0.f, gyp = 0.f, gym = 0.f, gzp = 0.f, gzm = 0.f;
    if (valid) {
      const float4 c4 = g[a];
      gb = c4.w;
      gxp = xp ? c4.x : 0.f;
      gyp = yp ? c4.y : 0.f;
      gzp = zp ? c4.z : 0.f;
      gxm = xm ? g[a - 1].x : 0.f;
      gym = ym ? g[a - ch.nx].y : 0.f;
      gzm = zm ? g[a - nxny].z : 0.f;
    }
    float *tf = Tout + ch.off * (long long)M + loc;
    float *qf = qout + ch.off * (long long)M + loc;
    for (int qc = 0; qc < n_chunks; ++qc, ++gq) {
      const int h = (int)(gq & 1);
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&sm.barFull[h], (uint32_t)(gq >> 1) & 1));
      tc_fence_after();
      uint32_t own[FA_SLICE], wym[FA_SLICE], wyp[FA_SLICE], wzm[FA_SLICE], wzp[FA_SLICE];
      if (ok) {
        const uint32_t tb = lane_base + (uint32_t)(h * FA_HALF);
        BLOCKOA_TMEM_LD16(tb + 0 * FA_N, own);
        BLOCKOA_TMEM_LD16(tb + 1 * FA_N, wym);
        BLOCKOA_TMEM_LD16(tb + 2 * FA_N, wyp);
        BLOCKOA_TMEM_LD16(tb + 3 * FA_N, wzm);
        BLOCKOA_TMEM_LD16(tb + 4 * FA_N, wzp);
        tmem_wait_ld();
      }
      tc_fence_before();
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&sm.barEmpty[h]);   // the half may take chunk gq + 2
      float *xs = sm.sX + (size_t)(wg * 2 + h) * FA_SLICE * FA_M;
#pragma unroll
      for (int i = 0; i < FA_SLICE; ++i) xs[i * FA_M + tl] = __uint_as_float(own[i]);
      if (bar_or(1 + wg, 128, !ok)) { fail = true; break; }
      if (valid) {
        const int f0 = qc * FA_N + wg * FA_SLICE;
#pragma unroll
        for (int i = 0; i < FA_SLICE; ++i) {
          const int m = f0 + i;
          if (m >= M) break;
          const float c = __uint_as_float(own[i]);
          float acc = gb * c;
          if (xp) acc += gxp * (c - xs[i * FA_M + tl + 1]);
          if (xm) acc += gxm * (c - xs[i * FA_M + tl - 1]);
          if (yp) acc += gyp * (c - __uint_as_float(wyp[i]));
          if (ym) acc += gym * (c - __uint_as_float(wym[i]));
          if (zp) acc += gzp * (c - __uint_as_float(wzp[i]));
          if (zm) acc += gzm * (c - __uint_as_float(wzm[i]));
          __stcs(tf + (long long)m * ch.n, c);
          __stcs(qf + (long long)m * ch.n, acc);
        }
      }
    }
  }
  if (fail && tl == 0) atomicExch(err, 1);
}

// One CTA walks rows blockIdx.x, + gridDim.x, ...; per row all field chunks.
__global__ void __launch_bounds__(FA_THREADS, 1)
fa_kernel(const FaRow *__restrict__ rows, int n_rows, const ChipDev *__restrict__ chips,
          const float4 *__restrict__ g, const __nv_bfloat16 *__restrict__ uimg,
          const __nv_bfloat16 *__restrict__ cimg, float *__restrict__ Tout, float *__restrict__ qout, int M,
          int Kdim, int n_chunks, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char smem[];
  const uint32_t a_bytes = FA_M * Kdim * 2, b_bytes = FA_N * Kdim * 2;
  FaSmem sm;
  sm.sA = smem;
  sm.sB = sm.sA + FA_W * a_bytes;
  sm.sX = reinterpret_cast<float *>(sm.sB + FA_NB * b_bytes);
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm.sX + 4 * FA_SLICE * FA_M);
  sm.barA = bars;
  sm.barB = bars + 1;
  sm.barFull = bars + 1 + FA_NB;
  sm.barEmpty = bars + 3 + FA_NB;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 5 + FA_NB);
  const int t = threadIdx.x, warp = t >> 5;
  if (t == 0) {
    mbar_init(sm.barA, 1);
    for (int i = 0; i < FA_NB; ++i) mbar_init(&sm.barB[i], 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(&sm.barFull[i], 1);
      mbar_init(&sm.barEmpty[i], FA_DRAIN / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(tslot, FA_TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int my_rows = n_rows > (int)blockIdx.x ? (n_rows - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  if (warp == FA_DRAIN / 32) {
    if ((t & 31) == 0) fa_produce(sm, rows, my_rows, tmem, uimg, cimg, Kdim, n_chunks, err);
  } else {
    fa_drain(sm, rows, my_rows, chips, g, tmem, Tout, qout, M, n_chunks, err);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, FA_TCOLS);
}

// The fused path covers chips whose rows fit one window (nx <= 128) and
// bases of up to 32 columns (five row images in shared memory).
bool fa_supported(const blockoa_operator *op, int s) {
  if (s > 32) return false;
  for (const ChipDev &c : op->chips)
    if (c.nx > FA_M) return false;
  return true;
}

int launch_combine_apply(blockoa_operator *op, const double *U, const double *C, float *T, float *q, int s,
                         int M, cudaStream_t st) {
  const int Sp = (s + 15) / 16 * 16, K = 3 * Sp;
  const int n_chunks = (M + FA_N - 1) / FA_N;
  std::vector<FaRow> rows;
  std::vector<long long> base(op->n_chips, 0);
  for (int c = 0; c < op->n_chips; ++c) {
    base[c] = (long long)rows.size();
    const ChipDev &cd = op->chips[c];
    for (int z = 0; z < cd.nz; ++z)
      for (int y = 0; y < cd.ny; ++y) {
        FaRow r = {};
        r.chip = c;
        r.z = z;
        r.y = y;
        rows.push_back(r);
      }
  }
  for (FaRow &r : rows) {
    const ChipDev &cd = op->chips[r.chip];
    auto idx = [&](int z, int y) { return (int)(base[r.chip] + (long long)z * cd.ny + y); };
    r.img[0] = idx(r.z, r.y);
    r.img[1] = r.y > 0 ? idx(r.z, r.y - 1) : -1;
    r.img[2] = r.y + 1 < cd.ny ? idx(r.z, r.y + 1) : -1;
    r.img[3] = r.z > 0 ? idx(r.z - 1, r.y) : -1;
    r.img[4] = r.z + 1 < cd.nz ? idx(r.z + 1, r.y) : -1;
  }
  const int n_rows = (int)rows.size();
  const size_t a_bytes = (size_t)FA_M * K * 2, b_bytes = (size_t)FA_N * K * 2;
  const size_t smem =
      FA_W * a_bytes + FA_NB * b_bytes + (size_t)4 * FA_SLICE * FA_M * 4 + (5 + FA_NB) * sizeof(uint64_t) + 16;
  void *d_rows = nullptr, *uimg = nullptr, *cimg = nullptr, *err = nullptr;
  int rc = pool_alloc(op, &d_rows, sizeof(FaRow) * rows.size(), st);
  if (!rc) rc = pool_alloc(op, &uimg, a_bytes * rows.size(), st);
  if (!rc) rc = pool_alloc(op, &cimg, b_bytes * n_chunks * op->n_chips, st);
  if (!rc) rc = pool_alloc(op, &err, 8, st);
  auto done = [&](int code) {
    pool_free(d_rows, st); pool_free(uimg, st); pool_free(cimg, st); pool_free(err, st);
    return code;
  };
  if (rc) return done(rc);
  static size_t attr_smem = 0;
  if (smem > attr_smem) {
    cudaError_t ea = cudaFuncSetAttribute(fa_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (ea != cudaSuccess) return done(cuda_status(ea, "combine_apply shared memory"));
    attr_smem = smem;
  }
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, op->device);
  cudaError_t e = cudaMemcpyAsync(d_rows, rows.data(), sizeof(FaRow) * rows.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 8, st);
  if (e == cudaSuccess) {
    cudaEvent_t ev0, ev1;
    time_begin(op, st, &ev0);
    g_launches += 3;
    fa_split_rows_kernel<<<2048, 256, 0, st>>>((const FaRow *)d_rows, n_rows, op->d_chips, U, s, Sp,
                                              (__nv_bfloat16 *)uimg);
    fa_split_c_kernel<<<512, 256, 0, st>>>(C, op->n_chips, s, Sp, M, n_chunks, (__nv_bfloat16 *)cimg);
    time_end(op, st, KC_SPLIT, ev0);
    time_begin(op, st, &ev1);
    fa_kernel<<<(unsigned)std::min(n_rows, nsm), FA_THREADS, smem, st>>>(
        (const FaRow *)d_rows, n_rows, op->d_chips, reinterpret_cast<const float4 *>(op->g32),
        (const __nv_bfloat16 *)uimg, (const __nv_bfloat16 *)cimg, T, q, M, K, n_chunks, (int *)err);
    e = cudaGetLastError();
    time_end(op, st, KC_COMBINE_APPLY, ev1);
  }
  if (e != cudaSuccess) return done(cuda_status(e, "combine_apply"));
  op->h_flag[0] = 0;
  e = read_small(op->h_flag, err, 8, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return done(cuda_status(e, "combine_apply"));
  return done(op->h_flag[0] ? BLOCKOA_ERR_TIMEOUT : BLOCKOA_OK);
}

}  // namespace blockoa
