// Operator action q = A T (Eq. 6, Sec. III-C) on field-major data, the
// float64 pair-consistency check, and the float64 true residual B - A X of
// block vectors used by iterative refinement.
//
// Stencil, difference form (cell a, neighbours b):
//   (A t)_a = sum_b G_ab (t_a - t_b) + Gb_a t_a
// with G to +x/+y/+z stored on the cell (cx, cy, cz), G to -x/-y/-z stored
// on the neighbour, and the Robin conductance cb.
#include <vector>

#include "common.cuh"

namespace blockoa {

template <typename T> struct Coef4;
template <> struct Coef4<float> { using type = float4; };
template <> struct Coef4<double> { using type = Coef64; };

__device__ __forceinline__ float4 load_coef_(const float *g, long long a) {
  return __ldg(reinterpret_cast<const float4 *>(g) + a);
}
__device__ __forceinline__ Coef64 load_coef_(const double *g, long long a) {
  const double2 lo = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a);
  const double2 hi = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a + 1);
  return Coef64{lo.x, lo.y, hi.x, hi.y};
}
template <typename T>
__device__ __forceinline__ typename Coef4<T>::type load_coef(const T *g, long long a) {
  return load_coef_(g, a);
}

// Field tiles: 32 (x) by FT_Y (y) columns of one chip, marching along z.
constexpr int FT_X = 32;
constexpr int FT_Y = 8;

struct FieldTile {
  int chip;
  int x0, y0;
  int pad;
};

static std::vector<FieldTile> field_tiles(const blockoa_operator *op) {
  std::vector<FieldTile> t;
  for (int c = 0; c < op->n_chips; ++c) {
    const ChipDev &ch = op->chips[c];
    for (int y = 0; y < ch.ny; y += FT_Y)
      for (int x = 0; x < ch.nx; x += FT_X) t.push_back({c, x, y, 0});
  }
  return t;
}

// q = A T for F consecutive fields: a 2.5D stencil with an asynchronous
// plane pipeline.  A CTA of 32 x 8 threads owns a 32 x 8 column tile of one
// chip and marches z for AF fields.  Each z-plane of the tile, with a halo
// of one row above and below and four cells left and right (16-byte aligned
// rows), is copied into a shared-memory ring of planes by cp.async, AD + 1
// planes ahead of the plane being computed, so every value of T leaves L2
// once (plus the halo) and the copies overlap the arithmetic.  One barrier
// per plane.  Positions outside the chip are zero once and never written
// (their faces have zero conductance).
constexpr int AX = 32, AY = 8, AF = 8;
constexpr int AD = 2;               // planes in flight beyond z + 1
constexpr int RING = AD + 2;        // slots: z, z + 1 and AD planes in flight
constexpr int RW = AX + 8;          // row of a staged plane: x0-4 .. x0+35
constexpr int RH = AY + 2;          // rows y0-1 .. y0+8

struct ApplyTile {
  int chip, x0, y0, pad;
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Issue the copies of plane z of the tile for every field into ring slot z % RING.
template <typename T>
__device__ __forceinline__ void stage_plane(T *ring, const T *__restrict__ Tin, long long fb,
                                            long long nstride, int nf, int z, int nx, int ny,
                                            int x0, int y0, bool vec) {
  constexpr int VE = 16 / (int)sizeof(T);     // elements per 16-byte chunk
  constexpr int CPR = RW / VE;                 // chunks per row
  const int tid = threadIdx.y * AX + threadIdx.x;
  const long long zo = (long long)z * nx * ny;
  T *slot = ring + (z % RING) * (AF * RH * RW);
  const int xs = x0 - 4;
  if (vec) {
    for (int i = tid; i < nf * RH * CPR; i += AX * AY) {
      const int f = i / (RH * CPR), rem = i % (RH * CPR);
      const int r = rem / CPR, cch = rem % CPR;
      const int y = y0 - 1 + r, x = xs + cch * VE;
      if (y < 0 || y >= ny || x < 0 || x + VE > nx) continue;
      cp_async16(slot + (f * RH + r) * RW + cch * VE, Tin + fb + f * nstride + zo + (long long)y * nx + x);
    }
  } else {
    for (int i = tid; i < nf * RH * RW; i += AX * AY) {
      const int f = i / (RH * RW), rem = i % (RH * RW);
      const int r = rem / RW, c = rem % RW;
      const int y = y0 - 1 + r, x = xs + c;
      if (y < 0 || y >= ny || x < 0 || x >= nx) continue;
      if (sizeof(T) == 4) cp_async4(slot + (f * RH + r) * RW + c, Tin + fb + f * nstride + zo + (long long)y * nx + x);
      else slot[(f * RH + r) * RW + c] = Tin[fb + f * nstride + zo + (long long)y * nx + x];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(AX *AY)
apply_fields_kernel(const ApplyTile *__restrict__ tiles, const ChipDev *__restrict__ chips,
                    const T *__restrict__ g, const T *__restrict__ ltab,
                    const T *__restrict__ Tin, T *__restrict__ qout, int M) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ring = reinterpret_cast<T *>(smem_raw);        // [RING][AF][RH][RW]
  __shared__ T scy[AY + 1][AX];
  const ApplyTile tile = tiles[blockIdx.x];
  const ChipDev ch = chips[tile.chip];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * AX + tx;
  const int x = tile.x0 + tx, y = tile.y0 + ty;
  const int nx = ch.nx, ny = ch.ny, nz = ch.nz;
  const int nxny = nx * ny;
  const bool in = x < nx && y < ny;
  const int m0 = blockIdx.y * AF;
  const int nf = M - m0 < AF ? M - m0 : AF;
  const long long fb = ch.off * (long long)M + (long long)m0 * ch.n;
  const int loc0 = y * nx + x;
  // 16-byte copies need 16-byte aligned rows and field strides
  const bool vec = ((nx * (int)sizeof(T)) % 16 == 0) && ((ch.n * (long long)sizeof(T)) % 16 == 0) &&
                   (((fb * (long long)sizeof(T)) % 16) == 0);
  for (int i = tid; i < RING * AF * RH * RW; i += AX * AY) ring[i] = T(0);
  __syncthreads();
  for (int zz = 0; zz <= AD; ++zz) {
    if (zz < nz) stage_plane<T>(ring, Tin, fb, ch.n, nf, zz, nx, ny, tile.x0, tile.y0, vec);
    cp_async_commit();
  }
  const int px = tx + 4, py = ty + 1;    // own position in a staged plane
  T czm = T(0);
  T prev[AF];                            // T at z - 1 of the own cell, per field
#pragma unroll
  for (int f = 0; f < AF; ++f) prev[f] = T(0);
  for (int z = 0; z < nz; ++z) {
    // planes up to z + 1 have landed; the AD - 1 newest copies may be pending
    cp_async_wait<AD - 1>();
    const long long a = ch.off + (long long)z * nxny + loc0;
    typename Coef4<T>::type c4;
    T cxm, cym_l = T(0);
    if (ch.layered) {
      // layered chip: conductances from the z-row's table, no per-cell loads
      const T *lt = ltab + (ch.lz + z) * kLT;
      const T gx = __ldg(lt), gy = __ldg(lt + 1);
      const int cx = (x == 0 ? 1 : 0) | (x == nx - 1 ? 2 : 0);
      const int cy = (y == 0 ? 1 : 0) | (y == ny - 1 ? 2 : 0);
      c4.x = x + 1 < nx ? gx : T(0);
      c4.y = y + 1 < ny ? gy : T(0);
      c4.z = __ldg(lt + 2);
      c4.w = __ldg(lt + 4 + 4 * cx + cy);
      cxm = x > 0 ? gx : T(0);
      cym_l = y > 0 ? gy : T(0);
    } else {
      if (in) c4 = load_coef<T>(g, a);
      else { c4.x = T(0); c4.y = T(0); c4.z = T(0); c4.w = T(0); }
      cxm = __shfl_up_sync(0xffffffffu, c4.x, 1);
      if (tx == 0) cxm = (tile.x0 > 0 && y < ny) ? load_coef<T>(g, a - 1).x : T(0);
      if (x == 0) cxm = T(0);
      scy[ty + 1][tx] = c4.y;
      if (ty == 0) scy[0][tx] = (tile.y0 > 0 && x < nx) ? load_coef<T>(g, a - nx).y : T(0);
    }
    __syncthreads();
    if (z + AD + 1 < nz) stage_plane<T>(ring, Tin, fb, ch.n, nf, z + AD + 1, nx, ny, tile.x0, tile.y0, vec);
    cp_async_commit();
    const T cym = ch.layered ? cym_l : (y > 0 ? scy[ty][tx] : T(0));
    const T *pc = ring + (z % RING) * (AF * RH * RW);
    const T *pn = ring + ((z + 1) % RING) * (AF * RH * RW);
#pragma unroll
    for (int f = 0; f < AF; ++f) {
      const int o = (f * RH + py) * RW + px;
      const T c = pc[o];
      if (in && f < nf) {
        T r = c4.w * c;
        r += c4.x * (c - pc[o + 1]);
        r += cxm * (c - pc[o - 1]);
        r += c4.y * (c - pc[o + RW]);
        r += cym * (c - pc[o - RW]);
        r += c4.z * (c - (z + 1 < nz ? pn[o] : c));
        r += czm * (c - prev[f]);
        qout[fb + (long long)f * ch.n + (long long)z * nxny + loc0] = r;
      }
      prev[f] = c;
    }
    czm = c4.z;
    __syncthreads();
  }
  cp_async_wait<0>();
}

// four consecutive values from shared memory (16-byte aligned)
template <typename T, int unused>
__device__ __forceinline__ void ld4(T *d, const T *p, int, int) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    const double2 b = *reinterpret_cast<const double2 *>(p + 2);
    d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
  }
}
// four consecutive values to global memory (16-byte aligned, streaming)
template <typename T>
__device__ __forceinline__ void st4g(T *p, const T *v) {
  if constexpr (sizeof(T) == 4) {
    __stcs(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
  } else {
    __stcs(reinterpret_cast<double2 *>(p), make_double2(v[0], v[1]));
    __stcs(reinterpret_cast<double2 *>(p + 2), make_double2(v[2], v[3]));
  }
}

// Vectorised form for layered chips whose rows and fields are 16-byte
// aligned: a thread owns 4 consecutive x-cells (one 16-byte vector per
// row), a CTA of 32 x 8 threads a 128 x 8 column tile, VF fields, and a ring
// of three staged planes (z, z + 1 landed, z + 2 in flight).  Each thread's
// staging chunks are fixed over the march, so their offsets are computed
// once; per plane a chunk costs one add and one cp.async.
constexpr int VX = 128, VRW = VX + 8, VRING = 3;

template <typename T, int VF>
__global__ void __launch_bounds__(256)
apply_fields_vec_kernel(const ApplyTile *__restrict__ tiles, const ChipDev *__restrict__ chips,
                        const T *__restrict__ ltab, const T *__restrict__ Tin,
                        T *__restrict__ qout, int M) {
  constexpr int VE = 16 / (int)sizeof(T);            // elements per 16-byte chunk
  constexpr int CPR = VRW / VE;                       // chunks per staged row
  constexpr int SLOT = VF * RH * VRW;                 // elements per staged plane
  constexpr int NCH = VF * RH * CPR;                  // chunks per staged plane
  constexpr int PER = (NCH + 255) / 256;              // chunks per thread
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *ring = reinterpret_cast<T *>(smem_raw);          // [VRING][VF][RH][VRW]
  const ApplyTile tile = tiles[blockIdx.x];
  const ChipDev ch = chips[tile.chip];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  const int nx = ch.nx, ny = ch.ny, nz = ch.nz, nxny = nx * ny;
  const int x = tile.x0 + 4 * tx, y = tile.y0 + ty;
  const bool in = x < nx && y < ny;                   // nx is a multiple of 4
  const int m0 = blockIdx.y * VF;
  const int nf = M - m0 < VF ? M - m0 : VF;
  const T *src = Tin + ch.off * (long long)M + (long long)m0 * ch.n;
  T *dst = qout + ch.off * (long long)M + (long long)m0 * ch.n;
  // fixed staging chunks: smem offset within a slot, element offset within a plane
  int c_sm[PER], c_gl[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = tid + 256 * k;
    c_sm[k] = -1;
    c_gl[k] = 0;
    if (i < NCH) {
      const int f = i / (RH * CPR), rem = i % (RH * CPR);
      const int r = rem / CPR, cch = rem % CPR;
      const int yy = tile.y0 - 1 + r, xx = tile.x0 - 4 + cch * VE;
      if (f < nf && yy >= 0 && yy < ny && xx >= 0 && xx + VE <= nx) {
        c_sm[k] = (f * RH + r) * VRW + cch * VE;
        c_gl[k] = f * (int)ch.n + yy * nx + xx;
      }
    }
  }
  for (int i = tid; i < VRING * SLOT; i += 256) ring[i] = T(0);
  __syncthreads();
  auto stage = [&](int z) {
    T *slot = ring + (z % VRING) * SLOT;
    const T *plane = src + (long long)z * nxny;
#pragma unroll
    for (int k = 0; k < PER; ++k)
      if (c_sm[k] >= 0) cp_async16(slot + c_sm[k], plane + c_gl[k]);
  };
  stage(0);
  cp_async_commit();
  if (nz > 1) stage(1);
  cp_async_commit();
  // edge classes of the four cells (layer tables: 4 * cx + cy)
  const int cyc = (y == 0 ? 1 : 0) | (y == ny - 1 ? 2 : 0);
  int cls[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) cls[j] = 4 * ((x + j == 0 ? 1 : 0) | (x + j == nx - 1 ? 2 : 0)) + cyc;
  const int p0 = 4 + 4 * tx, pr = ty + 1;            // own position in a staged row
  T prev[VF][4];
#pragma unroll
  for (int f = 0; f < VF; ++f)
#pragma unroll
    for (int j = 0; j < 4; ++j) prev[f][j] = T(0);
  T czm = T(0);
  for (int z = 0; z < nz; ++z) {
    cp_async_wait<0>();
    __syncthreads();
    if (z + 2 < nz) stage(z + 2);
    cp_async_commit();
    const T *lt = ltab + (ch.lz + z) * kLT;
    const T gx = __ldg(lt), gy = __ldg(lt + 1), gz = __ldg(lt + 2);
    const T cyp = y + 1 < ny ? gy : T(0), cym = y > 0 ? gy : T(0);
    T cb[4], cxp[4], cxm[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      cb[j] = __ldg(lt + 4 + cls[j]);
      cxp[j] = x + j + 1 < nx ? gx : T(0);
      cxm[j] = x + j > 0 ? gx : T(0);
    }
    const T czp = gz;   // zero on the bottom row by construction
    const T *pc = ring + (z % VRING) * SLOT;
    const T *pn = ring + ((z + 1) % VRING) * SLOT;
#pragma unroll
    for (int f = 0; f < VF; ++f) {
      const int o = (f * RH + pr) * VRW + p0;
      T c[4], up[4], dn[4], zp[4];
      ld4<T, 1>(c, pc + o, 0, 0);
      ld4<T, 1>(up, pc + o - VRW, 0, 0);
      ld4<T, 1>(dn, pc + o + VRW, 0, 0);
      ld4<T, 1>(zp, pn + o, 0, 0);
      const T left = pc[o - 1], right = pc[o + 4];
      if (in && f < nf) {
        T r[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const T xl = j == 0 ? left : c[j - 1];
          const T xr = j == 3 ? right : c[j + 1];
          T v = cb[j] * c[j];
          v += cxp[j] * (c[j] - xr);
          v += cxm[j] * (c[j] - xl);
          v += cyp * (c[j] - dn[j]);
          v += cym * (c[j] - up[j]);
          v += czp * (c[j] - (z + 1 < nz ? zp[j] : c[j]));
          v += czm * (c[j] - prev[f][j]);
          r[j] = v;
        }
        st4g<T>(dst + (long long)f * ch.n + (long long)z * nxny + (long long)y * nx + x, r);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) prev[f][j] = c[j];
    }
    czm = czp;
  }
  cp_async_wait<0>();
}

int launch_apply_fields(const blockoa_operator *op, const void *Tin, void *qout, int M, int dtype,
                        cudaStream_t st) {
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  if (!mop->apply_blocks) {
    // launch table: 32 x 8 column tiles of every chip (built once per operator)
    std::vector<ApplyTile> tiles;
    for (int c = 0; c < op->n_chips; ++c) {
      const ChipDev &ch = op->chips[c];
      for (int y = 0; y < ch.ny; y += AY)
        for (int x = 0; x < ch.nx; x += AX) tiles.push_back({c, x, y, 0});
    }
    void *d = nullptr;
    BLOCKOA_CUDA(cudaMalloc(&d, sizeof(ApplyTile) * tiles.size()));
    cudaError_t e = cudaMemcpy(d, tiles.data(), sizeof(ApplyTile) * tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_status(e, "apply table"); }
    mop->apply_blocks = d;
    mop->n_apply_blocks = (int)tiles.size();
  }
  // vectorised kernel when every chip is layered and 16-byte aligned
  bool vec_ok = true;
  for (int c = 0; c < op->n_chips; ++c) {
    const ChipDev &ch = op->chips[c];
    vec_ok = vec_ok && ch.layered && ch.nx % 4 == 0 && ch.n % 4 == 0 && ch.off % 4 == 0;
  }
  constexpr int VF32 = 4, VF64 = 2;
  const size_t smv32 = sizeof(float) * VRING * VF32 * RH * VRW;
  const size_t smv64 = sizeof(double) * VRING * VF64 * RH * VRW;
  const size_t sm32 = sizeof(float) * RING * AF * RH * RW, sm64 = sizeof(double) * RING * AF * RH * RW;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(apply_fields_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm32);
    cudaFuncSetAttribute(apply_fields_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm64);
    cudaFuncSetAttribute(apply_fields_vec_kernel<float, VF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv32);
    cudaFuncSetAttribute(apply_fields_vec_kernel<double, VF64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smv64);
    attr = true;
  }
  if (vec_ok && !mop->apply_vec_blocks) {
    std::vector<ApplyTile> tiles;
    for (int c = 0; c < op->n_chips; ++c) {
      const ChipDev &ch = op->chips[c];
      for (int y = 0; y < ch.ny; y += AY)
        for (int x = 0; x < ch.nx; x += VX) tiles.push_back({c, x, y, 0});
    }
    void *d = nullptr;
    BLOCKOA_CUDA(cudaMalloc(&d, sizeof(ApplyTile) * tiles.size()));
    cudaError_t e = cudaMemcpy(d, tiles.data(), sizeof(ApplyTile) * tiles.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_status(e, "apply table"); }
    mop->apply_vec_blocks = d;
    mop->n_apply_vec_blocks = (int)tiles.size();
  }
  cudaEvent_t ev;
  time_begin(mop, st, &ev);
  g_launches += 1;
  if (vec_ok) {
    dim3 block(32, AY);
    if (dtype == BLOCKOA_FP64) {
      dim3 grid((unsigned)op->n_apply_vec_blocks, (unsigned)((M + VF64 - 1) / VF64));
      apply_fields_vec_kernel<double, VF64><<<grid, block, smv64, st>>>(
          (const ApplyTile *)op->apply_vec_blocks, op->d_chips, op->lt64, (const double *)Tin,
          (double *)qout, M);
    } else {
      dim3 grid((unsigned)op->n_apply_vec_blocks, (unsigned)((M + VF32 - 1) / VF32));
      apply_fields_vec_kernel<float, VF32><<<grid, block, smv32, st>>>(
          (const ApplyTile *)op->apply_vec_blocks, op->d_chips, op->lt32, (const float *)Tin,
          (float *)qout, M);
    }
  } else {
    dim3 grid((unsigned)op->n_apply_blocks, (unsigned)((M + AF - 1) / AF));
    dim3 block(AX, AY);
    if (dtype == BLOCKOA_FP64)
      apply_fields_kernel<double><<<grid, block, sm64, st>>>(
          (const ApplyTile *)op->apply_blocks, op->d_chips, op->g64, op->lt64, (const double *)Tin,
          (double *)qout, M);
    else
      apply_fields_kernel<float><<<grid, block, sm32, st>>>(
          (const ApplyTile *)op->apply_blocks, op->d_chips, op->g32, op->lt32, (const float *)Tin,
          (float *)qout, M);
  }
  cudaError_t e = cudaGetLastError();
  time_end(mop, st, KC_APPLY, ev);
  return cuda_status(e, "apply_fields");
}

// ---------------------------------------------------------------- pair check
// Per (chip, field): sum (A64 t - q)^2 and sum q^2, with A applied in float64
// to the stored values of t.
template <typename T>
__global__ void __launch_bounds__(FT_X *FT_Y)
pair_check_kernel(const FieldTile *__restrict__ tiles, const ChipDev *__restrict__ chips,
                  const double *__restrict__ g, const T *__restrict__ Tin,
                  const T *__restrict__ qin, int M, double *__restrict__ acc) {
  const FieldTile tile = tiles[blockIdx.x];
  const ChipDev ch = chips[tile.chip];
  const int m = blockIdx.y;
  const int x = tile.x0 + threadIdx.x;
  const int y = tile.y0 + threadIdx.y;
  double num = 0.0, den = 0.0;
  if (x < ch.nx && y < ch.ny) {
    const long long nxny = (long long)ch.nx * ch.ny;
    const T *tf = Tin + ch.off * (long long)M + (long long)m * ch.n;
    const T *qf = qin + ch.off * (long long)M + (long long)m * ch.n;
    for (int z = 0; z < ch.nz; ++z) {
      const long long loc = z * nxny + (long long)y * ch.nx + x;
      const long long a = ch.off + loc;
      const Coef64 c4 = load_coef<double>(g, a);
      const double c = (double)tf[loc];
      double r = c4.w * c;
      if (x + 1 < ch.nx) r += c4.x * (c - (double)tf[loc + 1]);
      if (x > 0) r += load_coef<double>(g, a - 1).x * (c - (double)tf[loc - 1]);
      if (y + 1 < ch.ny) r += c4.y * (c - (double)tf[loc + ch.nx]);
      if (y > 0) r += load_coef<double>(g, a - ch.nx).y * (c - (double)tf[loc - ch.nx]);
      if (z + 1 < ch.nz) r += c4.z * (c - (double)tf[loc + nxny]);
      if (z > 0) r += load_coef<double>(g, a - nxny).z * (c - (double)tf[loc - nxny]);
      const double qv = (double)qf[loc];
      num += (r - qv) * (r - qv);
      den += qv * qv;
    }
  }
  // block reduction
  __shared__ double sn[FT_X * FT_Y / 32], sd[FT_X * FT_Y / 32];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  const int t = threadIdx.y * FT_X + threadIdx.x;
  if ((t & 31) == 0) { sn[t >> 5] = num; sd[t >> 5] = den; }
  __syncthreads();
  if (t == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < FT_X * FT_Y / 32; ++w) { a += sn[w]; b += sd[w]; }
    atomicAdd(&acc[2 * ((long long)tile.chip * M + m)], a);
    atomicAdd(&acc[2 * ((long long)tile.chip * M + m) + 1], b);
  }
}

__global__ void pair_finish_kernel(const double *__restrict__ acc, double *__restrict__ e, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) {
    double num = acc[2 * i], den = acc[2 * i + 1];
    e[i] = den > 0.0 ? sqrt(num / den) : sqrt(num);
  }
}

int launch_pair_check(const blockoa_operator *op, const void *Tin, const void *qin, int M,
                      int dtype, double *e_pair, cudaStream_t st) {
  std::vector<FieldTile> tiles = field_tiles(op);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_tiles = nullptr, *acc = nullptr;
  long long npair = (long long)op->n_chips * M;
  int rc = pool_alloc(mop, &d_tiles, sizeof(FieldTile) * tiles.size(), st);
  if (!rc) rc = pool_alloc(mop, &acc, sizeof(double) * 2 * npair, st);
  if (rc) { pool_free(d_tiles, st); pool_free(acc, st); return rc; }
  cudaError_t e = cudaMemcpyAsync(d_tiles, tiles.data(), sizeof(FieldTile) * tiles.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double) * 2 * npair, st);
  if (e == cudaSuccess) {
    dim3 grid((unsigned)tiles.size(), (unsigned)M);
    dim3 block(FT_X, FT_Y);
    g_launches += 2;
    if (dtype == BLOCKOA_FP64)
      pair_check_kernel<double><<<grid, block, 0, st>>>((const FieldTile *)d_tiles, op->d_chips,
                                                        op->g64, (const double *)Tin,
                                                        (const double *)qin, M, (double *)acc);
    else
      pair_check_kernel<float><<<grid, block, 0, st>>>((const FieldTile *)d_tiles, op->d_chips,
                                                       op->g64, (const float *)Tin,
                                                       (const float *)qin, M, (double *)acc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    pair_finish_kernel<<<(unsigned)((npair + 255) / 256), 256, 0, st>>>((const double *)acc, e_pair, npair);
    e = cudaGetLastError();
  }
  pool_free(d_tiles, st);
  pool_free(acc, st);
  return cuda_status(e, "pair_check");
}

// ---------------------------------------------------------------- float64 residual
// R = B - A X for block vectors [n_total][S] (float64), and per-chip column
// norms ||R_j||^2 accumulated into rn2[chip][S].  One thread owns one cell
// and two columns.
template <int S>
__global__ void __launch_bounds__(256)
residual64_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                  const double *__restrict__ g, const double *__restrict__ B,
                  const double *__restrict__ X, double *__restrict__ R, double *__restrict__ rn2,
                  double *__restrict__ slot) {
  constexpr int TPC = S / 2;           // threads per cell
  constexpr int CPB = 256 / TPC;       // cells per pass
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  const int j = (threadIdx.x % TPC) * 2;
  double s0 = 0.0, s1 = 0.0;
  for (long long a = u.begin + threadIdx.x / TPC; a < u.end; a += CPB) {
    const long long loc = a - ch.off;
    const int x = (int)(loc % ch.nx);
    const int y = (int)((loc / ch.nx) % ch.ny);
    const int z = (int)(loc / nxny);
    const Coef64 c4 = load_coef<double>(g, a);
    const double2 c = *reinterpret_cast<const double2 *>(X + a * S + j);
    double r0 = c4.w * c.x, r1 = c4.w * c.y;
    auto nb = [&](long long b, double gg) {
      const double2 v = *reinterpret_cast<const double2 *>(X + b * S + j);
      r0 += gg * (c.x - v.x);
      r1 += gg * (c.y - v.y);
    };
    if (x + 1 < ch.nx) nb(a + 1, c4.x);
    if (x > 0) nb(a - 1, load_coef<double>(g, a - 1).x);
    if (y + 1 < ch.ny) nb(a + ch.nx, c4.y);
    if (y > 0) nb(a - ch.nx, load_coef<double>(g, a - ch.nx).y);
    if (z + 1 < ch.nz) nb(a + nxny, c4.z);
    if (z > 0) nb(a - nxny, load_coef<double>(g, a - nxny).z);
    const double2 b = *reinterpret_cast<const double2 *>(B + a * S + j);
    const double o0 = b.x - r0, o1 = b.y - r1;
    *reinterpret_cast<double2 *>(R + a * S + j) = make_double2(o0, o1);
    s0 += o0 * o0;
    s1 += o1 * o1;
  }
  // reduce over the cells of this CTA: threads with equal (tid % TPC) share columns
  __shared__ double red[256 * 2];
  red[2 * threadIdx.x] = s0;
  red[2 * threadIdx.x + 1] = s1;
  __syncthreads();
  if (threadIdx.x < TPC) {
    double a0 = 0.0, a1 = 0.0;
    for (int t = threadIdx.x; t < 256; t += TPC) { a0 += red[2 * t]; a1 += red[2 * t + 1]; }
    if (slot) {   // deterministic: this unit's partial sums, reduced in a fixed order afterwards
      slot[(long long)blockIdx.x * S + j] = a0;
      slot[(long long)blockIdx.x * S + j + 1] = a1;
    } else {
      atomicAdd(&rn2[(long long)u.chip * S + j], a0);
      atomicAdd(&rn2[(long long)u.chip * S + j + 1], a1);
    }
  }
}

// AU = A U for a float64 block of s columns (any s), [n][s] cell-major; one
// thread per (cell, column) entry of its unit.
__global__ void __launch_bounds__(256)
apply_block64_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                     const double *__restrict__ g, const double *__restrict__ U, double *__restrict__ AU, int s) {
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  const long long total = (u.end - u.begin) * s;
  for (long long i = threadIdx.x; i < total; i += blockDim.x) {
    const long long a = u.begin + i / s;
    const int j = (int)(i % s);
    const long long loc = a - ch.off;
    const int x = (int)(loc % ch.nx);
    const int y = (int)((loc / ch.nx) % ch.ny);
    const int z = (int)(loc / nxny);
    const Coef64 c4 = load_coef<double>(g, a);
    const double c = U[a * s + j];
    double r = c4.w * c;
    if (x + 1 < ch.nx) r += c4.x * (c - U[(a + 1) * s + j]);
    if (x > 0) r += load_coef<double>(g, a - 1).x * (c - U[(a - 1) * s + j]);
    if (y + 1 < ch.ny) r += c4.y * (c - U[(a + ch.nx) * s + j]);
    if (y > 0) r += load_coef<double>(g, a - ch.nx).y * (c - U[(a - ch.nx) * s + j]);
    if (z + 1 < ch.nz) r += c4.z * (c - U[(a + nxny) * s + j]);
    if (z > 0) r += load_coef<double>(g, a - nxny).z * (c - U[(a - nxny) * s + j]);
    AU[a * s + j] = r;
  }
}

int launch_apply_block64(const blockoa_operator *op, const double *U, double *AU, int s, cudaStream_t st) {
  std::vector<Unit> units = make_units(op, 512);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_units = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    g_launches += 1;
    apply_block64_kernel<<<(unsigned)units.size(), 256, 0, st>>>((const Unit *)d_units, op->d_chips, op->g64,
                                                                  U, AU, s);
    e = cudaGetLastError();
  }
  pool_free(d_units, st);
  return cuda_status(e, "apply_block64");
}

// Relative residual of a candidate block solution, per chip and column:
// acc[chip][j][0] += ||B_j - A X_j||^2 and acc[chip][j][1] += ||B_j||^2 over
// the cells of a unit (one thread per (cell, column) entry, float64 stencil
// in difference form, column sums in shared memory, one atomic per column
// and CTA).  s <= 64.
__global__ void __launch_bounds__(256)
residual_ratio_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                      const double *__restrict__ g, const double *__restrict__ B,
                      const double *__restrict__ X, int s, double *__restrict__ acc) {
  __shared__ double sn[64], sd[64];
  for (int j = threadIdx.x; j < 64; j += blockDim.x) { sn[j] = 0.0; sd[j] = 0.0; }
  __syncthreads();
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  const long long total = (u.end - u.begin) * s;
  for (long long i = threadIdx.x; i < total; i += blockDim.x) {
    const long long a = u.begin + i / s;
    const int j = (int)(i % s);
    const long long loc = a - ch.off;
    const int x = (int)(loc % ch.nx);
    const int y = (int)((loc / ch.nx) % ch.ny);
    const int z = (int)(loc / nxny);
    const Coef64 c4 = load_coef<double>(g, a);
    const double c = X[a * s + j];
    double r = c4.w * c;
    if (x + 1 < ch.nx) r += c4.x * (c - X[(a + 1) * s + j]);
    if (x > 0) r += load_coef<double>(g, a - 1).x * (c - X[(a - 1) * s + j]);
    if (y + 1 < ch.ny) r += c4.y * (c - X[(a + ch.nx) * s + j]);
    if (y > 0) r += load_coef<double>(g, a - ch.nx).y * (c - X[(a - ch.nx) * s + j]);
    if (z + 1 < ch.nz) r += c4.z * (c - X[(a + nxny) * s + j]);
    if (z > 0) r += load_coef<double>(g, a - nxny).z * (c - X[(a - nxny) * s + j]);
    const double b = B[a * s + j];
    const double e = b - r;
    atomicAdd(&sn[j], e * e);
    atomicAdd(&sd[j], b * b);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < s; j += blockDim.x) {
    atomicAdd(&acc[((long long)u.chip * s + j) * 2], sn[j]);
    atomicAdd(&acc[((long long)u.chip * s + j) * 2 + 1], sd[j]);
  }
}

// ratio = sqrt(num / den); a zero right-hand side gives 0 when the residual
// is zero too, +inf otherwise.
__global__ void residual_ratio_finish_kernel(const double *__restrict__ acc, double *__restrict__ ratio, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double num = acc[2 * i], den = acc[2 * i + 1];
  ratio[i] = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
}

int launch_residual_ratio(const blockoa_operator *op, const double *B, const double *X, int s,
                          double *ratio, cudaStream_t st) {
  std::vector<Unit> units = make_units(op, 256);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  const int n = op->n_chips * s;
  void *d_units = nullptr, *acc = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (!rc) rc = pool_alloc(mop, &acc, sizeof(double) * 2 * (size_t)n, st);
  if (rc) {
    pool_free(d_units, st);
    return rc;
  }
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, sizeof(double) * 2 * (size_t)n, st);
  if (e == cudaSuccess) {
    g_launches += 2;
    residual_ratio_kernel<<<(unsigned)units.size(), 256, 0, st>>>((const Unit *)d_units, op->d_chips, op->g64,
                                                                  B, X, s, (double *)acc);
    residual_ratio_finish_kernel<<<(n + 255) / 256, 256, 0, st>>>((const double *)acc, ratio, n);
    e = cudaGetLastError();
  }
  pool_free(d_units, st);
  pool_free(acc, st);
  return cuda_status(e, "residual_ratio");
}

int launch_residual64(const blockoa_operator *op, const double *B, const double *X, double *R,
                      int S, double *rn2, cudaStream_t st, bool det) {
  std::vector<Unit> units = make_units(op, 512);   // float64-bound: enough CTAs for every SM
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_units = nullptr, *d_slot = nullptr, *d_range = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (rc) return rc;
  auto done = [&](int code) {
    pool_free(d_units, st);
    pool_free(d_slot, st);
    pool_free(d_range, st);
    return code;
  };
  std::vector<int> range(2 * (size_t)op->n_chips, 0);   // first unit and unit count of each chip
  if (det) {
    for (size_t k = units.size(); k-- > 0;) range[units[k].chip] = (int)k;
    for (const Unit &u : units) range[op->n_chips + u.chip] += 1;
    rc = pool_alloc(mop, &d_slot, sizeof(double) * units.size() * S, st);
    if (!rc) rc = pool_alloc(mop, &d_range, sizeof(int) * range.size(), st);
    if (rc) return done(rc);
  }
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && det)
    e = cudaMemcpyAsync(d_range, range.data(), sizeof(int) * range.size(), cudaMemcpyHostToDevice, st);
  cudaEvent_t ev = nullptr;
  if (e == cudaSuccess) {
    const unsigned nb = (unsigned)units.size();
    const Unit *du = (const Unit *)d_units;
    double *sl = (double *)d_slot;
    time_begin(mop, st, &ev);
    g_launches += 1;
    switch (S) {
      case 8: residual64_kernel<8><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2, sl); break;
      case 16: residual64_kernel<16><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2, sl); break;
      case 32: residual64_kernel<32><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2, sl); break;
      case 64: residual64_kernel<64><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2, sl); break;
      default: return done(BLOCKOA_ERR_INVALID);
    }
    e = cudaGetLastError();
    time_end(mop, st, KC_RESIDUAL64, ev);
    if (e == cudaSuccess && det)
      e = launch_ordered_reduce(sl, S, (const int *)d_range, (const int *)d_range + op->n_chips, nullptr,
                                op->n_chips, 4, S, rn2, nullptr, 0, st);
  }
  return done(cuda_status(e, "residual64"));
}

}  // namespace blockoa
