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
template <> struct Coef4<double> { using type = double4; };

__device__ __forceinline__ float4 load_coef_(const float *g, long long a) {
  return __ldg(reinterpret_cast<const float4 *>(g) + a);
}
__device__ __forceinline__ double4 load_coef_(const double *g, long long a) {
  const double2 lo = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a);
  const double2 hi = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a + 1);
  return make_double4(lo.x, lo.y, hi.x, hi.y);
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

// q = A T for F consecutive fields of a block of consecutive cells.  One
// thread owns one cell: its own and its -x/-y/-z neighbours' conductances
// are loaded once and reused for the F fields; neighbour values come
// through L1 (x) and L2 (y and z planes), so each value of T is read from
// HBM about once.  Consecutive threads own consecutive cells of a row, so
// every load and store of a warp is one 128-byte line.
constexpr int AP_CELLS = 256;

struct CellBlock {
  int chip, pad;
  long long begin;  // first cell (global numbering)
};

template <typename T, int F>
__global__ void __launch_bounds__(AP_CELLS)
apply_fields_kernel(const CellBlock *__restrict__ blocks, const ChipDev *__restrict__ chips,
                    const T *__restrict__ g, const T *__restrict__ Tin, T *__restrict__ qout,
                    int M) {
  const CellBlock blk = blocks[blockIdx.x];
  const ChipDev ch = chips[blk.chip];
  const long long a = blk.begin + threadIdx.x;
  const int m0 = blockIdx.y * F;
  if (a >= ch.off + ch.n) return;
  const int loc = (int)(a - ch.off);
  const int nx = ch.nx, ny = ch.ny, nxny = nx * ny;
  const int x = loc % nx, y = (loc / nx) % ny, z = loc / nxny;
  const auto c4 = load_coef<T>(g, a);
  const T cxm = x > 0 ? load_coef<T>(g, a - 1).x : T(0);
  const T cym = y > 0 ? load_coef<T>(g, a - nx).y : T(0);
  const T czm = z > 0 ? load_coef<T>(g, a - nxny).z : T(0);
  // neighbour offsets, 0 (the cell itself) where the face is a boundary
  const int oxp = x + 1 < nx ? 1 : 0, oxm = x > 0 ? -1 : 0;
  const int oyp = y + 1 < ny ? nx : 0, oym = y > 0 ? -nx : 0;
  const int ozp = z + 1 < ch.nz ? nxny : 0, ozm = z > 0 ? -nxny : 0;
  const long long fb = ch.off * (long long)M + loc;
  const int nf = M - m0 < F ? M - m0 : F;
#pragma unroll
  for (int f = 0; f < F; ++f) {
    if (f < nf) {
      const T *tp = Tin + fb + (long long)(m0 + f) * ch.n;
      const T c = __ldg(tp);
      const T vxp = __ldg(tp + oxp), vxm = __ldg(tp + oxm);
      const T vyp = __ldg(tp + oyp), vym = __ldg(tp + oym);
      const T vzp = __ldg(tp + ozp), vzm = __ldg(tp + ozm);
      T r = c4.w * c;
      r += c4.x * (c - vxp);
      r += cxm * (c - vxm);
      r += c4.y * (c - vyp);
      r += cym * (c - vym);
      r += c4.z * (c - vzp);
      r += czm * (c - vzm);
      qout[fb + (long long)(m0 + f) * ch.n] = r;
    }
  }
}

int launch_apply_fields(const blockoa_operator *op, const void *Tin, void *qout, int M, int dtype,
                        cudaStream_t st) {
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  if (!mop->apply_blocks) {
    // launch table: 256-cell blocks of every chip (built once per operator)
    std::vector<CellBlock> blocks;
    for (int c = 0; c < op->n_chips; ++c)
      for (long long b = 0; b < op->chips[c].n; b += AP_CELLS)
        blocks.push_back({c, 0, op->chips[c].off + b});
    void *d = nullptr;
    BLOCKOA_CUDA(cudaMalloc(&d, sizeof(CellBlock) * blocks.size()));
    cudaError_t e = cudaMemcpy(d, blocks.data(), sizeof(CellBlock) * blocks.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_status(e, "apply table"); }
    mop->apply_blocks = d;
    mop->n_apply_blocks = (int)blocks.size();
  }
  constexpr int F = 8;
  dim3 grid((unsigned)op->n_apply_blocks, (unsigned)((M + F - 1) / F));
  cudaEvent_t ev;
  time_begin(mop, st, &ev);
  g_launches += 1;
  if (dtype == BLOCKOA_FP64)
    apply_fields_kernel<double, F><<<grid, AP_CELLS, 0, st>>>(
        (const CellBlock *)op->apply_blocks, op->d_chips, op->g64, (const double *)Tin, (double *)qout, M);
  else
    apply_fields_kernel<float, F><<<grid, AP_CELLS, 0, st>>>(
        (const CellBlock *)op->apply_blocks, op->d_chips, op->g32, (const float *)Tin, (float *)qout, M);
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
      const double4 c4 = load_coef<double>(g, a);
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
                  const double *__restrict__ X, double *__restrict__ R, double *__restrict__ rn2) {
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
    const double4 c4 = load_coef<double>(g, a);
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
    atomicAdd(&rn2[(long long)u.chip * S + j], a0);
    atomicAdd(&rn2[(long long)u.chip * S + j + 1], a1);
  }
}

int launch_residual64(const blockoa_operator *op, const double *B, const double *X, double *R,
                      int S, double *rn2, cudaStream_t st) {
  std::vector<Unit> units = make_units(op, 1024);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_units = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(),
                                  cudaMemcpyHostToDevice, st);
  cudaEvent_t ev = nullptr;
  if (e == cudaSuccess) {
    const unsigned nb = (unsigned)units.size();
    const Unit *du = (const Unit *)d_units;
    time_begin(mop, st, &ev);
    g_launches += 1;
    switch (S) {
      case 8: residual64_kernel<8><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2); break;
      case 16: residual64_kernel<16><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2); break;
      case 32: residual64_kernel<32><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2); break;
      case 64: residual64_kernel<64><<<nb, 256, 0, st>>>(du, op->d_chips, op->g64, B, X, R, rn2); break;
      default: pool_free(d_units, st); return BLOCKOA_ERR_INVALID;
    }
    e = cudaGetLastError();
    time_end(mop, st, KC_RESIDUAL64, ev);
  }
  pool_free(d_units, st);
  return cuda_status(e, "residual64");
}

}  // namespace blockoa
