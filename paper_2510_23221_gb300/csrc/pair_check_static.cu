// Pair-consistency check that allocates nothing (no counterpart in the
// paper): the same float64 check as blockoa_pair_check, for callers that
// must not allocate device memory during the call.
//
// Who needs it: serving processes whose device memory is reserved up front
// by their own pool (a stray cudaMalloc competes with that budget and can
// fail or fragment it), fixed-budget deployments that forbid allocation
// after start-up, and loops that must not stall on cudaMalloc / cudaFree,
// which can synchronise the device.  blockoa_pair_check allocates a small
// accumulator and a launch table from the library's stream-ordered pool on
// every call; this variant uses a fixed file-scope device array instead.
//
// Limits and sharing: the array holds 2 * BLOCKOA_STATIC_PAIR_MAX float64
// accumulators (512 KB, kept by every GPU that loads the library until the
// process exits).  All calls on a device share it: each call clears it on
// its stream before use, so calls that overlap on the GPU (different
// streams, or concurrent host threads) race and must be serialised by the
// caller.
#include <mutex>

#include "common.cuh"

namespace blockoa {

constexpr int kStaticPairMax = BLOCKOA_STATIC_PAIR_MAX;

// [pair][2]: sum (A t - q)^2 and sum q^2.  In host code this name is only a
// stand-in for the symbol; kernels receive its device address.
static __device__ __align__(256) double g_pair_scratch[2 * kStaticPairMax];

constexpr int PS_X = 32, PS_Y = 8;

__device__ __forceinline__ Coef64 ps_coef(const double *g, long long a) {
  const double2 lo = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a);
  const double2 hi = __ldg(reinterpret_cast<const double2 *>(g) + 2 * a + 1);
  return Coef64{lo.x, lo.y, hi.x, hi.y};
}

__global__ void ps_clear_kernel(double *acc, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) acc[i] = 0.0;
}

// Grid: x = tile of a chip (32 x 8 columns, tiles past the chip's end idle),
// y = field, z = chip.  The chip table is the operator's device copy.
template <typename T>
__global__ void __launch_bounds__(PS_X *PS_Y)
ps_check_kernel(const ChipDev *__restrict__ chips, const double *__restrict__ g,
                const T *__restrict__ Tin, const T *__restrict__ qin, int M,
                double *__restrict__ acc) {
  const ChipDev ch = chips[blockIdx.z];
  const int tiles_x = (ch.nx + PS_X - 1) / PS_X;
  const int tiles_y = (ch.ny + PS_Y - 1) / PS_Y;
  if ((int)blockIdx.x >= tiles_x * tiles_y) return;
  const int m = blockIdx.y;
  const int x = (blockIdx.x % tiles_x) * PS_X + threadIdx.x;
  const int y = (blockIdx.x / tiles_x) * PS_Y + threadIdx.y;
  double num = 0.0, den = 0.0;
  if (x < ch.nx && y < ch.ny) {
    const long long nxny = (long long)ch.nx * ch.ny;
    const T *tf = Tin + ch.off * (long long)M + (long long)m * ch.n;
    const T *qf = qin + ch.off * (long long)M + (long long)m * ch.n;
    for (int z = 0; z < ch.nz; ++z) {
      const long long loc = z * nxny + (long long)y * ch.nx + x;
      const long long a = ch.off + loc;
      const Coef64 c4 = ps_coef(g, a);
      const double c = (double)tf[loc];
      double r = c4.w * c;
      if (x + 1 < ch.nx) r += c4.x * (c - (double)tf[loc + 1]);
      if (x > 0) r += ps_coef(g, a - 1).x * (c - (double)tf[loc - 1]);
      if (y + 1 < ch.ny) r += c4.y * (c - (double)tf[loc + ch.nx]);
      if (y > 0) r += ps_coef(g, a - ch.nx).y * (c - (double)tf[loc - ch.nx]);
      if (z + 1 < ch.nz) r += c4.z * (c - (double)tf[loc + nxny]);
      if (z > 0) r += ps_coef(g, a - nxny).z * (c - (double)tf[loc - nxny]);
      const double qv = (double)qf[loc];
      num += (r - qv) * (r - qv);
      den += qv * qv;
    }
  }
  __shared__ double sn[PS_X * PS_Y / 32], sd[PS_X * PS_Y / 32];
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_xor_sync(0xffffffffu, num, o);
    den += __shfl_xor_sync(0xffffffffu, den, o);
  }
  const int t = threadIdx.y * PS_X + threadIdx.x;
  if ((t & 31) == 0) { sn[t >> 5] = num; sd[t >> 5] = den; }
  __syncthreads();
  if (t == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < PS_X * PS_Y / 32; ++w) { a += sn[w]; b += sd[w]; }
    const long long p = (long long)blockIdx.z * M + m;
    atomicAdd(&acc[2 * p], a);
    atomicAdd(&acc[2 * p + 1], b);
  }
}

__global__ void ps_finish_kernel(const double *__restrict__ acc, double *__restrict__ e, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double num = acc[2 * i], den = acc[2 * i + 1];
    e[i] = den > 0.0 ? sqrt(num / den) : sqrt(num);
  }
}

// Device address of the scratch array, looked up once per device.
static double *scratch_for_current_device(int *status) {
  static std::mutex mu;
  static double *ptrs[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { *status = cuda_status(e, "pair_check_static: cudaGetDevice"); return nullptr; }
  if (dev < 0 || dev >= 64) { *status = BLOCKOA_ERR_INVALID; return nullptr; }
  std::lock_guard<std::mutex> lock(mu);
  if (!ptrs[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_pair_scratch);
    if (e != cudaSuccess || !p) {
      *status = cuda_status(e != cudaSuccess ? e : cudaErrorInvalidSymbol,
                            "pair_check_static: cudaGetSymbolAddress");
      return nullptr;
    }
    ptrs[dev] = (double *)p;
  }
  *status = BLOCKOA_OK;
  return ptrs[dev];
}

}  // namespace blockoa

using namespace blockoa;

extern "C" int blockoa_pair_check_static(const blockoa_operator *op, const void *T, const void *q,
                                         int M, int dtype, double *e_pair, blockoa_stream stream) {
  if (!op || M < 0 || (dtype != BLOCKOA_FP64 && dtype != BLOCKOA_MIXED)) return BLOCKOA_ERR_INVALID;
  if (M == 0) return BLOCKOA_OK;
  if (!T || !q || !e_pair || M > 65535 || op->n_chips > 65535) return BLOCKOA_ERR_INVALID;
  const long long n_pairs = (long long)op->n_chips * M;
  if (n_pairs > kStaticPairMax) {
    set_last_error(cudaErrorInvalidValue,
                   "blockoa_pair_check_static: n_chips * M exceeds BLOCKOA_STATIC_PAIR_MAX");
    return BLOCKOA_ERR_INVALID;
  }
  int rc = BLOCKOA_OK;
  double *acc = scratch_for_current_device(&rc);
  if (rc) return rc;
  int max_tiles = 1;
  for (const ChipDev &c : op->chips) {
    const int t = ((c.nx + PS_X - 1) / PS_X) * ((c.ny + PS_Y - 1) / PS_Y);
    if (t > max_tiles) max_tiles = t;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int n_acc = (int)(2 * n_pairs);
  ps_clear_kernel<<<(n_acc + 255) / 256, 256, 0, st>>>(acc, n_acc);
  dim3 grid((unsigned)max_tiles, (unsigned)M, (unsigned)op->n_chips);
  dim3 block(PS_X, PS_Y);
  if (dtype == BLOCKOA_FP64)
    ps_check_kernel<double><<<grid, block, 0, st>>>(op->d_chips, op->g64, (const double *)T,
                                                    (const double *)q, M, acc);
  else
    ps_check_kernel<float><<<grid, block, 0, st>>>(op->d_chips, op->g64, (const float *)T,
                                                   (const float *)q, M, acc);
  ps_finish_kernel<<<(int)((n_pairs + 255) / 256), 256, 0, st>>>(acc, e_pair, (int)n_pairs);
  g_launches += 3;
  return cuda_status(cudaGetLastError(), "pair_check_static");
}
