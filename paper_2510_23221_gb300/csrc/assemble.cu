// Operator assembly (Eq. 1 -> Eq. 2, Sec. II-B), right-hand sides (Eq. 2),
// operator lifetime, status strings and shared host utilities.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <algorithm>

#include "common.cuh"

namespace blockoa {

static thread_local char g_last_error[256] = "";
std::atomic<long long> g_launches{0};

void time_begin(blockoa_operator *op, cudaStream_t st, cudaEvent_t *ev) {
  (void)op;
  *ev = nullptr;
  if (cudaEventCreate(ev) != cudaSuccess) { cudaGetLastError(); *ev = nullptr; return; }
  cudaEventRecord(*ev, st);
}

void time_end(blockoa_operator *op, cudaStream_t st, int kclass, cudaEvent_t ev0) {
  if (!ev0) return;
  cudaEvent_t ev1 = nullptr;
  if (cudaEventCreate(&ev1) != cudaSuccess) { cudaGetLastError(); cudaEventDestroy(ev0); return; }
  cudaEventRecord(ev1, st);
  op->times.pend_class.push_back(kclass);
  op->times.pend_ev.push_back(ev0);
  op->times.pend_ev.push_back(ev1);
  op->times.launches[kclass] += 1;
}

void add_time(blockoa_operator *op, int kclass, double ms) {
  op->times.ms[kclass] += ms;
  op->times.samples[kclass] += 1;
}

void add_launches(blockoa_operator *op, int kclass, long long n) { op->times.launches[kclass] += n; }

static void resolve_times(blockoa_operator *op) {
  KernelTimes &kt = op->times;
  for (size_t i = 0; i < kt.pend_class.size(); ++i) {
    cudaEvent_t a = kt.pend_ev[2 * i], b = kt.pend_ev[2 * i + 1];
    float ms = 0.f;
    if (cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
      add_time(op, kt.pend_class[i], ms);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  cudaGetLastError();
  kt.pend_class.clear();
  kt.pend_ev.clear();
}

void set_last_error(cudaError_t e, const char *where) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s", where, cudaGetErrorString(e));
}

int cuda_status(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return BLOCKOA_OK;
  set_last_error(e, where);
  cudaGetLastError();  // clear a non-sticky error so later calls can proceed
  return e == cudaErrorMemoryAllocation ? BLOCKOA_ERR_OOM : BLOCKOA_ERR_CUDA;
}

static cudaMemPool_t device_pool(int dev) {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!pools[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    uint64_t keep = UINT64_MAX;  // keep freed blocks for reuse by later calls
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = p;
  }
  return pools[dev];
}

int pool_alloc(blockoa_operator *op, void **p, size_t bytes, cudaStream_t st) {
  *p = nullptr;
  if (bytes == 0) return BLOCKOA_OK;
  cudaError_t e = op->pool ? cudaMallocFromPoolAsync(p, bytes, op->pool, st)
                           : cudaMallocAsync(p, bytes, st);
  if (e != cudaSuccess) return cuda_status(e, "workspace allocation");
  return BLOCKOA_OK;
}

void pool_free(void *p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

std::vector<Unit> make_units(const blockoa_operator *op, long long cells) {
  std::vector<Unit> units;
  for (int c = 0; c < op->n_chips; ++c) {
    const ChipDev &ch = op->chips[c];
    for (long long b = 0; b < ch.n; b += cells) {
      Unit u;
      u.chip = c;
      u.pad = 0;
      u.begin = ch.off + b;
      u.end = ch.off + (b + cells < ch.n ? b + cells : ch.n);
      units.push_back(u);
    }
  }
  return units;
}

long long pick_unit_cells(const blockoa_operator *op, long long align, long long min_cells,
                          int target_ctas) {
  long long want = (op->n_total + target_ctas - 1) / target_ctas;
  if (want < min_cells) want = min_cells;
  return (want + align - 1) / align * align;
}

// ---------------------------------------------------------------- assembly
struct ChipPhys {
  double dx, dy, h_top, h_bottom, h_side;
  long long zoff;       // first z-row of the chip in the z tables
  long long kcell_off;  // offset into the per-cell k array, or -1
};

// Face conductance S / (d_a/(2 k_a) + d_b/(2 k_b)), float64 without contraction.
__device__ __forceinline__ double series_g(double area, double da, double ka, double db,
                                           double kb) {
  double ra = __ddiv_rn(da, __dmul_rn(2.0, ka));
  double rb = __ddiv_rn(db, __dmul_rn(2.0, kb));
  return __ddiv_rn(area, __dadd_rn(ra, rb));
}

// Robin face conductance S / (d/(2k) + 1/h).
__device__ __forceinline__ double robin_g(double area, double d, double k, double h) {
  double r = __dadd_rn(__ddiv_rn(d, __dmul_rn(2.0, k)), __ddiv_rn(1.0, h));
  return __ddiv_rn(area, r);
}

__global__ void assemble_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                                const ChipPhys *__restrict__ phys, const double *__restrict__ zk,
                                const double *__restrict__ zdz, const double *__restrict__ kcell,
                                double *__restrict__ g64, float *__restrict__ g32) {
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const ChipPhys ph = phys[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  for (long long a = u.begin + threadIdx.x; a < u.end; a += blockDim.x) {
    const long long loc = a - ch.off;
    const int x = (int)(loc % ch.nx);
    const int y = (int)((loc / ch.nx) % ch.ny);
    const int z = (int)(loc / nxny);
    auto kof = [&](long long l, int zz) -> double {
      return ph.kcell_off >= 0 ? kcell[ph.kcell_off + l] : zk[ph.zoff + zz];
    };
    const double ka = kof(loc, z);
    const double dz = zdz[ph.zoff + z];
    double cx = 0.0, cy = 0.0, cz = 0.0, cb = 0.0;
    if (x + 1 < ch.nx) cx = series_g(__dmul_rn(ph.dy, dz), ph.dx, ka, ph.dx, kof(loc + 1, z));
    if (y + 1 < ch.ny) cy = series_g(__dmul_rn(ph.dx, dz), ph.dy, ka, ph.dy, kof(loc + ch.nx, z));
    if (z + 1 < ch.nz)
      cz = series_g(__dmul_rn(ph.dx, ph.dy), dz, ka, zdz[ph.zoff + z + 1], kof(loc + nxny, z + 1));
    // Robin faces, summed in the order top, bottom, x-low, x-high, y-low, y-high.
    if (ph.h_top > 0.0 && z == 0) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, ph.dy), dz, ka, ph.h_top));
    if (ph.h_bottom > 0.0 && z == ch.nz - 1)
      cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, ph.dy), dz, ka, ph.h_bottom));
    if (ph.h_side > 0.0) {
      if (x == 0) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dy, dz), ph.dx, ka, ph.h_side));
      if (x == ch.nx - 1) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dy, dz), ph.dx, ka, ph.h_side));
      if (y == 0) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, dz), ph.dy, ka, ph.h_side));
      if (y == ch.ny - 1) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, dz), ph.dy, ka, ph.h_side));
    }
    reinterpret_cast<Coef64 *>(g64)[a] = Coef64{cx, cy, cz, cb};
    reinterpret_cast<float4 *>(g32)[a] =
        make_float4((float)cx, (float)cy, (float)cz, (float)cb);
  }
}

// 1 / diag(A) per cell: the sum of the cell's face conductances and its
// Robin conductance (float64, then rounded to float32).
__global__ void inv_diag_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                                const double *__restrict__ g64, double *__restrict__ d64,
                                float *__restrict__ d32) {
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  const Coef64 *g = reinterpret_cast<const Coef64 *>(g64);
  for (long long a = u.begin + threadIdx.x; a < u.end; a += blockDim.x) {
    const long long loc = a - ch.off;
    const int x = (int)(loc % ch.nx), y = (int)((loc / ch.nx) % ch.ny), z = (int)(loc / nxny);
    const Coef64 c = g[a];
    double d = c.x + c.y + c.z + c.w;
    if (x > 0) d += g[a - 1].x;
    if (y > 0) d += g[a - ch.nx].y;
    if (z > 0) d += g[a - nxny].z;
    const double inv = d > 0.0 ? 1.0 / d : 0.0;
    d64[a] = inv;
    d32[a] = (float)inv;
  }
}

// z-line preconditioner factors: M is the part of A that couples cells of
// one (x, y) column (the full diagonal and the vertical conductances), a
// tridiagonal matrix per column.  One thread per column runs the Thomas
// elimination and stores 1 / den_z, den_0 = d_0, den_z = d_z - e_z^2 / den_{z-1}
// with e_z the conductance between z-1 and z (float64, same diagonal sum as
// inv_diag_kernel).  M^-1 r is then, with f_z the conductance from z to z+1,
//   w_z = (r_z + e_z w_{z-1}) / den_z,   x_z = w_z + f_z / den_z x_{z+1}.
__global__ void zfactor_kernel(const ChipDev *__restrict__ chips, int n_chips, const double *__restrict__ g64,
                               double *__restrict__ z64, float *__restrict__ z32) {
  const int c = blockIdx.y;
  if (c >= n_chips) return;
  const ChipDev ch = chips[c];
  const long long nxny = (long long)ch.nx * ch.ny;
  const Coef64 *g = reinterpret_cast<const Coef64 *>(g64);
  for (long long col = blockIdx.x * (long long)blockDim.x + threadIdx.x; col < nxny;
       col += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(col % ch.nx), y = (int)(col / ch.nx);
    double den_prev = 1.0;
    for (int z = 0; z < ch.nz; ++z) {
      const long long a = ch.off + z * nxny + col;
      const Coef64 cf = g[a];
      double d = cf.x + cf.y + cf.z + cf.w;
      if (x > 0) d += g[a - 1].x;
      if (y > 0) d += g[a - ch.nx].y;
      double e = 0.0;
      if (z > 0) {
        e = g[a - nxny].z;
        d += e;
      }
      const double den = z > 0 ? d - e * e / den_prev : d;
      const double inv = den > 0.0 ? 1.0 / den : 0.0;
      z64[a] = inv;
      z32[a] = (float)inv;
      den_prev = den;
    }
  }
}

// One thread per z-row of a layered chip: the row's interior face
// conductances and the Robin conductance of every edge class, with the same
// float64 operations (and order) as assemble_kernel.
__global__ void layer_table_kernel(const ChipDev *__restrict__ chips, const ChipPhys *__restrict__ phys,
                                   const double *__restrict__ zk, const double *__restrict__ zdz,
                                   int n_chips, double *__restrict__ lt64, float *__restrict__ lt32) {
  const int c = blockIdx.x;
  if (c >= n_chips) return;
  const ChipDev ch = chips[c];
  const ChipPhys ph = phys[c];
  if (!ch.layered) return;
  for (int z = threadIdx.x; z < ch.nz; z += blockDim.x) {
    const double ka = zk[ph.zoff + z], dz = zdz[ph.zoff + z];
    double rec[kLT];
    for (int i = 0; i < kLT; ++i) rec[i] = 0.0;
    rec[0] = ch.nx > 1 ? series_g(__dmul_rn(ph.dy, dz), ph.dx, ka, ph.dx, ka) : 0.0;
    rec[1] = ch.ny > 1 ? series_g(__dmul_rn(ph.dx, dz), ph.dy, ka, ph.dy, ka) : 0.0;
    rec[2] = z + 1 < ch.nz ? series_g(__dmul_rn(ph.dx, ph.dy), dz, ka, zdz[ph.zoff + z + 1], zk[ph.zoff + z + 1]) : 0.0;
    for (int cx = 0; cx < 4; ++cx)
      for (int cy = 0; cy < 4; ++cy) {
        double cb = 0.0;
        if (ph.h_top > 0.0 && z == 0) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, ph.dy), dz, ka, ph.h_top));
        if (ph.h_bottom > 0.0 && z == ch.nz - 1)
          cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, ph.dy), dz, ka, ph.h_bottom));
        if (ph.h_side > 0.0) {
          if (cx & 1) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dy, dz), ph.dx, ka, ph.h_side));
          if (cx & 2) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dy, dz), ph.dx, ka, ph.h_side));
          if (cy & 1) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, dz), ph.dy, ka, ph.h_side));
          if (cy & 2) cb = __dadd_rn(cb, robin_g(__dmul_rn(ph.dx, dz), ph.dy, ka, ph.h_side));
        }
        rec[4 + 4 * cx + cy] = cb;
      }
    for (int i = 0; i < kLT; ++i) {
      lt64[(ch.lz + z) * kLT + i] = rec[i];
      lt32[(ch.lz + z) * kLT + i] = (float)rec[i];
    }
  }
}

// ---------------------------------------------------------------- right-hand sides
struct RhsChip {
  double area;          // dx * dy
  long long dens_off;   // offset of the chip's [s][ny][nx] density block
};

__global__ void build_rhs_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                                 const RhsChip *__restrict__ rc, const double *__restrict__ dens,
                                 double *__restrict__ B, int s) {
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const RhsChip r = rc[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  const long long total = (u.end - u.begin) * s;
  for (long long t = threadIdx.x; t < total; t += blockDim.x) {
    const long long a = u.begin + t / s;
    const int j = (int)(t % s);
    const long long loc = a - ch.off;
    double v = 0.0;
    if (loc < nxny) v = __dmul_rn(dens[r.dens_off + (long long)j * nxny + loc], r.area);
    B[a * s + j] = v;
  }
}

// Volumetric sources: B[a][j] = qv_j(a) * V(a), V = dx dy dz of the cell's
// z-row (per-z-row volumes computed on the host, indexed by ChipDev::lz).
__global__ void build_rhs_volume_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                                        const long long *__restrict__ q_off, const double *__restrict__ vol,
                                        const double *__restrict__ qv, double *__restrict__ B, int s) {
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const long long nxny = (long long)ch.nx * ch.ny;
  const long long base = q_off[u.chip];
  const long long total = (u.end - u.begin) * s;
  for (long long t = threadIdx.x; t < total; t += blockDim.x) {
    const long long a = u.begin + t / s;
    const int j = (int)(t % s);
    const long long loc = a - ch.off;
    B[a * s + j] = __dmul_rn(qv[base + (long long)j * ch.n + loc], vol[ch.lz + loc / nxny]);
  }
}

}  // namespace blockoa

using namespace blockoa;

// ---------------------------------------------------------------- C ABI
extern "C" const char *blockoa_status_string(int status) {
  switch (status) {
    case BLOCKOA_OK: return "ok";
    case BLOCKOA_ERR_INVALID: return "invalid argument";
    case BLOCKOA_ERR_CUDA: return "CUDA error";
    case BLOCKOA_ERR_BREAKDOWN: return "breakdown (NaN/Inf or rank-0 Gram matrix)";
    case BLOCKOA_ERR_NOT_CONVERGED: return "not converged within maxiter";
    case BLOCKOA_ERR_TIMEOUT: return "device wait timed out";
    case BLOCKOA_ERR_OOM: return "out of device memory";
    default: return "unknown status";
  }
}

extern "C" const char *blockoa_last_error(void) { return g_last_error; }

static bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }
// film coefficient: >= 0, and +inf for a face held at the reference temperature
static bool film_ok(double v) { return v >= 0.0 && !std::isnan(v); }

namespace blockoa {
__global__ void read_small_kernel(const unsigned long long *__restrict__ src, unsigned long long *dst, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}
}  // namespace blockoa

cudaError_t blockoa::read_small(void *host_pinned, const void *dev, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  void *dptr = nullptr;
  cudaError_t e = cudaHostGetDevicePointer(&dptr, host_pinned, 0);
  if (e != cudaSuccess) return e;
  g_launches += 1;
  read_small_kernel<<<1, 256, 0, st>>>((const unsigned long long *)dev, (unsigned long long *)dptr,
                                       (int)(bytes / 8));
  return cudaGetLastError();
}

// Host-side validation of the chip descriptions and the tables the assembly
// kernels read.
struct ChipTables {
  std::vector<ChipDev> tab;
  std::vector<ChipPhys> phys;
  std::vector<double> zk, zdz, kcell;
  long long n_total = 0;
};

static int build_tables(const blockoa_chip_desc *chips, int n_chips, ChipTables &t) {
  if (!chips || n_chips <= 0) return BLOCKOA_ERR_INVALID;
  t.tab.assign(n_chips, ChipDev());
  t.phys.assign(n_chips, ChipPhys());
  long long off = 0;
  for (int c = 0; c < n_chips; ++c) {
    const blockoa_chip_desc &d = chips[c];
    if (d.nx < 1 || d.ny < 1 || d.n_layers < 1 || !d.layer_nz || !d.layer_dz) return BLOCKOA_ERR_INVALID;
    if (!d.k_cell && !d.layer_k) return BLOCKOA_ERR_INVALID;
    if (!finite_pos(d.dx) || !finite_pos(d.dy)) return BLOCKOA_ERR_INVALID;
    if (!film_ok(d.h_top) || !film_ok(d.h_bottom) || !film_ok(d.h_side))
      return BLOCKOA_ERR_INVALID;
    long long nz = 0;
    ChipPhys ph;
    ph.dx = d.dx; ph.dy = d.dy; ph.h_top = d.h_top; ph.h_bottom = d.h_bottom; ph.h_side = d.h_side;
    ph.zoff = (long long)t.zk.size();
    for (int l = 0; l < d.n_layers; ++l) {
      if (d.layer_nz[l] < 1 || !finite_pos(d.layer_dz[l])) return BLOCKOA_ERR_INVALID;
      double kl = d.layer_k ? d.layer_k[l] : 1.0;
      if (!d.k_cell && !finite_pos(kl)) return BLOCKOA_ERR_INVALID;
      for (int r = 0; r < d.layer_nz[l]; ++r) {
        t.zk.push_back(kl);
        t.zdz.push_back(d.layer_dz[l]);
      }
      nz += d.layer_nz[l];
    }
    if (nz > (1 << 30)) return BLOCKOA_ERR_INVALID;
    long long n = (long long)d.nx * d.ny * nz;
    if (n > (1LL << 40)) return BLOCKOA_ERR_INVALID;
    ph.kcell_off = -1;
    if (d.k_cell) {
      ph.kcell_off = (long long)t.kcell.size();
      for (long long i = 0; i < n; ++i) {
        if (!finite_pos(d.k_cell[i])) return BLOCKOA_ERR_INVALID;
        t.kcell.push_back(d.k_cell[i]);
      }
    }
    t.tab[c].nx = d.nx; t.tab[c].ny = d.ny; t.tab[c].nz = (int)nz;
    t.tab[c].layered = d.k_cell ? 0 : 1;
    t.tab[c].n = n; t.tab[c].off = off;
    t.tab[c].lz = ph.zoff;
    t.phys[c] = ph;
    off += n;
  }
  t.n_total = off;
  return BLOCKOA_OK;
}

// Upload the tables and run the assembly kernels into the operator's
// (already allocated) arrays: conductances, 1/diag, z-line factors, layer
// tables.  Temporaries come from the stream-ordered pool.
static int run_assembly(blockoa_operator *op, const ChipTables &t, cudaStream_t st) {
  const int n_chips = op->n_chips;
  std::vector<Unit> units = make_units(op, 4096);
  void *d_units = nullptr, *d_phys = nullptr, *d_zk = nullptr, *d_zdz = nullptr, *d_kc = nullptr;
  auto done = [&](int code) {
    pool_free(d_units, st); pool_free(d_phys, st); pool_free(d_zk, st);
    pool_free(d_zdz, st); pool_free(d_kc, st);
    return code;
  };
  int rc;
  if ((rc = pool_alloc(op, &d_units, sizeof(Unit) * units.size(), st))) return done(rc);
  if ((rc = pool_alloc(op, &d_phys, sizeof(ChipPhys) * n_chips, st))) return done(rc);
  if ((rc = pool_alloc(op, &d_zk, sizeof(double) * t.zk.size(), st))) return done(rc);
  if ((rc = pool_alloc(op, &d_zdz, sizeof(double) * t.zdz.size(), st))) return done(rc);
  if (!t.kcell.empty() && (rc = pool_alloc(op, &d_kc, sizeof(double) * t.kcell.size(), st))) return done(rc);
  // Host tables are pageable; cudaMemcpyAsync from pageable memory returns
  // only after the source has been consumed, so the vectors may die after.
  cudaError_t e = cudaMemcpyAsync(op->d_chips, t.tab.data(), sizeof(ChipDev) * n_chips, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_phys, t.phys.data(), sizeof(ChipPhys) * n_chips, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_zk, t.zk.data(), sizeof(double) * t.zk.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_zdz, t.zdz.data(), sizeof(double) * t.zdz.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && d_kc) e = cudaMemcpyAsync(d_kc, t.kcell.data(), sizeof(double) * t.kcell.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return done(cuda_status(e, "upload chip tables"));
  g_launches += 1;
  assemble_kernel<<<(unsigned)units.size(), 256, 0, st>>>(
      (const Unit *)d_units, op->d_chips, (const ChipPhys *)d_phys, (const double *)d_zk,
      (const double *)d_zdz, (const double *)d_kc, op->g64, op->g32);
  e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_status(e, "assemble_kernel"));
  g_launches += 2;
  inv_diag_kernel<<<(unsigned)units.size(), 256, 0, st>>>((const Unit *)d_units, op->d_chips, op->g64,
                                                          op->dinv64, op->dinv32);
  {
    long long maxcols = 1;
    for (const ChipDev &cd : op->chips) maxcols = std::max<long long>(maxcols, (long long)cd.nx * cd.ny);
    dim3 zg((unsigned)std::min<long long>((maxcols + 255) / 256, 1024), (unsigned)n_chips);
    zfactor_kernel<<<zg, 256, 0, st>>>(op->d_chips, n_chips, op->g64, op->zinv64, op->zinv32);
    g_launches += 1;
  }
  layer_table_kernel<<<(unsigned)n_chips, 64, 0, st>>>(op->d_chips, (const ChipPhys *)d_phys,
                                                      (const double *)d_zk, (const double *)d_zdz,
                                                      n_chips, op->lt64, op->lt32);
  e = cudaGetLastError();
  if (e != cudaSuccess) return done(cuda_status(e, "layer_table_kernel"));
  return done(BLOCKOA_OK);
}

extern "C" int blockoa_assemble(const blockoa_chip_desc *chips, int n_chips,
                                blockoa_stream stream, blockoa_operator **out) {
  if (!out) return BLOCKOA_ERR_INVALID;
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)stream;
  ChipTables t;
  int rc = build_tables(chips, n_chips, t);
  if (rc) return rc;

  blockoa_operator *op = new blockoa_operator();
  cudaGetDevice(&op->device);
  op->pool = device_pool(op->device);
  op->n_chips = n_chips;
  op->n_total = t.n_total;
  op->chips = t.tab;
  op->n_zrows = (long long)t.zk.size();
  op->cell_area.resize(n_chips);
  for (int c = 0; c < n_chips; ++c) op->cell_area[c] = chips[c].dx * chips[c].dy;
  op->zrow_dz = t.zdz;
  auto fail = [&](int code) {
    blockoa_destroy(op);
    return code;
  };
  cudaError_t e;
  e = cudaMalloc((void **)&op->d_chips, sizeof(ChipDev) * n_chips);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc chips"));
  e = cudaMalloc((void **)&op->g64, sizeof(double) * 4 * op->n_total);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc g64"));
  e = cudaMalloc((void **)&op->g32, sizeof(float) * 4 * op->n_total);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc g32"));
  e = cudaMalloc((void **)&op->dinv64, sizeof(double) * op->n_total);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc dinv64"));
  e = cudaMalloc((void **)&op->dinv32, sizeof(float) * op->n_total);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc dinv32"));
  e = cudaMalloc((void **)&op->zinv64, sizeof(double) * op->n_total);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc zinv64"));
  e = cudaMalloc((void **)&op->zinv32, sizeof(float) * op->n_total);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc zinv32"));
  e = cudaMalloc((void **)&op->lt64, sizeof(double) * kLT * t.zk.size());
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc lt64"));
  e = cudaMalloc((void **)&op->lt32, sizeof(float) * kLT * t.zk.size());
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMalloc lt32"));
  e = cudaMallocHost((void **)&op->h_flag, 2 * sizeof(int));
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaMallocHost flag"));
  if ((rc = run_assembly(op, t, st))) return fail(rc);
  *out = op;
  return BLOCKOA_OK;
}

extern "C" int blockoa_reassemble(blockoa_operator *op, const blockoa_chip_desc *chips, int n_chips,
                                  blockoa_stream stream) {
  if (!op) return BLOCKOA_ERR_INVALID;
  ChipTables t;
  int rc = build_tables(chips, n_chips, t);
  if (rc) return rc;
  // same geometry: chip count, grid of every chip and layer rows
  if (n_chips != op->n_chips || t.n_total != op->n_total || (long long)t.zk.size() != op->n_zrows)
    return BLOCKOA_ERR_INVALID;
  for (int c = 0; c < n_chips; ++c) {
    const ChipDev &a = t.tab[c], &b = op->chips[c];
    if (a.nx != b.nx || a.ny != b.ny || a.nz != b.nz || a.n != b.n || a.off != b.off || a.lz != b.lz)
      return BLOCKOA_ERR_INVALID;
  }
  op->chips = t.tab;   // the layered flag may change with the conductivity description
  for (int c = 0; c < n_chips; ++c) op->cell_area[c] = chips[c].dx * chips[c].dy;
  op->zrow_dz = t.zdz;
  return run_assembly(op, t, (cudaStream_t)stream);
}

extern "C" int blockoa_operator_size(const blockoa_operator *op, int chip, int64_t *n_cells,
                                     int64_t *cell_offset, int *nx, int *ny, int *nz) {
  if (!op || chip < 0 || chip >= op->n_chips) return BLOCKOA_ERR_INVALID;
  const ChipDev &c = op->chips[chip];
  if (n_cells) *n_cells = c.n;
  if (cell_offset) *cell_offset = c.off;
  if (nx) *nx = c.nx;
  if (ny) *ny = c.ny;
  if (nz) *nz = c.nz;
  return BLOCKOA_OK;
}

extern "C" int blockoa_operator_total(const blockoa_operator *op, int64_t *n_total, int *n_chips) {
  if (!op) return BLOCKOA_ERR_INVALID;
  if (n_total) *n_total = op->n_total;
  if (n_chips) *n_chips = op->n_chips;
  return BLOCKOA_OK;
}

extern "C" int blockoa_build_rhs(const blockoa_operator *op, const double *density, double *B,
                                 int s, blockoa_stream stream) {
  if (!op || s < 0) return BLOCKOA_ERR_INVALID;
  if (s == 0) return BLOCKOA_OK;
  if (!density || !B) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<RhsChip> rcs(op->n_chips);
  long long doff = 0;
  for (int c = 0; c < op->n_chips; ++c) {
    rcs[c].area = op->cell_area[c];
    rcs[c].dens_off = doff;
    doff += (long long)s * op->chips[c].nx * op->chips[c].ny;
  }
  std::vector<Unit> units = make_units(op, 2048);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_units = nullptr, *d_rc = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (!rc) rc = pool_alloc(mop, &d_rc, sizeof(RhsChip) * rcs.size(), st);
  if (rc) { pool_free(d_units, st); pool_free(d_rc, st); return rc; }
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_rc, rcs.data(), sizeof(RhsChip) * rcs.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    g_launches += 1;
    build_rhs_kernel<<<(unsigned)units.size(), 256, 0, st>>>((const Unit *)d_units, op->d_chips,
                                                           (const RhsChip *)d_rc, density, B, s);
    e = cudaGetLastError();
  }
  pool_free(d_units, st);
  pool_free(d_rc, st);
  return cuda_status(e, "build_rhs");
}

extern "C" int blockoa_build_rhs_volume(const blockoa_operator *op, const double *qv, double *B, int s,
                                        blockoa_stream stream) {
  if (!op || s < 0) return BLOCKOA_ERR_INVALID;
  if (s == 0) return BLOCKOA_OK;
  if (!qv || !B) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<long long> qoff(op->n_chips);
  std::vector<double> vol(op->n_zrows);
  long long off = 0;
  for (int c = 0; c < op->n_chips; ++c) {
    const ChipDev &ch = op->chips[c];
    qoff[c] = off;
    off += (long long)s * ch.n;
    for (int z = 0; z < ch.nz; ++z) vol[ch.lz + z] = op->cell_area[c] * op->zrow_dz[ch.lz + z];
  }
  std::vector<Unit> units = make_units(op, 2048);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_units = nullptr, *d_off = nullptr, *d_vol = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (!rc) rc = pool_alloc(mop, &d_off, sizeof(long long) * qoff.size(), st);
  if (!rc) rc = pool_alloc(mop, &d_vol, sizeof(double) * vol.size(), st);
  if (rc) { pool_free(d_units, st); pool_free(d_off, st); pool_free(d_vol, st); return rc; }
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_off, qoff.data(), sizeof(long long) * qoff.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_vol, vol.data(), sizeof(double) * vol.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    g_launches += 1;
    build_rhs_volume_kernel<<<(unsigned)units.size(), 256, 0, st>>>(
        (const Unit *)d_units, op->d_chips, (const long long *)d_off, (const double *)d_vol, qv, B, s);
    e = cudaGetLastError();
  }
  pool_free(d_units, st);
  pool_free(d_off, st);
  pool_free(d_vol, st);
  return cuda_status(e, "build_rhs_volume");
}

extern "C" int blockoa_export_conductances(const blockoa_operator *op, int chip, double *gx,
                                           double *gy, double *gz, double *gb) {
  if (!op || chip < 0 || chip >= op->n_chips) return BLOCKOA_ERR_INVALID;
  const ChipDev &c = op->chips[chip];
  std::vector<double> g((size_t)c.n * 4);
  BLOCKOA_CUDA(cudaDeviceSynchronize());
  BLOCKOA_CUDA(cudaMemcpy(g.data(), op->g64 + 4 * c.off, sizeof(double) * 4 * c.n,
                          cudaMemcpyDeviceToHost));
  size_t ix = 0, iy = 0, iz = 0;
  for (int z = 0; z < c.nz; ++z)
    for (int y = 0; y < c.ny; ++y)
      for (int x = 0; x < c.nx; ++x) {
        size_t a = ((size_t)z * c.ny + y) * c.nx + x;
        if (gx && x + 1 < c.nx) gx[ix] = g[4 * a + 0];
        if (x + 1 < c.nx) ++ix;
        if (gy && y + 1 < c.ny) gy[iy] = g[4 * a + 1];
        if (y + 1 < c.ny) ++iy;
        if (gz && z + 1 < c.nz) gz[iz] = g[4 * a + 2];
        if (z + 1 < c.nz) ++iz;
        if (gb) gb[a] = g[4 * a + 3];
      }
  return BLOCKOA_OK;
}

extern "C" void blockoa_destroy(blockoa_operator *op) {
  if (!op) return;
  cudaDeviceSynchronize();
  free_solve_ws(op->solve_ws);
  resolve_times(op);
  if (op->apply_blocks) cudaFree(op->apply_blocks);
  if (op->apply_vec_blocks) cudaFree(op->apply_vec_blocks);
  if (op->d_chips) cudaFree(op->d_chips);
  if (op->g64) cudaFree(op->g64);
  if (op->g32) cudaFree(op->g32);
  if (op->dinv64) cudaFree(op->dinv64);
  if (op->dinv32) cudaFree(op->dinv32);
  if (op->zinv64) cudaFree(op->zinv64);
  if (op->zinv32) cudaFree(op->zinv32);
  if (op->lt64) cudaFree(op->lt64);
  if (op->lt32) cudaFree(op->lt32);
  if (op->h_flag) cudaFreeHost(op->h_flag);
  cudaGetLastError();
  delete op;
}

static const char *kKernelNames[KC_COUNT] = {
    "spmm_gram", "alpha_solve", "update_gram", "beta_solve", "p_update",
    "residual64", "combine_tc", "split_bf16x3", "apply_fields", "combine_fp64", "zline_second",
    "combine_apply"};

extern "C" int blockoa_kernel_times(blockoa_operator *op, int max_kernels, double *timed_ms,
                                    long long *timed_launches, long long *launches,
                                    const char **names) {
  if (!op || max_kernels < 0) return BLOCKOA_ERR_INVALID;
  resolve_times(op);
  const int n = max_kernels < KC_COUNT ? max_kernels : KC_COUNT;
  for (int k = 0; k < n; ++k) {
    if (timed_ms) timed_ms[k] = op->times.ms[k];
    if (timed_launches) timed_launches[k] = op->times.samples[k];
    if (launches) launches[k] = op->times.launches[k];
    if (names) names[k] = kKernelNames[k];
  }
  return KC_COUNT;
}

extern "C" int blockoa_reset_kernel_times(blockoa_operator *op) {
  if (!op) return BLOCKOA_ERR_INVALID;
  resolve_times(op);
  for (int k = 0; k < KC_COUNT; ++k) {
    op->times.ms[k] = 0.0;
    op->times.samples[k] = 0;
    op->times.launches[k] = 0;
  }
  return BLOCKOA_OK;
}

extern "C" long long blockoa_launch_count(void) { return g_launches.load(); }
