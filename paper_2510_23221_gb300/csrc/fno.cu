// Fourier neural operator for the learned warm start of block CG: forward,
// backward and Adam, in hand-written kernels (float32 arithmetic, bfloat16
// weight copies).  The network and its adjoints are spelled out in
// include/blockoa.h; the data layout is channels-last: activations
// [batch][cell][channel] with cells in (z, y, x) order, x fastest.
//
// The truncated transform runs as three separable stages, each a small
// dense contraction against a twiddle table exp(-2 pi i k n / N) computed on
// the host in float64:
//   x (real -> complex, one CTA per grid row, row and twiddles in shared
//   memory), y and z (complex -> complex, one thread per output); the
//   inverse runs the same stages backwards with conjugate twiddles, the
//   per-kz weights w_c and 1/(nx ny nz), taking the real part in the x stage.
// The backward pass reuses them: the gradient of the mode coefficients is a
// forward transform of the layer's output gradient with weights w_c/N, and
// the gradient of the layer input is an unweighted inverse transform.
// Per-mode channel mixing (and its gradient, accumulated without atomics:
// one CTA owns one mode) keeps the 32 x 32 complex weights in shared memory.
#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "common.cuh"

struct blockoa_fno {
  int device = 0;
  blockoa_fno_shape sh{};
  long long n_params = 0;
  long long oP = 0, obP = 0, oW = 0, ob = 0, oRr = 0, oRi = 0, oQ1 = 0, oc1 = 0, oQ2 = 0, oc2 = 0;
  float *params = nullptr, *grads = nullptr, *m1 = nullptr, *m2 = nullptr;
  __nv_bfloat16 *wb = nullptr;    // bfloat16 copy of the parameters
  float2 *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr;   // exp(-2 pi i k n / N)
  float *wz = nullptr;            // [3][mz]: inverse weights w_c, ones, backward w_c / N
  float *v = nullptr, *u = nullptr, *a1 = nullptr, *h = nullptr, *kbuf = nullptr, *d1 = nullptr,
        *d2 = nullptr;
  float2 *xh = nullptr, *yh = nullptr, *dxh = nullptr, *s1 = nullptr, *s2 = nullptr;
  const float *x_keep = nullptr;  // input of the last forward with keep = 1 (caller memory)
  int kept_batch = 0;
  std::vector<void *> allocs;
};

namespace blockoa {

namespace {

constexpr int FNO_W = 32;

__device__ __forceinline__ float gelu_f(float x) { return x * 0.5f * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.f + erff(x * 0.70710678118654752f)) + x * __expf(-0.5f * x * x) * 0.39894228040143268f;
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmul_conj_b(float2 a, float2 b) {   // a conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// ---------------------------------------------------------------- pointwise layers
// y[n][o] = act(sum_i W'[o][i] x[n][i] + bias[o] + add[n][o]) for CO outputs in
// chunks of COC per thread.  W' is the layer's weight W [CO][CI] or, with
// trans, the transpose of a stored [CI][CO] matrix (the backward pass of a
// layer).  pre (optional) receives the value before the activation.
template <int CI, int COC>
__global__ void __launch_bounds__(256) pw_fwd_kernel(const float *__restrict__ x, long long rows, int CO,
                                                     const __nv_bfloat16 *__restrict__ w, int trans,
                                                     const float *__restrict__ bias,
                                                     const float *__restrict__ add, float *__restrict__ pre,
                                                     float *__restrict__ y, int act, int accumulate) {
  extern __shared__ float sw[];   // [CO][CI]
  for (int e = threadIdx.x; e < CO * CI; e += blockDim.x) {
    const int o = e / CI, i = e % CI;
    sw[e] = __bfloat162float(trans ? w[(long long)i * CO + o] : w[e]);
  }
  __syncthreads();
  const int chunks = CO / COC;
  const long long items = rows * chunks;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < items;
       it += (long long)gridDim.x * blockDim.x) {
    const int ch = (int)(it / rows);   // threads of a warp share the chunk (broadcast weight reads)
    const long long r = it % rows;
    float acc[COC];
#pragma unroll
    for (int c = 0; c < COC; ++c) acc[c] = bias ? bias[ch * COC + c] : 0.f;
    const float *xr = x + r * CI;
#pragma unroll 4
    for (int i = 0; i < CI; ++i) {
      const float xi = xr[i];
#pragma unroll
      for (int c = 0; c < COC; ++c) acc[c] = fmaf(sw[(ch * COC + c) * CI + i], xi, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < COC; ++c) {
      const long long k = r * CO + ch * COC + c;
      float val = acc[c] + (add ? add[k] : 0.f);
      if (pre) pre[k] = val;
      if (act) val = gelu_f(val);
      y[k] = accumulate ? y[k] + val : val;
    }
  }
}

// dW[o][i] += sum_n dy[n][o] x[n][i], db[o] += sum_n dy[n][o]: persistent CTAs
// stage 32-row tiles of x and dy in shared memory; each thread owns fixed
// (o, i) entries and adds them once at the end.
template <int CI, int CO>
__global__ void __launch_bounds__(256) pw_grad_kernel(const float *__restrict__ x, const float *__restrict__ dy,
                                                      long long rows, float *__restrict__ dW,
                                                      float *__restrict__ db) {
  constexpr int TR = 32;
  constexpr int NE = CO * CI + CO;                 // weights then biases
  constexpr int EPT = (NE + 255) / 256;
  __shared__ float sx[TR][CI], sd[TR][CO];
  float acc[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) acc[k] = 0.f;
  const long long per = (rows + gridDim.x - 1) / gridDim.x;
  const long long r0 = blockIdx.x * per, r1 = r0 + per < rows ? r0 + per : rows;
  for (long long base = r0; base < r1; base += TR) {
    const int nr = (int)(r1 - base < TR ? r1 - base : TR);
    __syncthreads();
    for (int e = threadIdx.x; e < TR * CI; e += 256) sx[e / CI][e % CI] = e / CI < nr ? x[(base + e / CI) * CI + e % CI] : 0.f;
    for (int e = threadIdx.x; e < TR * CO; e += 256) sd[e / CO][e % CO] = e / CO < nr ? dy[(base + e / CO) * CO + e % CO] : 0.f;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int e = threadIdx.x + 256 * k;
      if (e < CO * CI) {
        const int o = e / CI, i = e % CI;
        float s = acc[k];
        for (int r = 0; r < TR; ++r) s = fmaf(sd[r][o], sx[r][i], s);
        acc[k] = s;
      } else if (e < NE) {
        const int o = e - CO * CI;
        float s = acc[k];
        for (int r = 0; r < TR; ++r) s += sd[r][o];
        acc[k] = s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    const int e = threadIdx.x + 256 * k;
    if (e < CO * CI) atomicAdd(dW + e, acc[k]);
    else if (e < NE) atomicAdd(db + (e - CO * CI), acc[k]);
  }
}

// g[k] *= gelu'(u[k])
__global__ void gelu_bwd_kernel(float *__restrict__ g, const float *__restrict__ u, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    g[k] *= gelu_grad_f(u[k]);
}

// ---------------------------------------------------------------- truncated transform
// x stage, forward: out[r][a][i] = sum_x tw_x[a][x] in[r][x][i] (real in).
__global__ void __launch_bounds__(256) dft_x_fwd_kernel(const float *__restrict__ in, float2 *__restrict__ out,
                                                        const float2 *__restrict__ tw, int nx, int mx) {
  extern __shared__ float smx[];   // [nx][W] row, then [mx][nx] twiddles
  float *row = smx;
  float2 *t = reinterpret_cast<float2 *>(smx + nx * FNO_W);
  const long long r = blockIdx.x;
  for (int e = threadIdx.x; e < nx * FNO_W; e += blockDim.x) row[e] = in[r * nx * FNO_W + e];
  for (int e = threadIdx.x; e < mx * nx; e += blockDim.x) t[e] = tw[e];
  __syncthreads();
  for (int o = threadIdx.x; o < mx * FNO_W; o += blockDim.x) {
    const int a = o / FNO_W, i = o % FNO_W;
    float re = 0.f, im = 0.f;
    for (int xx = 0; xx < nx; ++xx) {
      const float v = row[xx * FNO_W + i];
      const float2 w = t[a * nx + xx];
      re = fmaf(w.x, v, re);
      im = fmaf(w.y, v, im);
    }
    out[(r * mx + a) * FNO_W + i] = make_float2(re, im);
  }
}

// x stage, inverse: out[r][x][i] (=|+=) scale * sum_a Re(in[r][a][i] conj(tw_x[a][x])).
__global__ void __launch_bounds__(256) dft_x_inv_kernel(const float2 *__restrict__ in, float *__restrict__ out,
                                                        const float2 *__restrict__ tw, int nx, int mx,
                                                        float scale, int accumulate) {
  extern __shared__ float smx[];
  float2 *coef = reinterpret_cast<float2 *>(smx);   // [mx][W]
  float2 *t = coef + mx * FNO_W;                    // [mx][nx]
  const long long r = blockIdx.x;
  for (int e = threadIdx.x; e < mx * FNO_W; e += blockDim.x) coef[e] = in[r * mx * FNO_W + e];
  for (int e = threadIdx.x; e < mx * nx; e += blockDim.x) t[e] = tw[e];
  __syncthreads();
  for (int o = threadIdx.x; o < nx * FNO_W; o += blockDim.x) {
    const int xx = o / FNO_W, i = o % FNO_W;
    float s = 0.f;
    for (int a = 0; a < mx; ++a) {
      const float2 c = coef[a * FNO_W + i];
      const float2 w = t[a * nx + xx];
      s = fmaf(c.x, w.x, s);   // Re(c conj(w)) = c.x w.x + c.y w.y
      s = fmaf(c.y, w.y, s);
    }
    const long long k = (r * nx + xx) * FNO_W + i;
    out[k] = accumulate ? out[k] + scale * s : scale * s;
  }
}

// y stage: forward out[q][b][a][i] = sum_y tw_y[b][y] in[q][y][a][i];
// inverse out[q][y][a][i] = sum_b conj(tw_y[b][y]) in[q][b][a][i].
template <bool FWD>
__global__ void dft_y_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw,
                             long long nq, int ny, int my, int mx) {
  const int nin = FWD ? ny : my, nout = FWD ? my : ny;
  const long long total = nq * nout * mx * FNO_W;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % FNO_W);
    const int a = (int)((o / FNO_W) % mx);
    const int j = (int)((o / ((long long)FNO_W * mx)) % nout);
    const long long q = o / ((long long)FNO_W * mx * nout);
    const float2 *src = in + ((q * nin) * mx + a) * FNO_W + i;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < nin; ++k) {
      const float2 v = src[(long long)k * mx * FNO_W];
      const float2 w = FWD ? tw[j * ny + k] : tw[k * ny + j];
      const float2 p = FWD ? cmul(w, v) : cmul_conj_b(v, w);
      re += p.x;
      im += p.y;
    }
    out[o] = make_float2(re, im);
  }
}

// z stage: forward out[n][c][p][i] = wz[c] sum_z tw_z[c][z] in[n][z][p][i];
// inverse out[n][z][p][i] = sum_c wz[c] conj(tw_z[c][z]) in[n][c][p][i].
template <bool FWD>
__global__ void dft_z_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, const float2 *__restrict__ tw,
                             const float *__restrict__ wz, int batch, int nz, int mz, int np) {
  const int nin = FWD ? nz : mz, nout = FWD ? mz : nz;
  const long long total = (long long)batch * nout * np * FNO_W;
  for (long long o = blockIdx.x * (long long)blockDim.x + threadIdx.x; o < total; o += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(o % FNO_W);
    const int p = (int)((o / FNO_W) % np);
    const int j = (int)((o / ((long long)FNO_W * np)) % nout);
    const long long n = o / ((long long)FNO_W * np * nout);
    float re = 0.f, im = 0.f;
    for (int k = 0; k < nin; ++k) {
      const float2 v = in[((n * nin + k) * np + p) * FNO_W + i];
      const float2 w = FWD ? tw[j * nz + k] : tw[k * nz + j];
      const float s = FWD ? 1.f : wz[k];
      const float2 q = FWD ? cmul(w, v) : cmul_conj_b(v, w);
      re = fmaf(s, q.x, re);
      im = fmaf(s, q.y, im);
    }
    const float s = FWD ? wz[j] : 1.f;
    out[o] = make_float2(s * re, s * im);
  }
}

// ---------------------------------------------------------------- mode mixing
// yh[n][m][o] = sum_i xh[n][m][i] R[m][i][o]; one CTA per mode.
__global__ void __launch_bounds__(256) mix_fwd_kernel(const float2 *__restrict__ xh, float2 *__restrict__ yh,
                                                      const __nv_bfloat16 *__restrict__ rr,
                                                      const __nv_bfloat16 *__restrict__ ri, int batch, int nm) {
  __shared__ float2 R[FNO_W][FNO_W];
  const int m = blockIdx.x;
  for (int e = threadIdx.x; e < FNO_W * FNO_W; e += blockDim.x)
    R[e / FNO_W][e % FNO_W] = make_float2(__bfloat162float(rr[(long long)m * FNO_W * FNO_W + e]),
                                          __bfloat162float(ri[(long long)m * FNO_W * FNO_W + e]));
  __syncthreads();
  const int o = threadIdx.x % FNO_W;
  for (int n = threadIdx.x / FNO_W; n < batch; n += blockDim.x / FNO_W) {
    const float2 *x = xh + ((long long)n * nm + m) * FNO_W;
    float2 acc = make_float2(0.f, 0.f);
    for (int i = 0; i < FNO_W; ++i) {
      const float2 p = cmul(x[i], R[i][o]);
      acc.x += p.x;
      acc.y += p.y;
    }
    yh[((long long)n * nm + m) * FNO_W + o] = acc;
  }
}

// dxh[n][m][i] = sum_o dyh[n][m][o] conj(R[m][i][o]);
// dR[m][i][o] += sum_n conj(xh[n][m][i]) dyh[n][m][o]  (this CTA owns mode m).
__global__ void __launch_bounds__(256) mix_bwd_kernel(const float2 *__restrict__ xh, const float2 *__restrict__ dyh,
                                                      float2 *__restrict__ dxh, const __nv_bfloat16 *__restrict__ rr,
                                                      const __nv_bfloat16 *__restrict__ ri, float *__restrict__ grr,
                                                      float *__restrict__ gri, int batch, int nm) {
  __shared__ float2 R[FNO_W][FNO_W];
  const int m = blockIdx.x;
  const long long wo = (long long)m * FNO_W * FNO_W;
  for (int e = threadIdx.x; e < FNO_W * FNO_W; e += blockDim.x)
    R[e / FNO_W][e % FNO_W] = make_float2(__bfloat162float(rr[wo + e]), __bfloat162float(ri[wo + e]));
  __syncthreads();
  const int lane = threadIdx.x % FNO_W;
  for (int n = threadIdx.x / FNO_W; n < batch; n += blockDim.x / FNO_W) {
    const float2 *dy = dyh + ((long long)n * nm + m) * FNO_W;
    float2 acc = make_float2(0.f, 0.f);
    for (int o = 0; o < FNO_W; ++o) {
      const float2 p = cmul_conj_b(dy[o], R[lane][o]);
      acc.x += p.x;
      acc.y += p.y;
    }
    dxh[((long long)n * nm + m) * FNO_W + lane] = acc;
  }
  for (int e = threadIdx.x; e < FNO_W * FNO_W; e += blockDim.x) {
    const int i = e / FNO_W, o = e % FNO_W;
    float2 acc = make_float2(0.f, 0.f);
    for (int n = 0; n < batch; ++n) {
      const float2 p = cmul_conj_b(dyh[((long long)n * nm + m) * FNO_W + o], xh[((long long)n * nm + m) * FNO_W + i]);
      acc.x += p.x;
      acc.y += p.y;
    }
    grr[wo + e] += acc.x;
    gri[wo + e] += acc.y;
  }
}

// ---------------------------------------------------------------- loss, Adam
__global__ void mse_kernel(const float *__restrict__ y, const float *__restrict__ t, long long n, float *__restrict__ dy,
                           float *__restrict__ loss) {
  __shared__ float part[8];
  float s = 0.f;
  const float inv = 1.f / (float)n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const float d = y[k] - t[k];
    dy[k] = 2.f * d * inv;
    s = fmaf(d, d, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
    atomicAdd(loss, tot * inv);
  }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const float gk = g[k];
    const float mk = b1 * m[k] + (1.f - b1) * gk;
    const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
    m[k] = mk;
    v[k] = vk;
    const float pk = p[k] - lr * (mk / c1) / (sqrtf(vk / c2) + eps);
    p[k] = pk;
    wb[k] = __float2bfloat16(pk);
  }
}

__global__ void to_bf16_kernel(const float *__restrict__ p, __nv_bfloat16 *__restrict__ wb, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
    wb[k] = __float2bfloat16(p[k]);
}

// ---------------------------------------------------------------- host helpers
unsigned grid_for(long long work, int block = 256) {
  long long g = (work + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : (g > 65535LL * 16 ? 65535LL * 16 : g));
}

bool shape_ok(const blockoa_fno_shape *s) {
  return s && s->nx >= 1 && s->ny >= 1 && s->nz >= 1 && s->c_in >= 1 && s->c_in <= 8 && s->width == FNO_W &&
         s->hidden >= 32 && s->hidden <= 256 && s->hidden % 32 == 0 && s->layers >= 1 && s->layers <= 16 &&
         s->mx >= 2 && s->my >= 2 && s->mz >= 1 && s->mx % 2 == 0 && s->my % 2 == 0 && s->mx <= s->nx &&
         s->my <= s->ny && s->mz <= s->nz && s->max_batch >= 1 && s->nx <= 512 && s->ny <= 4096 &&
         s->nz <= 4096 && (long long)s->mx * s->my * s->mz <= 65535;
}

long long count_params(const blockoa_fno_shape &s) {
  const long long W = s.width, L = s.layers, M = (long long)s.mx * s.my * s.mz;
  return W * s.c_in + W + L * W * W + L * W + 2 * L * M * W * W + (long long)s.hidden * W + s.hidden + s.hidden + 1;
}

template <typename P>
cudaError_t fno_alloc(blockoa_fno *net, P **p, size_t bytes) {
  void *q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) {
    net->allocs.push_back(q);
    *p = (P *)q;
  }
  return e;
}

void twiddles(std::vector<float2> &t, int m, int n, bool centred) {
  t.resize((size_t)m * n);
  const double two_pi = 6.283185307179586476925286766559;
  for (int a = 0; a < m; ++a) {
    const long long k = centred ? a - m / 2 : a;
    for (int x = 0; x < n; ++x) {
      const long long kx = (k * x) % n;   // exact phase reduction
      const double th = -two_pi * (double)kx / (double)n;
      t[(size_t)a * n + x] = make_float2((float)std::cos(th), (float)std::sin(th));
    }
  }
}

// Spectral branch of layer l: out = K_l(in) (forward) through the scratch buffers.
void spectral_forward(blockoa_fno *net, int l, const float *in, float *out, int batch, cudaStream_t st) {
  const blockoa_fno_shape &s = net->sh;
  const long long rows = (long long)batch * s.nz * s.ny;
  const int nm = s.mx * s.my * s.mz, np = s.mx * s.my;
  const size_t smx = (size_t)s.nx * FNO_W * sizeof(float) + (size_t)s.mx * s.nx * sizeof(float2);
  float2 *xh = net->xh + (long long)l * s.max_batch * nm * FNO_W;
  dft_x_fwd_kernel<<<(unsigned)rows, 256, smx, st>>>(in, net->s1, net->tw_x, s.nx, s.mx);
  dft_y_kernel<true><<<grid_for((long long)batch * s.nz * s.my * s.mx * FNO_W), 256, 0, st>>>(
      net->s1, net->s2, net->tw_y, (long long)batch * s.nz, s.ny, s.my, s.mx);
  dft_z_kernel<true><<<grid_for((long long)batch * s.mz * np * FNO_W), 256, 0, st>>>(
      net->s2, xh, net->tw_z, net->wz + s.mz, batch, s.nz, s.mz, np);
  const long long R0 = net->oRr + (long long)l * nm * FNO_W * FNO_W;
  const long long I0 = net->oRi + (long long)l * nm * FNO_W * FNO_W;
  mix_fwd_kernel<<<nm, 256, 0, st>>>(xh, net->yh, net->wb + R0, net->wb + I0, batch, nm);
  dft_z_kernel<false><<<grid_for((long long)batch * s.nz * np * FNO_W), 256, 0, st>>>(
      net->yh, net->s2, net->tw_z, net->wz, batch, s.nz, s.mz, np);
  dft_y_kernel<false><<<grid_for((long long)batch * s.nz * s.ny * s.mx * FNO_W), 256, 0, st>>>(
      net->s2, net->s1, net->tw_y, (long long)batch * s.nz, s.ny, s.my, s.mx);
  const size_t smi = (size_t)s.mx * FNO_W * sizeof(float2) + (size_t)s.mx * s.nx * sizeof(float2);
  dft_x_inv_kernel<<<(unsigned)rows, 256, smi, st>>>(net->s1, out, net->tw_x, s.nx, s.mx,
                                                       1.f / ((float)s.nx * s.ny * s.nz), 0);
  g_launches += 7;
}

template <int CI, int COC>
void pw(blockoa_fno *net, const float *x, long long rows, int CO, long long woff, int trans, const float *bias,
        const float *add, float *pre, float *y, int act, int accumulate, cudaStream_t st) {
  const size_t sm = (size_t)CO * CI * sizeof(float);
  pw_fwd_kernel<CI, COC><<<grid_for(rows * (CO / COC)), 256, sm, st>>>(x, rows, CO, net->wb + woff, trans, bias, add,
                                                                      pre, y, act, accumulate);
  g_launches += 1;
}

template <int CI, int CO>
void pw_grad(blockoa_fno *net, const float *x, const float *dy, long long rows, long long woff, long long boff,
             cudaStream_t st) {
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, net->device);
  long long g = (rows + 255) / 256;
  const long long cap = 2LL * nsm;
  pw_grad_kernel<CI, CO><<<(unsigned)(g < cap ? (g < 1 ? 1 : g) : cap), 256, 0, st>>>(x, dy, rows, net->grads + woff,
                                                                                       net->grads + boff);
  g_launches += 1;
}

// Prediction of the basis from the network's per-sample outputs: sample j
// of chip c, y[off_c * s + j * n_c + a], scaled by scale[c * s + j] into the
// block vector X[(off_c + a) * s + j] (float64).
__global__ void fno_basis_kernel(const Unit *__restrict__ units, const ChipDev *__restrict__ chips,
                                 const float *__restrict__ y, const double *__restrict__ scale, int s,
                                 double *__restrict__ X) {
  const Unit u = units[blockIdx.x];
  const ChipDev ch = chips[u.chip];
  const long long total = (u.end - u.begin) * s;
  for (long long i = threadIdx.x; i < total; i += blockDim.x) {
    const long long a = u.begin + i / s;
    const int j = (int)(i % s);
    const float v = y[ch.off * s + (long long)j * ch.n + (a - ch.off)];
    X[a * s + j] = (double)v * scale[(long long)u.chip * s + j];
  }
}

}  // namespace
}  // namespace blockoa

using namespace blockoa;

extern "C" int blockoa_fno_basis(const blockoa_operator *op, const float *y, const double *scale, int s,
                                 double *X, blockoa_stream stream) {
  if (!op || s < 1 || s > 4096 || !y || !scale || !X) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<Unit> units = make_units(op, 512);
  blockoa_operator *mop = const_cast<blockoa_operator *>(op);
  void *d_units = nullptr;
  int rc = pool_alloc(mop, &d_units, sizeof(Unit) * units.size(), st);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(d_units, units.data(), sizeof(Unit) * units.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    g_launches += 1;
    fno_basis_kernel<<<(unsigned)units.size(), 256, 0, st>>>((const Unit *)d_units, op->d_chips, y, scale, s, X);
    e = cudaGetLastError();
  }
  pool_free(d_units, st);
  return cuda_status(e, "blockoa_fno_basis");
}

extern "C" int blockoa_fno_param_count(const blockoa_fno_shape *shape, int64_t *count) {
  if (!shape_ok(shape) || !count) return BLOCKOA_ERR_INVALID;
  *count = count_params(*shape);
  return BLOCKOA_OK;
}

extern "C" int blockoa_fno_create(const blockoa_fno_shape *shape, const float *params, blockoa_fno **out) {
  if (!out) return BLOCKOA_ERR_INVALID;
  *out = nullptr;
  if (!shape_ok(shape) || !params) return BLOCKOA_ERR_INVALID;
  blockoa_fno *net = new blockoa_fno();
  net->sh = *shape;
  const blockoa_fno_shape &s = net->sh;
  cudaGetDevice(&net->device);
  const long long W = FNO_W, L = s.layers, M = (long long)s.mx * s.my * s.mz, H = s.hidden;
  net->n_params = count_params(s);
  long long o = 0;
  net->oP = o; o += W * s.c_in;
  net->obP = o; o += W;
  net->oW = o; o += L * W * W;
  net->ob = o; o += L * W;
  net->oRr = o; o += L * M * W * W;
  net->oRi = o; o += L * M * W * W;
  net->oQ1 = o; o += H * W;
  net->oc1 = o; o += H;
  net->oQ2 = o; o += H;
  net->oc2 = o; o += 1;
  const long long B = s.max_batch, N = (long long)s.nx * s.ny * s.nz;
  const size_t np = (size_t)net->n_params;
  auto fail = [&](cudaError_t e) {
    const int rc = cuda_status(e, "blockoa_fno_create");
    blockoa_fno_destroy(net);
    return rc;
  };
  cudaError_t e = cudaSuccess;
#define FNO_ALLOC(ptr, bytes) \
  if ((e = fno_alloc(net, &(ptr), (bytes))) != cudaSuccess) return fail(e)
  FNO_ALLOC(net->params, np * 4);
  FNO_ALLOC(net->grads, np * 4);
  FNO_ALLOC(net->m1, np * 4);
  FNO_ALLOC(net->m2, np * 4);
  FNO_ALLOC(net->wb, np * 2);
  FNO_ALLOC(net->tw_x, (size_t)s.mx * s.nx * sizeof(float2));
  FNO_ALLOC(net->tw_y, (size_t)s.my * s.ny * sizeof(float2));
  FNO_ALLOC(net->tw_z, (size_t)s.mz * s.nz * sizeof(float2));
  FNO_ALLOC(net->wz, (size_t)3 * s.mz * sizeof(float));
  FNO_ALLOC(net->v, (size_t)(L + 1) * B * N * W * 4);
  FNO_ALLOC(net->u, (size_t)L * B * N * W * 4);
  FNO_ALLOC(net->a1, (size_t)B * N * H * 4);
  FNO_ALLOC(net->h, (size_t)B * N * H * 4);
  FNO_ALLOC(net->kbuf, (size_t)B * N * W * 4);
  FNO_ALLOC(net->d1, (size_t)B * N * H * 4);
  FNO_ALLOC(net->d2, (size_t)B * N * H * 4);
  FNO_ALLOC(net->xh, (size_t)L * B * M * W * sizeof(float2));
  FNO_ALLOC(net->yh, (size_t)B * M * W * sizeof(float2));
  FNO_ALLOC(net->dxh, (size_t)B * M * W * sizeof(float2));
  FNO_ALLOC(net->s1, (size_t)B * s.nz * s.ny * s.mx * W * sizeof(float2));
  FNO_ALLOC(net->s2, (size_t)B * s.nz * (s.ny > s.my ? s.ny : s.my) * s.mx * W * sizeof(float2));
#undef FNO_ALLOC
  std::vector<float2> t;
  twiddles(t, s.mx, s.nx, true);
  if ((e = cudaMemcpy(net->tw_x, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  twiddles(t, s.my, s.ny, true);
  if ((e = cudaMemcpy(net->tw_y, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  twiddles(t, s.mz, s.nz, false);
  if ((e = cudaMemcpy(net->tw_z, t.data(), t.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  std::vector<float> wz(3 * (size_t)s.mz);
  for (int c = 0; c < s.mz; ++c) {
    wz[c] = c == 0 ? 1.f : 2.f;
    wz[s.mz + c] = 1.f;
    wz[2 * s.mz + c] = (float)((c == 0 ? 1.0 : 2.0) / ((double)s.nx * s.ny * s.nz));
  }
  if ((e = cudaMemcpy(net->wz, wz.data(), wz.size() * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(net->params, params, np * 4, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(net->grads, 0, np * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(net->m1, 0, np * 4)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(net->m2, 0, np * 4)) != cudaSuccess) return fail(e);
  to_bf16_kernel<<<grid_for((long long)np), 256>>>(net->params, net->wb, (long long)np);
  g_launches += 1;
  const size_t smx = (size_t)s.nx * FNO_W * sizeof(float) + (size_t)s.mx * s.nx * sizeof(float2);
  if (smx > 48 * 1024)
    cudaFuncSetAttribute(dft_x_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx);
  const size_t smi = (size_t)s.mx * (FNO_W + s.nx) * sizeof(float2);
  if (smi > 48 * 1024)
    cudaFuncSetAttribute(dft_x_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi);
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return fail(e);
  *out = net;
  return BLOCKOA_OK;
}

extern "C" int blockoa_fno_forward(blockoa_fno *net, const float *x, float *y, int batch, int keep,
                                   blockoa_stream stream) {
  if (!net || !x || !y || batch < 1 || batch > net->sh.max_batch) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const blockoa_fno_shape &s = net->sh;
  const long long N = (long long)s.nx * s.ny * s.nz, rows = (long long)batch * N, W = FNO_W;
  const long long vstride = (long long)s.max_batch * N * W;
  float *v0 = net->v;
  switch (s.c_in) {
#define CASE_CIN(C) \
  case C: pw<C, 32>(net, x, rows, FNO_W, net->oP, 0, net->params + net->obP, nullptr, nullptr, v0, 0, 0, st); break;
    CASE_CIN(1) CASE_CIN(2) CASE_CIN(3) CASE_CIN(4) CASE_CIN(5) CASE_CIN(6) CASE_CIN(7) CASE_CIN(8)
#undef CASE_CIN
    default: return BLOCKOA_ERR_INVALID;
  }
  for (int l = 0; l < s.layers; ++l) {
    const float *vin = net->v + l * vstride;
    float *vout = net->v + (l + 1) * vstride;
    spectral_forward(net, l, vin, net->kbuf, batch, st);
    pw<32, 32>(net, vin, rows, FNO_W, net->oW + (long long)l * W * W, 0, net->params + net->ob + (long long)l * W,
               net->kbuf, net->u + l * vstride, vout, l < s.layers - 1 ? 1 : 0, 0, st);
  }
  const float *vL = net->v + s.layers * vstride;
  pw<32, 32>(net, vL, rows, s.hidden, net->oQ1, 0, net->params + net->oc1, nullptr, net->a1, net->h, 1, 0, st);
  switch (s.hidden) {
#define CASE_H(Hh) \
  case Hh: pw<Hh, 1>(net, net->h, rows, 1, net->oQ2, 0, net->params + net->oc2, nullptr, nullptr, y, 0, 0, st); break;
    CASE_H(32) CASE_H(64) CASE_H(96) CASE_H(128) CASE_H(160) CASE_H(192) CASE_H(224) CASE_H(256)
#undef CASE_H
    default: return BLOCKOA_ERR_INVALID;
  }
  if (keep) {
    net->x_keep = x;
    net->kept_batch = batch;
  }
  return cuda_status(cudaGetLastError(), "blockoa_fno_forward");
}

extern "C" int blockoa_fno_mse(const blockoa_fno *net, const float *y, const float *target, int batch, float *dy,
                               float *loss, blockoa_stream stream) {
  if (!net || !y || !target || !dy || !loss || batch < 1 || batch > net->sh.max_batch) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = (long long)batch * net->sh.nx * net->sh.ny * net->sh.nz;
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return cuda_status(e, "blockoa_fno_mse");
  const long long g = (n + 255) / 256;
  mse_kernel<<<(unsigned)(g < 1024 ? g : 1024), 256, 0, st>>>(y, target, n, dy, loss);
  g_launches += 1;
  return cuda_status(cudaGetLastError(), "blockoa_fno_mse");
}

extern "C" int blockoa_fno_backward(blockoa_fno *net, const float *dy, int batch, blockoa_stream stream) {
  if (!net || !dy || batch < 1 || batch != net->kept_batch || !net->x_keep) return BLOCKOA_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  const blockoa_fno_shape &s = net->sh;
  const long long N = (long long)s.nx * s.ny * s.nz, rows = (long long)batch * N, W = FNO_W;
  const long long vstride = (long long)s.max_batch * N * W;
  const int nm = s.mx * s.my * s.mz, np = s.mx * s.my;
  // projection: dQ2, dc2; dh = Q2^T dy; da1 = dh gelu'(a1); dQ1, dc1; dv = Q1^T da1
  switch (s.hidden) {
#define CASE_H(Hh)                                                                                  \
  case Hh:                                                                                          \
    pw_grad<Hh, 1>(net, net->h, dy, rows, net->oQ2, net->oc2, st);                                 \
    pw<1, 32>(net, dy, rows, Hh, net->oQ2, 1, nullptr, nullptr, nullptr, net->d1, 0, 0, st);       \
    gelu_bwd_kernel<<<grid_for(rows * Hh), 256, 0, st>>>(net->d1, net->a1, rows * Hh);              \
    pw_grad<32, Hh>(net, net->v + s.layers * vstride, net->d1, rows, net->oQ1, net->oc1, st);      \
    pw<Hh, 32>(net, net->d1, rows, FNO_W, net->oQ1, 1, nullptr, nullptr, nullptr, net->d2, 0, 0, st); \
    break;
    CASE_H(32) CASE_H(64) CASE_H(96) CASE_H(128) CASE_H(160) CASE_H(192) CASE_H(224) CASE_H(256)
#undef CASE_H
    default: return BLOCKOA_ERR_INVALID;
  }
  g_launches += 1;
  const size_t smx = (size_t)s.nx * FNO_W * sizeof(float) + (size_t)s.mx * s.nx * sizeof(float2);
  const size_t smi = (size_t)s.mx * (FNO_W + s.nx) * sizeof(float2);
  float *dv = net->d2, *dn = net->d1;
  for (int l = s.layers - 1; l >= 0; --l) {
    if (l < s.layers - 1) {
      gelu_bwd_kernel<<<grid_for(rows * W), 256, 0, st>>>(dv, net->u + l * vstride, rows * W);   // du
      g_launches += 1;
    }
    const float *vin = net->v + l * vstride;
    pw_grad<32, 32>(net, vin, dv, rows, net->oW + (long long)l * W * W, net->ob + (long long)l * W, st);
    // dYh = (w_c / N) * forward transform of du
    dft_x_fwd_kernel<<<(unsigned)((long long)batch * s.nz * s.ny), 256, smx, st>>>(dv, net->s1, net->tw_x, s.nx, s.mx);
    dft_y_kernel<true><<<grid_for((long long)batch * s.nz * s.my * s.mx * W), 256, 0, st>>>(
        net->s1, net->s2, net->tw_y, (long long)batch * s.nz, s.ny, s.my, s.mx);
    dft_z_kernel<true><<<grid_for((long long)batch * s.mz * np * W), 256, 0, st>>>(
        net->s2, net->yh, net->tw_z, net->wz + 2 * s.mz, batch, s.nz, s.mz, np);
    const long long R0 = net->oRr + (long long)l * nm * W * W, I0 = net->oRi + (long long)l * nm * W * W;
    mix_bwd_kernel<<<nm, 256, 0, st>>>(net->xh + (long long)l * s.max_batch * nm * W, net->yh, net->dxh,
                                       net->wb + R0, net->wb + I0, net->grads + R0, net->grads + I0, batch, nm);
    // dv_in = W_l^T du + unweighted inverse transform of dXh
    pw<32, 32>(net, dv, rows, FNO_W, net->oW + (long long)l * W * W, 1, nullptr, nullptr, nullptr, dn, 0, 0, st);
    dft_z_kernel<false><<<grid_for((long long)batch * s.nz * np * W), 256, 0, st>>>(
        net->dxh, net->s2, net->tw_z, net->wz + s.mz, batch, s.nz, s.mz, np);
    dft_y_kernel<false><<<grid_for((long long)batch * s.nz * s.ny * s.mx * W), 256, 0, st>>>(
        net->s2, net->s1, net->tw_y, (long long)batch * s.nz, s.ny, s.my, s.mx);
    dft_x_inv_kernel<<<(unsigned)((long long)batch * s.nz * s.ny), 256, smi, st>>>(net->s1, dn, net->tw_x, s.nx,
                                                                                  s.mx, 1.f, 1);
    g_launches += 7;
    float *tmp = dv;
    dv = dn;
    dn = tmp;
  }
  switch (s.c_in) {
#define CASE_CIN(C) \
  case C: pw_grad<C, 32>(net, net->x_keep, dv, rows, net->oP, net->obP, st); break;
    CASE_CIN(1) CASE_CIN(2) CASE_CIN(3) CASE_CIN(4) CASE_CIN(5) CASE_CIN(6) CASE_CIN(7) CASE_CIN(8)
#undef CASE_CIN
    default: return BLOCKOA_ERR_INVALID;
  }
  return cuda_status(cudaGetLastError(), "blockoa_fno_backward");
}

extern "C" int blockoa_fno_zero_grad(blockoa_fno *net, blockoa_stream stream) {
  if (!net) return BLOCKOA_ERR_INVALID;
  return cuda_status(cudaMemsetAsync(net->grads, 0, (size_t)net->n_params * 4, (cudaStream_t)stream),
                     "blockoa_fno_zero_grad");
}

extern "C" int blockoa_fno_adam_step(blockoa_fno *net, float lr, float beta1, float beta2, float eps, int t,
                                     blockoa_stream stream) {
  if (!net || t < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f))
    return BLOCKOA_ERR_INVALID;
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  adam_kernel<<<grid_for(net->n_params), 256, 0, (cudaStream_t)stream>>>(net->params, net->grads, net->m1, net->m2,
                                                                          net->wb, net->n_params, lr, beta1, beta2,
                                                                          eps, c1, c2);
  g_launches += 1;
  return cuda_status(cudaGetLastError(), "blockoa_fno_adam_step");
}

extern "C" int blockoa_fno_get_params(const blockoa_fno *net, float *params) {
  if (!net || !params) return BLOCKOA_ERR_INVALID;
  return cuda_status(cudaMemcpy(params, net->params, (size_t)net->n_params * 4, cudaMemcpyDeviceToHost),
                     "blockoa_fno_get_params");
}

extern "C" int blockoa_fno_get_grads(const blockoa_fno *net, float *grads) {
  if (!net || !grads) return BLOCKOA_ERR_INVALID;
  return cuda_status(cudaMemcpy(grads, net->grads, (size_t)net->n_params * 4, cudaMemcpyDeviceToHost),
                     "blockoa_fno_get_grads");
}

extern "C" void blockoa_fno_destroy(blockoa_fno *net) {
  if (!net) return;
  cudaDeviceSynchronize();
  for (void *p : net->allocs) cudaFree(p);
  cudaGetLastError();
  delete net;
}
