// Learned subgrid correction: a 3-layer periodic 3x3 convolutional network (12 -> 32 -> 32 -> 4
// channels, tanh after the first two layers) that predicts the residual between the exact
// filtered subgrid terms and the analytic Delta^2/12 closure of Sec. 2.1 / Sec. 3.  This file
// holds its training kernels (binary32 forward, back-propagation, Adam), its inference kernel
// (bf16 operands on the tensor cores through mma.sync m16n8k16, binary32 accumulation), and the
// kernels that build features and training targets from filtered fine-grid fields.
//
// Conventions (shared with the C ABI): activations are [batch][channel][H][W] binary32 planes on
// a periodic H x W grid; parameters are one flat binary32 vector holding, per layer,
// W[co][ci][dy+1][dx+1] then b[co], with y[co](x) = b[co] + sum W[co][ci][dy+1][dx+1] a[ci](x+(dx,dy)).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbmhd.h"
#include "lbmhd_handle.h"
#include "lbmhd_internal.cuh"

namespace lbmhd_gpu {
namespace {

constexpr int kC0 = 12, kC1 = 32, kC2 = 32, kC3 = 4;
constexpr int kP1 = kC1 * kC0 * 9 + kC1;          // 3488
constexpr int kP2 = kC2 * kC1 * 9 + kC2;          // 9248
constexpr int kP3 = kC3 * kC2 * 9 + kC3;          // 1156
constexpr int kNumParams = kP1 + kP2 + kP3;       // 13892
constexpr int kThreads = 256;
constexpr int kWeightCellsPerBlock = 1024;        // cells per block in the weight-gradient pass

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// ---- binary32 forward: one thread per cell, all CO outputs ----------------------------------
template <int CI, int CO, bool TANH>
__global__ void conv_fwd_kernel(const float* __restrict__ in, const float* __restrict__ params,
                                int batch, int H, int W, float* __restrict__ out) {
  __shared__ float sw[CO * CI * 9 + CO];
  for (int i = threadIdx.x; i < CO * CI * 9 + CO; i += blockDim.x) sw[i] = params[i];
  __syncthreads();
  const long plane = (long)H * W;
  const long total = (long)batch * plane;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < total; c += (long)gridDim.x * blockDim.x) {
    const int b = (int)(c / plane);
    const int cell = (int)(c % plane);
    const int y = cell / W, x = cell % W;
    int off[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) off[t] = wrapi(y + t / 3 - 1, H) * W + wrapi(x + t % 3 - 1, W);
    float acc[CO];
#pragma unroll
    for (int co = 0; co < CO; ++co) acc[co] = sw[CO * CI * 9 + co];
    const float* ib = in + (size_t)b * CI * plane;
    for (int ci = 0; ci < CI; ++ci) {
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const float v = ib[(size_t)ci * plane + off[t]];
#pragma unroll
        for (int co = 0; co < CO; ++co) acc[co] = fmaf(sw[(co * CI + ci) * 9 + t], v, acc[co]);
      }
    }
    float* ob = out + (size_t)b * CO * plane;
#pragma unroll
    for (int co = 0; co < CO; ++co) ob[(size_t)co * plane + cell] = TANH ? tanhf(acc[co]) : acc[co];
  }
}

// ---- back-propagation -------------------------------------------------------------------------
// da[ci](z) = sum_co sum_d W[co][ci][d] dy[co](z - d); then times (1 - a^2) if the input came
// from a tanh (a = that activation).
template <int CI, int CO, bool TANH_IN>
__global__ void conv_bwd_data_kernel(const float* __restrict__ dy, const float* __restrict__ params,
                                     const float* __restrict__ a_in, int batch, int H, int W,
                                     float* __restrict__ da) {
  __shared__ float sw[CO * CI * 9];
  for (int i = threadIdx.x; i < CO * CI * 9; i += blockDim.x) sw[i] = params[i];
  __syncthreads();
  const long plane = (long)H * W;
  const long total = (long)batch * plane;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < total; c += (long)gridDim.x * blockDim.x) {
    const int b = (int)(c / plane);
    const int cell = (int)(c % plane);
    const int y = cell / W, x = cell % W;
    int off[9];  // z - d for tap d
#pragma unroll
    for (int t = 0; t < 9; ++t) off[t] = wrapi(y - (t / 3 - 1), H) * W + wrapi(x - (t % 3 - 1), W);
    float acc[CI];
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) acc[ci] = 0.f;
    const float* db = dy + (size_t)b * CO * plane;
    for (int co = 0; co < CO; ++co) {
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const float g = db[(size_t)co * plane + off[t]];
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) acc[ci] = fmaf(sw[(co * CI + ci) * 9 + t], g, acc[ci]);
      }
    }
    const float* ab = a_in + (size_t)b * CI * plane;
    float* ob = da + (size_t)b * CI * plane;
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) {
      float v = acc[ci];
      if (TANH_IN) {
        const float a = ab[(size_t)ci * plane + cell];
        v *= (1.f - a * a);
      }
      ob[(size_t)ci * plane + cell] = v;
    }
  }
}

// Per-block partial weight gradients over kWeightCellsPerBlock cells:
// dW[co][ci][d] = sum_z dy[co](z) a[ci](z + d),  db[co] = sum_z dy[co](z).
template <int CI, int CO>
__global__ void conv_bwd_weight_kernel(const float* __restrict__ dy, const float* __restrict__ a,
                                       int batch, int H, int W, float* __restrict__ partials) {
  constexpr int NW = CO * CI * 9 + CO;
  const long plane = (long)H * W;
  const long total = (long)batch * plane;
  const long c0 = (long)blockIdx.x * kWeightCellsPerBlock;
  const long c1 = c0 + kWeightCellsPerBlock < total ? c0 + kWeightCellsPerBlock : total;
  for (int w = threadIdx.x; w < NW; w += blockDim.x) {
    float acc = 0.f;
    if (w < CO * CI * 9) {
      const int co = w / (CI * 9), ci = (w / 9) % CI, t = w % 9;
      const int ddy = t / 3 - 1, ddx = t % 3 - 1;
      for (long c = c0; c < c1; ++c) {
        const int b = (int)(c / plane);
        const int cell = (int)(c % plane);
        const int y = cell / W, x = cell % W;
        const float g = dy[(size_t)b * CO * plane + (size_t)co * plane + cell];
        const float v = a[(size_t)b * CI * plane + (size_t)ci * plane + wrapi(y + ddy, H) * W + wrapi(x + ddx, W)];
        acc = fmaf(g, v, acc);
      }
    } else {
      const int co = w - CO * CI * 9;
      for (long c = c0; c < c1; ++c) {
        const int b = (int)(c / plane);
        const int cell = (int)(c % plane);
        acc += dy[(size_t)b * CO * plane + (size_t)co * plane + cell];
      }
    }
    partials[(size_t)blockIdx.x * NW + w] = acc;
  }
}

// Sum the block partials in block order (deterministic).
__global__ void sum_partials_kernel(const float* __restrict__ partials, int nblocks, int nw,
                                    float* __restrict__ out) {
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nw; w += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * nw + w];
    out[w] = s;
  }
}

// dout = (out - target) / n and per-block partial sums of (out - target)^2.
__global__ void loss_grad_kernel(const float* __restrict__ out, const float* __restrict__ target, long n,
                                 float* __restrict__ dout, double* __restrict__ partial) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  const float inv = 1.f / (float)n;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float d = out[i] - target[i];
    dout[i] = d * inv;
    acc += (double)d * d;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                            float c1, float c2) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

// ---- bf16 tensor-core inference ----------------------------------------------------------------
// Layer as an implicit GEMM: Y[cell][co] = b[co] + sum_k X[cell][k] W[co][k], k = ci*9 + tap,
// K padded to a multiple of 16 with zeros.  A block stages a 3-row bf16 patch of its 64-cell
// row tile in shared memory; each warp computes 16 consecutive cells (M = 16) for all CO
// (N tiles of 8) with mma.sync.m16n8k16 (bf16 x bf16 -> f32), reading A from the patch.
// Fragment layouts of m16n8k16 (PTX ISA): with g = lane/4, q = lane%4,
//   A regs (2 bf16 each): (g, 2q..), (g+8, 2q..), (g, 2q+8..), (g+8, 2q+8..)
//   B regs: (k = 2q.., n = g), (k = 2q+8.., n = g)
//   C/D:    (g, 2q), (g, 2q+1), (g+8, 2q), (g+8, 2q+1)
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kMmaTile = 64;  // cells of one row per block (4 warps x 16)

template <int CI, int CO, bool TANH>
__global__ void __launch_bounds__(128) conv_fwd_mma_kernel(const float* __restrict__ in,
                                                           const float* __restrict__ params, int batch,
                                                           int H, int W, float* __restrict__ out) {
  constexpr int K = CI * 9;
  constexpr int KP = (K + 15) / 16 * 16;
  constexpr int NT = (CO + 7) / 8;        // n tiles of 8
  constexpr int NP = NT * 8;
  constexpr int PW = kMmaTile + 2;        // staged columns: the tile plus one on each side
  // weights as bf16 [NP][KP] (co major, zero padded), fp32 bias, the bf16 input patch
  // [CI][3 rows][PW] of the tile, and for every k = ci*9 + tap its offset in the patch
  __shared__ __nv_bfloat16 sw[NP * KP];
  __shared__ float sb[NP];
  __shared__ __nv_bfloat16 patch[CI * 3 * PW];
  __shared__ int koff[KP];
  for (int i = threadIdx.x; i < NP * KP; i += blockDim.x) {
    const int co = i / KP, k = i % KP;
    sw[i] = __float2bfloat16_rn(co < CO && k < K ? params[co * K + k] : 0.f);
  }
  for (int i = threadIdx.x; i < NP; i += blockDim.x) sb[i] = i < CO ? params[CO * K + i] : 0.f;
  for (int k = threadIdx.x; k < KP; k += blockDim.x) {
    const int ci = k / 9, t = k % 9;
    koff[k] = k < K ? ci * 3 * PW + (t / 3) * PW + (t % 3) : -1;
  }
  const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int wm = (threadIdx.x >> 5) * 16;  // this warp's first cell in the tile
  const long plane = (long)H * W;
  const int segs = (W + kMmaTile - 1) / kMmaTile;
  const long tiles = (long)batch * H * segs;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int b = (int)(tile / ((long)H * segs));
    const int rem = (int)(tile % ((long)H * segs));
    const int y = rem / segs, x0 = (rem % segs) * kMmaTile;
    const float* ib = in + (size_t)b * CI * plane;
    __syncthreads();  // the previous tile's patch is no longer read (and the tables are ready)
    for (int i = threadIdx.x; i < CI * 3 * PW; i += blockDim.x) {
      const int ci = i / (3 * PW), r = (i / PW) % 3, cc = i % PW;
      const int xx = x0 + cc - 1;
      patch[i] = (xx <= W) ? __float2bfloat16_rn(ib[(size_t)ci * plane + wrapi(y + r - 1, H) * W + wrapi(xx, W)])
                           : zero;
    }
    __syncthreads();
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      acc[n][0] = sb[n * 8 + 2 * q];
      acc[n][1] = sb[n * 8 + 2 * q + 1];
      acc[n][2] = acc[n][0];
      acc[n][3] = acc[n][1];
    }
    const int m0 = wm + g, m1 = wm + g + 8;
    auto av = [&](int ko, int m) -> __nv_bfloat16 { return ko >= 0 ? patch[ko + m] : zero; };
    auto pk = [](__nv_bfloat16 lo, __nv_bfloat16 hi) -> uint32_t {
      __nv_bfloat162 v = __halves2bfloat162(lo, hi);
      return *reinterpret_cast<uint32_t*>(&v);
    };
#pragma unroll 2
    for (int k0 = 0; k0 < KP; k0 += 16) {
      const int o0 = koff[k0 + 2 * q], o1 = koff[k0 + 2 * q + 1];
      const int o8 = koff[k0 + 2 * q + 8], o9 = koff[k0 + 2 * q + 9];
      uint32_t a[4];
      a[0] = pk(av(o0, m0), av(o1, m0));
      a[1] = pk(av(o0, m1), av(o1, m1));
      a[2] = pk(av(o8, m0), av(o9, m0));
      a[3] = pk(av(o8, m1), av(o9, m1));
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        const __nv_bfloat16* wb = sw + (n * 8 + g) * KP + k0;
        uint32_t bfr[2];
        bfr[0] = *reinterpret_cast<const uint32_t*>(wb + 2 * q);
        bfr[1] = *reinterpret_cast<const uint32_t*>(wb + 2 * q + 8);
        mma_bf16_16816(acc[n], a, bfr);
      }
    }
    float* ob = out + (size_t)b * CO * plane;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = wm + g + (r >= 2 ? 8 : 0);
        const int co = n * 8 + 2 * q + (r & 1);
        const int xx = x0 + m;
        if (co < CO && xx < W) {
          const float v = acc[n][r];
          ob[(size_t)co * plane + (size_t)y * W + xx] = TANH ? tanhf(v) : v;
        }
      }
    }
  }
}

int mma_grid(int batch, int H, int W) {
  long tiles = (long)batch * H * ((W + kMmaTile - 1) / kMmaTile);
  if (tiles > 152L * 8) tiles = 152L * 8;
  return tiles < 1 ? 1 : (int)tiles;
}

// ---- features and training targets ----------------------------------------------------------
// Coarse moments of a fine state by r x r box filter, including the filtered nonlinear products:
// out planes [0..4] = rho, Jx, Jy, Bx, By; [5] JxJy/rho - BxBy; [6] (Jx^2-Jy^2)/rho - (Bx^2-By^2);
// [7] (Jx^2+Jy^2)/rho; [8] (Jx By - Jy Bx)/rho.
__global__ void filter_products_kernel(const double* __restrict__ fine, int n, int r,
                                       double* __restrict__ coarse) {
  const int m = n / r;
  const long mm = (long)m * m, nn = (long)n * n;
  const double inv = 1.0 / ((double)r * r);
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < mm; c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % m), j = (int)(c / m);
    double s[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int yy = 0; yy < r; ++yy)
      for (int xx = 0; xx < r; ++xx) {
        const size_t f = (size_t)(j * r + yy) * n + (size_t)(i * r + xx);
        const double rho = fine[f], ux = fine[nn + f], uy = fine[2 * nn + f], bx = fine[3 * nn + f],
                     by = fine[4 * nn + f];
        const double jx = rho * ux, jy = rho * uy;
        s[0] += rho;
        s[1] += jx;
        s[2] += jy;
        s[3] += bx;
        s[4] += by;
        s[5] += jx * jy / rho - bx * by;
        s[6] += (jx * jx - jy * jy) / rho - (bx * bx - by * by);
        s[7] += (jx * jx + jy * jy) / rho;
        s[8] += (jx * by - jy * bx) / rho;
      }
    for (int k = 0; k < 9; ++k) coarse[(size_t)k * mm + c] = s[k] * inv;
  }
}

__device__ __forceinline__ double cdiff(const double* a, int m, int x, int y, int axis) {
  return axis == 0 ? 0.5 * (a[(size_t)y * m + wrapi(x + 1, m)] - a[(size_t)y * m + wrapi(x - 1, m)])
                   : 0.5 * (a[(size_t)wrapi(y + 1, m) * m + x] - a[(size_t)wrapi(y - 1, m) * m + x]);
}

// Features (12 channels: u, B and their central differences, each over its scale) of a coarse
// state given as rho, Jx, Jy, Bx, By planes (J = rho u); optionally the analytic closure a0..a3
// (k = delta^2/12) into `analytic` (4 planes), and, when `products` is given (planes 5..8 of
// filter_products_kernel), the training target (c - a)/out_scale into `target`.
__global__ void features_kernel(const double* __restrict__ st, int m, int velocity,
                                const float* __restrict__ in_scale, const float* __restrict__ out_scale,
                                double kd, float* __restrict__ x, float* __restrict__ analytic,
                                const double* __restrict__ products, float* __restrict__ target) {
  const long mm = (long)m * m;
  const double* rho = st;
  const double* p1 = st + mm;  // J_x, or u_x when `velocity`
  const double* p2 = st + 2 * mm;
  const double* bx = st + 3 * mm;
  const double* by = st + 4 * mm;
  auto jval = [&](int f, size_t o) -> double {  // J_x (f = 0) or J_y (f = 1) at cell o
    const double v = f == 0 ? p1[o] : p2[o];
    return velocity ? rho[o] * v : v;
  };
  auto uval = [&](int f, size_t o) -> double {  // u_x, u_y, B_x, B_y at cell o
    if (f >= 2) return f == 2 ? bx[o] : by[o];
    const double v = f == 0 ? p1[o] : p2[o];
    return velocity ? v : v / rho[o];
  };
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < mm; c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % m), j = (int)(c / m);
    const size_t xe = (size_t)j * m + wrapi(i + 1, m), xw = (size_t)j * m + wrapi(i - 1, m);
    const size_t yn = (size_t)wrapi(j + 1, m) * m + i, ys = (size_t)wrapi(j - 1, m) * m + i;
    // gradients of u and B for the features; of J and B for the closure
    double u[4], du[8], gj[4], gb[4];
    const double r0 = rho[c];
    for (int f = 0; f < 4; ++f) {
      u[f] = uval(f, c);
      du[2 * f] = 0.5 * (uval(f, xe) - uval(f, xw));
      du[2 * f + 1] = 0.5 * (uval(f, yn) - uval(f, ys));
    }
    gj[0] = 0.5 * (jval(0, xe) - jval(0, xw));
    gj[1] = 0.5 * (jval(0, yn) - jval(0, ys));
    gj[2] = 0.5 * (jval(1, xe) - jval(1, xw));
    gj[3] = 0.5 * (jval(1, yn) - jval(1, ys));
    gb[0] = cdiff(bx, m, i, j, 0);
    gb[1] = cdiff(bx, m, i, j, 1);
    gb[2] = cdiff(by, m, i, j, 0);
    gb[3] = cdiff(by, m, i, j, 1);
    for (int f = 0; f < 4; ++f) x[(size_t)f * mm + c] = (float)(u[f] / in_scale[f]);
    for (int f = 0; f < 8; ++f) x[(size_t)(4 + f) * mm + c] = (float)(du[f] / in_scale[4 + f]);
    if (analytic || target) {
      const double Gxx = gj[0] * gj[0] + gj[1] * gj[1], Gyy = gj[2] * gj[2] + gj[3] * gj[3];
      const double Gxy = gj[0] * gj[2] + gj[1] * gj[3];
      const double Hxx = gb[0] * gb[0] + gb[1] * gb[1], Hyy = gb[2] * gb[2] + gb[3] * gb[3];
      const double Hxy = gb[0] * gb[2] + gb[1] * gb[3];
      const double Kxy = gj[0] * gb[2] + gj[1] * gb[3], Kyx = gj[2] * gb[0] + gj[3] * gb[1];
      const double a[4] = {kd * (Gxy / r0 - Hxy), kd * ((Gxx - Gyy) / r0 - Hxx + Hyy),
                           kd * (Gxx + Gyy) / r0, kd * (Kxy - Kyx) / r0};
      if (analytic)
        for (int f = 0; f < 4; ++f) analytic[(size_t)f * mm + c] = (float)a[f];
      if (target && products) {
        const double jxc = jval(0, c), jyc = jval(1, c), bxc = bx[c], byc = by[c];
        const double cq[4] = {products[c] - (jxc * jyc / r0 - bxc * byc),
                              products[mm + c] - ((jxc * jxc - jyc * jyc) / r0 - (bxc * bxc - byc * byc)),
                              products[2 * mm + c] - (jxc * jxc + jyc * jyc) / r0,
                              products[3 * mm + c] - (jxc * byc - jyc * bxc) / r0};
        for (int f = 0; f < 4; ++f) target[(size_t)f * mm + c] = (float)((cq[f] - a[f]) / out_scale[f]);
      }
    }
  }
}

// correction (4 planes, physical units) = network output x out_scale; in place
__global__ void scale_output_kernel(float* __restrict__ out, long mm, const float* __restrict__ out_scale) {
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < 4 * mm; c += (long)gridDim.x * blockDim.x)
    out[c] *= out_scale[c / mm];
}

int grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  if (b > 152L * 16) b = 152L * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

int closure_num_params() { return kNumParams; }

// Inference on a coarse state: moments (rho, Jx, Jy, Bx, By planes, binary64) -> correction
// planes [4][m][m] in physical units, via features and the bf16 tensor-core network.
cudaError_t closure_correction(const float* params, const float* in_scale, const float* out_scale,
                               const double* state, int m, float* feat, float* a1, float* a2,
                               float* corr, cudaStream_t s) {
  const long mm = (long)m * m;
  features_kernel<<<grid_for(mm), kThreads, 0, s>>>(state, m, 1, in_scale, out_scale, 0.0, feat, nullptr,
                                                     nullptr, nullptr);
  const int blocks = mma_grid(1, m, m);
  conv_fwd_mma_kernel<kC0, kC1, true><<<blocks, 128, 0, s>>>(feat, params, 1, m, m, a1);
  conv_fwd_mma_kernel<kC1, kC2, true><<<blocks, 128, 0, s>>>(a1, params + kP1, 1, m, m, a2);
  conv_fwd_mma_kernel<kC2, kC3, false><<<blocks, 128, 0, s>>>(a2, params + kP1 + kP2, 1, m, m, corr);
  scale_output_kernel<<<grid_for(4 * mm), kThreads, 0, s>>>(corr, mm, out_scale);
  return cudaGetLastError();
}

}  // namespace lbmhd_gpu

// ---- the closure object and its C ABI -------------------------------------------------------
using namespace lbmhd_gpu;

struct lbmhd_closure {
  float* params = nullptr;  // device, binary32 master copy
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  float* scales = nullptr;  // device: in_scale[12], out_scale[4]
  float host_scales[16];
  int adam_t = 0;
  // training scratch (grown on demand)
  size_t cap_cells = 0;
  float *a1 = nullptr, *a2 = nullptr, *out = nullptr, *d3 = nullptr, *d2 = nullptr, *d1 = nullptr;
  float* wpart = nullptr;
  size_t wpart_cap = 0;
  double* lpart = nullptr;
  cudaStream_t stream = nullptr;
  std::string err;
};

namespace {
thread_local std::string g_cl_error;

int cfail(lbmhd_closure_t* c, int code, const char* msg) {
  if (c)
    c->err = msg;
  else
    g_cl_error = msg;
  return code;
}

#define CL_CUDA(c, call)                                                                         \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      char b_[256];                                                                              \
      snprintf(b_, sizeof b_, "%s: %s", #call, cudaGetErrorString(e_));                         \
      return cfail(c, e_ == cudaErrorMemoryAllocation ? LBMHD_ERR_OOM : LBMHD_ERR_CUDA, b_);   \
    }                                                                                            \
  } while (0)

int ensure_scratch(lbmhd_closure_t* c, size_t cells) {
  if (cells <= c->cap_cells) return LBMHD_OK;
  float** bufs[6] = {&c->a1, &c->a2, &c->out, &c->d3, &c->d2, &c->d1};
  const int ch[6] = {kC1, kC2, kC3, kC3, kC2, kC1};
  for (int i = 0; i < 6; ++i) {
    if (*bufs[i]) cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
    CL_CUDA(c, cudaMalloc(bufs[i], cells * ch[i] * sizeof(float)));
  }
  const size_t nblk = (cells + kWeightCellsPerBlock - 1) / kWeightCellsPerBlock;
  if (c->wpart) cudaFree(c->wpart);
  c->wpart = nullptr;
  CL_CUDA(c, cudaMalloc(&c->wpart, nblk * (size_t)kP2 * sizeof(float)));
  if (!c->lpart) CL_CUDA(c, cudaMalloc(&c->lpart, 152 * 16 * sizeof(double)));
  c->cap_cells = cells;
  return LBMHD_OK;
}

// forward (binary32) + loss + back-propagation into c->grad; *loss = mean squared error / 2
int forward_backward(lbmhd_closure_t* c, const float* x, const float* t, int batch, int h, int w,
                     double* loss) {
  const size_t cells = (size_t)batch * h * w;
  int rc = ensure_scratch(c, cells);
  if (rc) return rc;
  cudaStream_t s = c->stream;
  const float* p1 = c->params;
  const float* p2 = c->params + kP1;
  const float* p3 = c->params + kP1 + kP2;
  const int g = grid_for((long)cells);
  conv_fwd_kernel<kC0, kC1, true><<<g, kThreads, 0, s>>>(x, p1, batch, h, w, c->a1);
  conv_fwd_kernel<kC1, kC2, true><<<g, kThreads, 0, s>>>(c->a1, p2, batch, h, w, c->a2);
  conv_fwd_kernel<kC2, kC3, false><<<g, kThreads, 0, s>>>(c->a2, p3, batch, h, w, c->out);
  const long nout = (long)cells * kC3;
  const int lg = grid_for(nout) < 152 * 16 ? grid_for(nout) : 152 * 16;
  loss_grad_kernel<<<lg, kThreads, 0, s>>>(c->out, t, nout, c->d3, c->lpart);
  const int nblk = (int)((cells + kWeightCellsPerBlock - 1) / kWeightCellsPerBlock);
  // layer 3
  conv_bwd_weight_kernel<kC2, kC3><<<nblk, kThreads, 0, s>>>(c->d3, c->a2, batch, h, w, c->wpart);
  sum_partials_kernel<<<grid_for(kP3), kThreads, 0, s>>>(c->wpart, nblk, kP3, c->grad + kP1 + kP2);
  conv_bwd_data_kernel<kC2, kC3, true><<<g, kThreads, 0, s>>>(c->d3, p3, c->a2, batch, h, w, c->d2);
  // layer 2
  conv_bwd_weight_kernel<kC1, kC2><<<nblk, kThreads, 0, s>>>(c->d2, c->a1, batch, h, w, c->wpart);
  sum_partials_kernel<<<grid_for(kP2), kThreads, 0, s>>>(c->wpart, nblk, kP2, c->grad + kP1);
  conv_bwd_data_kernel<kC1, kC2, true><<<g, kThreads, 0, s>>>(c->d2, p2, c->a1, batch, h, w, c->d1);
  // layer 1
  conv_bwd_weight_kernel<kC0, kC1><<<nblk, kThreads, 0, s>>>(c->d1, x, batch, h, w, c->wpart);
  sum_partials_kernel<<<grid_for(kP1), kThreads, 0, s>>>(c->wpart, nblk, kP1, c->grad);
  CL_CUDA(c, cudaGetLastError());
  std::vector<double> lp(lg);
  CL_CUDA(c, cudaMemcpyAsync(lp.data(), c->lpart, lg * sizeof(double), cudaMemcpyDeviceToHost, s));
  CL_CUDA(c, cudaStreamSynchronize(s));
  double sum = 0.0;
  for (double v : lp) sum += v;
  if (loss) *loss = 0.5 * sum / (double)nout;
  return LBMHD_OK;
}

void destroy_closure(lbmhd_closure_t* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  float* bufs[] = {c->params, c->grad, c->adam_m, c->adam_v, c->scales, c->a1, c->a2, c->out, c->d3,
                   c->d2, c->d1, c->wpart};
  for (float* b : bufs)
    if (b) cudaFree(b);
  if (c->lpart) cudaFree(c->lpart);
  if (c->stream) cudaStreamDestroy(c->stream);
  delete c;
}
}  // namespace

extern "C" {

int lbmhd_closure_num_params(void) { return kNumParams; }

int lbmhd_closure_create(lbmhd_closure_t** out, const float* params, const float* in_scale,
                         const float* out_scale) {
  if (!out) return cfail(nullptr, LBMHD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!params || !in_scale || !out_scale) return cfail(nullptr, LBMHD_ERR_INVALID, "NULL argument");
  for (int i = 0; i < 12; ++i)
    if (!(in_scale[i] > 0.f)) return cfail(nullptr, LBMHD_ERR_INVALID, "in_scale must be > 0");
  for (int i = 0; i < 4; ++i)
    if (!(out_scale[i] > 0.f)) return cfail(nullptr, LBMHD_ERR_INVALID, "out_scale must be > 0");
  lbmhd_closure_t* c = new (std::nothrow) lbmhd_closure();
  if (!c) return cfail(nullptr, LBMHD_ERR_OOM, "host allocation failed");
  std::memcpy(c->host_scales, in_scale, 12 * sizeof(float));
  std::memcpy(c->host_scales + 12, out_scale, 4 * sizeof(float));
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  const size_t pb = kNumParams * sizeof(float);
  if (e == cudaSuccess) e = cudaMalloc(&c->params, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->grad, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->adam_m, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->adam_v, pb);
  if (e == cudaSuccess) e = cudaMalloc(&c->scales, 16 * sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(c->params, params, pb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->adam_m, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(c->adam_v, 0, pb);
  if (e == cudaSuccess) e = cudaMemcpy(c->scales, c->host_scales, 16 * sizeof(float), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    int rc = cfail(nullptr, e == cudaErrorMemoryAllocation ? LBMHD_ERR_OOM : LBMHD_ERR_CUDA,
                   cudaGetErrorString(e));
    destroy_closure(c);
    return rc;
  }
  *out = c;
  return LBMHD_OK;
}

int lbmhd_closure_get_params(lbmhd_closure_t* c, float* params) {
  if (!c || !params) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  CL_CUDA(c, cudaStreamSynchronize(c->stream));
  CL_CUDA(c, cudaMemcpy(params, c->params, kNumParams * sizeof(float), cudaMemcpyDeviceToHost));
  return LBMHD_OK;
}

int lbmhd_closure_set_params(lbmhd_closure_t* c, const float* params) {
  if (!c || !params) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  CL_CUDA(c, cudaStreamSynchronize(c->stream));
  CL_CUDA(c, cudaMemcpy(c->params, params, kNumParams * sizeof(float), cudaMemcpyHostToDevice));
  c->adam_t = 0;
  CL_CUDA(c, cudaMemset(c->adam_m, 0, kNumParams * sizeof(float)));
  CL_CUDA(c, cudaMemset(c->adam_v, 0, kNumParams * sizeof(float)));
  return LBMHD_OK;
}

int lbmhd_closure_gradient(lbmhd_closure_t* c, const float* x, const float* t, int batch, int h,
                           int w, float* grad, double* loss) {
  if (!c || !x || !t) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  if (batch < 1 || h < 1 || w < 1) return cfail(c, LBMHD_ERR_INVALID, "empty batch");
  int rc = forward_backward(c, x, t, batch, h, w, loss);
  if (rc) return rc;
  if (grad) CL_CUDA(c, cudaMemcpy(grad, c->grad, kNumParams * sizeof(float), cudaMemcpyDeviceToHost));
  return LBMHD_OK;
}

int lbmhd_closure_train_step(lbmhd_closure_t* c, const float* x, const float* t, int batch, int h,
                             int w, float lr, double* loss) {
  if (!c || !x || !t) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  if (batch < 1 || h < 1 || w < 1 || !(lr > 0.f)) return cfail(c, LBMHD_ERR_INVALID, "bad batch or rate");
  int rc = forward_backward(c, x, t, batch, h, w, loss);
  if (rc) return rc;
  c->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)c->adam_t), c2 = 1.f - powf(b2, (float)c->adam_t);
  adam_kernel<<<grid_for(kNumParams), kThreads, 0, c->stream>>>(c->params, c->grad, c->adam_m, c->adam_v,
                                                                kNumParams, lr, b1, b2, 1e-8f, c1, c2);
  CL_CUDA(c, cudaGetLastError());
  return LBMHD_OK;
}

int lbmhd_closure_forward(lbmhd_closure_t* c, const float* x, int batch, int h, int w, float* out,
                          int tensor_cores) {
  if (!c || !x || !out) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  if (batch < 1 || h < 1 || w < 1) return cfail(c, LBMHD_ERR_INVALID, "empty batch");
  const size_t cells = (size_t)batch * h * w;
  int rc = ensure_scratch(c, cells);
  if (rc) return rc;
  const float* p1 = c->params;
  const float* p2 = c->params + kP1;
  const float* p3 = c->params + kP1 + kP2;
  cudaStream_t s = c->stream;
  if (tensor_cores) {
    const int blocks = mma_grid(batch, h, w);
    conv_fwd_mma_kernel<kC0, kC1, true><<<blocks, 128, 0, s>>>(x, p1, batch, h, w, c->a1);
    conv_fwd_mma_kernel<kC1, kC2, true><<<blocks, 128, 0, s>>>(c->a1, p2, batch, h, w, c->a2);
    conv_fwd_mma_kernel<kC2, kC3, false><<<blocks, 128, 0, s>>>(c->a2, p3, batch, h, w, out);
  } else {
    const int g = grid_for((long)cells);
    conv_fwd_kernel<kC0, kC1, true><<<g, kThreads, 0, s>>>(x, p1, batch, h, w, c->a1);
    conv_fwd_kernel<kC1, kC2, true><<<g, kThreads, 0, s>>>(c->a1, p2, batch, h, w, c->a2);
    conv_fwd_kernel<kC2, kC3, false><<<g, kThreads, 0, s>>>(c->a2, p3, batch, h, w, out);
  }
  CL_CUDA(c, cudaGetLastError());
  CL_CUDA(c, cudaStreamSynchronize(s));
  return LBMHD_OK;
}

int lbmhd_closure_training_pair(lbmhd_closure_t* c, const double* fine, int n, int r, double delta,
                                float* x, float* t, double* work) {
  if (!c || !fine || !x || !t || !work) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  if (n < 3 || r < 1 || n % r || n / r < 3 || !(delta >= 0.0))
    return cfail(c, LBMHD_ERR_INVALID, "need r | n, n/r >= 3, delta >= 0");
  const int m = n / r;
  const long mm = (long)m * m;
  cudaStream_t s = c->stream;
  filter_products_kernel<<<grid_for(mm), kThreads, 0, s>>>(fine, n, r, work);
  features_kernel<<<grid_for(mm), kThreads, 0, s>>>(work, m, 0, c->scales, c->scales + 12,
                                                     delta * delta / 12.0, x, nullptr, work + 5 * mm, t);
  CL_CUDA(c, cudaGetLastError());
  CL_CUDA(c, cudaStreamSynchronize(s));
  return LBMHD_OK;
}

int lbmhd_closure_features(lbmhd_closure_t* c, const double* state, int m, double delta, float* x,
                           float* analytic) {
  if (!c || !state || !x) return cfail(c, LBMHD_ERR_INVALID, "NULL argument");
  if (m < 3) return cfail(c, LBMHD_ERR_INVALID, "m must be >= 3");
  features_kernel<<<grid_for((long)m * m), kThreads, 0, c->stream>>>(
      state, m, 1, c->scales, c->scales + 12, delta * delta / 12.0, x, analytic, nullptr, nullptr);
  CL_CUDA(c, cudaGetLastError());
  CL_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBMHD_OK;
}

const char* lbmhd_closure_last_error(const lbmhd_closure_t* c) {
  return c ? c->err.c_str() : g_cl_error.c_str();
}

void lbmhd_closure_free(lbmhd_closure_t* c) { destroy_closure(c); }

}  // extern "C"

namespace lbmhd_gpu {
// Device pointers of a closure's parameters and scales (for handles that attach it).
const float* closure_device_params(const lbmhd_closure_t* c) { return c->params; }
const float* closure_device_scales(const lbmhd_closure_t* c) { return c->scales; }
cudaStream_t closure_stream(const lbmhd_closure_t* c) { return c->stream; }
}  // namespace lbmhd_gpu
