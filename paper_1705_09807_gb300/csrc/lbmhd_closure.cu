// Learned subgrid correction: a 3-layer periodic 3x3 convolutional network (12 -> 32 -> 32 -> 4
// channels, tanh after the first two layers) that predicts the residual between the exact
// filtered subgrid terms and the analytic Delta^2/12 closure of Sec. 2.1 / Sec. 3.  This file
// holds its training kernels (binary32 forward, back-propagation, Adam), its inference kernel
// (all three layers fused in one kernel on the 5th-generation tensor cores: bf16 operands in
// shared memory, tcgen05.mma, fp32 accumulators in tensor memory), and the kernels that build
// features and training targets from filtered fine-grid fields.
//
// Conventions (shared with the C ABI): activations are [batch][channel][H][W] binary32 planes on
// a periodic H x W grid; parameters are one flat binary32 vector holding, per layer,
// W[co][ci][dy+1][dx+1] then b[co], with y[co](x) = b[co] + sum W[co][ci][dy+1][dx+1] a[ci](x+(dx,dy)).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbmhd.h"
#include "lbmhd_handle.h"
#include "lbmhd_internal.cuh"
#include "lbmhd_ptx.cuh"

namespace lbmhd_gpu {
namespace {

constexpr int kC0 = 12, kC1 = 32, kC2 = 32, kC3 = 4;
constexpr int kP1 = kC1 * kC0 * 9 + kC1;          // 3488
constexpr int kP2 = kC2 * kC1 * 9 + kC2;          // 9248
constexpr int kP3 = kC3 * kC2 * 9 + kC3;          // 1156
constexpr int kNumParams = kP1 + kP2 + kP3;       // 13892
constexpr int kThreads = 256;
constexpr int kWeightCellsPerBlock = 1024;        // cells per block in the weight-gradient pass
constexpr uint64_t kNetWaitNs = 2000000000ull;    // bound of every tensor-core completion wait

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

// ---- bf16 tensor-core inference: the whole network in one kernel (tcgen05 + TMEM) --------------
// A CTA computes a kTT x kTT tile of the output from a kPS x kPS patch (3 cells of halo, one per
// layer) held in shared memory as bf16.  Each 3x3 layer is, per 128-cell M tile, nine shifted
// implicit GEMMs per 16-channel K chunk, D[cell][co] += A[cell + dy kPS + dx][k] W_tap[co][k],
// issued by one thread as tcgen05.mma (M = 128, N = 32, or 16 for the 4-channel last layer,
// K = 16) with the fp32 accumulators in tensor memory; the epilogue reads them back with
// tcgen05.ld (one cell per thread), adds the bias, applies tanh and stores the next layer's bf16
// input.  The patch is indexed linearly (cell = row kPS + col), so the shifts wrap across rows:
// the results wrapped that way lie in the halo, which shrinks by one cell per layer, and are
// never used by the kept outputs.
//
// Shared-memory operand layouts (no swizzle, K-major core matrices of 8 rows x 16 bytes):
//   activations: [8-channel chunk][cell] x 16 B; consecutive cells 16 B apart, so an 8-cell group
//     is one core matrix (stride byte offset 128 B), the next 8 channels one chunk further
//     (leading byte offset kChunkBytes), and a shift by s cells is a start address 16 s B later.
//   weights: per (tap, 16-channel K chunk) an N x 16 block with (n, k) at (n%8) 16 + (n/8) 256 +
//     (k/8) 128 + (k%8) 2 bytes (leading byte offset 128, stride byte offset 256).
constexpr int kTT = 16;                       // output tile side
constexpr int kPS = kTT + 6;                  // patch side: 22
constexpr int kPatch = kPS * kPS;             // 484 cells
constexpr int kMT = 4;                        // M tiles of every layer: cells 0 .. 511
constexpr int kPadCells = 24;                 // zero cells before and after each chunk (>= kPS + 1)
constexpr int kChunkCells = kPadCells + kMT * 128 + kPadCells;  // 560
constexpr int kChunkBytes = kChunkCells * 16;                   // 8960
constexpr int kW1Bytes = 9 * 1 * 32 * 32;     // taps x K chunks x (N rows x 32 B)
constexpr int kW2Bytes = 9 * 2 * 32 * 32;
// Layer 3 multiplies the unshifted activations once by all nine taps' weights: N = 48 rows
// n = 4 tap + co (36 used), per K chunk; the epilogue sums the nine shifted partial products.
constexpr int kN3 = 48;
constexpr int kW3Bytes = 2 * kN3 * 32;
// partial products P[4 tap + co][cell - kP3Lo] (binary32) for the cells that the kept outputs
// (patch rows / cols 3 .. 18) reach through a tap: 3 kPS + 3 - (kPS + 1) .. 18 kPS + 18 + kPS + 1
constexpr int kP3Lo = 3 * kPS + 3 - (kPS + 1);                  // 46
constexpr int kP3Rows = (18 * kPS + 18 + kPS + 1) - kP3Lo + 1;  // 392
constexpr int kP3Cols = 36;
constexpr int kWBytes = kW1Bytes + kW2Bytes + kW3Bytes;         // 36864
constexpr int kBiasFloats = 32 + 32 + 16;
constexpr int kPackedBytes = kWBytes + kBiasFloats * 4;         // weights then biases
// shared memory map (bytes from the 128-byte aligned base)
constexpr int kSmW = 0;
constexpr int kSmXA = kSmW + kWBytes;                 // features, then layer-2 output (4 chunks)
constexpr int kSmX1 = kSmXA + 4 * kChunkBytes;        // layer-1 output (4 chunks)
constexpr int kSmBias = kSmX1 + 4 * kChunkBytes;      // 80 biases, 4 output scales, 12 1/in_scale
constexpr int kSmBar = kSmBias + (kBiasFloats + 4 + 12) * 4;  // layer barrier, weight-copy barrier
constexpr int kSmSlot = kSmBar + 16;
constexpr int kNetSmemBytes = kSmSlot + 8 + 128;      // + alignment slack
constexpr int kMS = kPS + 2;                          // moment grid side for the features: 24
constexpr uint32_t kTmemCols = 256;  // layers 1, 2: 4 M tiles x 32 fp32 columns; layer 3: 4 x 48
constexpr int kNetThreads = 256;  // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) ..
static_assert(kSmBar % 8 == 0, "mbarrier alignment");
static_assert(5 * kMS * kMS * 4 <= 4 * kChunkBytes, "moments fit in the layer-1 output buffer");
static_assert(kPadCells >= kPS + 1, "shifted reads stay inside a chunk");
static_assert(kP3Lo >= 0 && kP3Lo + kP3Rows <= kMT * 128, "layer-3 partial products lie in the M tiles");
static_assert(kP3Cols * kP3Rows * 4 <= 8 * kChunkBytes, "layer-3 partial products fit in the activation buffers");
static_assert(kMT * kN3 <= (int)kTmemCols, "layer-3 accumulators fit in the TMEM allocation");

// Weights and biases of the three layers in the shared-memory layout above (bf16 weights,
// fp32 biases, zero padding for ci >= CI and co >= CO).
__global__ void pack_net_kernel(const float* __restrict__ params, unsigned char* __restrict__ packed) {
  __nv_bfloat16* w = reinterpret_cast<__nv_bfloat16*>(packed);
  float* bias = reinterpret_cast<float*>(packed + kWBytes);
  const int nw = kWBytes / 2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + kBiasFloats; i += gridDim.x * blockDim.x) {
    if (i >= nw) {
      const int j = i - nw;
      const int layer = j < 32 ? 0 : (j < 64 ? 1 : 2);
      const int co = j - 32 * layer;
      const int CI = layer == 0 ? kC0 : kC1, CO = layer == 2 ? kC3 : kC1;
      const int base = layer == 0 ? 0 : (layer == 1 ? kP1 : kP1 + kP2);
      bias[j] = co < CO ? params[base + CO * CI * 9 + co] : 0.f;
      continue;
    }
    int byte = 2 * i;
    if (byte >= kW1Bytes + kW2Bytes) {
      // layer 3: per K chunk one N = 48 block, row n = 4 tap + co
      byte -= kW1Bytes + kW2Bytes;
      const int kc = byte / (kN3 * 32), in = byte % (kN3 * 32);
      const int n = (in / 256) * 8 + (in % 128) / 16;
      const int k = ((in % 256) / 128) * 8 + (in % 16) / 2;
      const int tap = n / kC3, co = n % kC3, ci = 16 * kc + k;
      w[i] = __float2bfloat16_rn(n < 9 * kC3 && ci < kC2 ? params[kP1 + kP2 + co * kC2 * 9 + ci * 9 + tap] : 0.f);
      continue;
    }
    int N, nkc, CI, CO, base;
    if (byte < kW1Bytes) {
      N = 32, nkc = 1, CI = kC0, CO = kC1, base = 0;
    } else {
      N = 32, nkc = 2, CI = kC1, CO = kC2, base = kP1, byte -= kW1Bytes;
    }
    const int blk = byte / (N * 32), in = byte % (N * 32);
    const int tap = blk / nkc, kc = blk % nkc;
    const int n = (in / 256) * 8 + (in % 128) / 16;
    const int k = ((in % 256) / 128) * 8 + (in % 16) / 2;
    const int ci = 16 * kc + k;
    w[i] = __float2bfloat16_rn(n < CO && ci < CI ? params[base + n * CI * 9 + ci * 9 + tap] : 0.f);
  }
}

__device__ __forceinline__ int wrap_mod(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ float tanh_approx(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Issue one layer: for each M tile, 9 taps x nkc K chunks into TMEM columns mt * n; then commit.
template <int N, int NKC, int FIRST, int NTILES>
__device__ __forceinline__ void issue_layer(uint32_t sbase, int act_off, int w_off, uint32_t tmem, uint64_t* bar) {
  // Descriptors of the layer's first A and B operands; every other operand differs only in its
  // start address, which the descriptor holds in 16-byte units in its low bits (no carry: all
  // addresses lie inside this CTA's shared memory), so it is the base plus a constant.
  constexpr uint32_t idesc = idesc_bf16_f32(128, N);
  const uint64_t a0 = smem_desc(sbase + act_off + (kPadCells + FIRST) * 16, kChunkBytes, 128);
  const uint64_t b0 = smem_desc(sbase + w_off, 128, 256);
#pragma unroll
  for (int mt = 0; mt < NTILES; ++mt) {
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int shift = (tap / 3 - 1) * kPS + (tap % 3 - 1);  // cells
#pragma unroll
      for (int kc = 0; kc < NKC; ++kc) {
        const uint64_t a = a0 + (uint64_t)(int64_t)(mt * 128 + shift + 2 * kc * (kChunkBytes / 16));
        const uint64_t b = b0 + (uint64_t)((tap * NKC + kc) * N * 2);
        tc_mma_bf16(tmem + mt * N, a, b, idesc, (tap | kc) != 0);
      }
    }
  }
  tc_commit(bar);
}

// Layer 3 (32 -> 4 channels): per M tile and K chunk ONE MMA of the unshifted activations by the
// N = 48 block of all nine taps' weights (row n = 4 tap + co), into TMEM columns mt * 48.  Column
// 4 t + co of row m then holds the tap-t partial product sum_k A[m][k] W_t[co][k]; the output at
// cell c is sum_t D[c + shift_t][4 t + co] (layer3_epilogue).  The nine shifted MMAs per chunk of
// the other layers re-read the activations nine times from shared memory, the bound of their
// phases; with four output channels that re-read cost layer 3 54 MMAs for 8 here.
__device__ __forceinline__ void issue_layer3(uint32_t sbase, int act_off, int w_off, uint32_t tmem, uint64_t* bar) {
  constexpr uint32_t idesc = idesc_bf16_f32(128, kN3);
  const uint64_t a0 = smem_desc(sbase + act_off + kPadCells * 16, kChunkBytes, 128);
  const uint64_t b0 = smem_desc(sbase + w_off, 128, 256);
#pragma unroll
  for (int mt = 0; mt < kMT; ++mt) {
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      const uint64_t a = a0 + (uint64_t)(mt * 128 + 2 * kc * (kChunkBytes / 16));
      const uint64_t b = b0 + (uint64_t)(kc * kN3 * 2);
      tc_mma_bf16(tmem + mt * kN3, a, b, idesc, kc != 0);
    }
  }
  tc_commit(bar);
}

// Layer-3 partial products TMEM -> shared memory P[col][cell - kP3Lo] (binary32, col = 4 tap +
// co < 36), for the cells kP3Lo .. kP3Lo + kP3Rows - 1.  Warp w reads the 32 lanes of quarter
// w % 4; warps 0-3 take columns 0-15 and 32-35, warps 4-7 columns 16-31.
__device__ __forceinline__ void layer3_partials(uint32_t tmem, float* __restrict__ P) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
#pragma unroll 1
  for (int mt = 0; mt < kMT; ++mt) {
    const uint32_t t = tmem + ((uint32_t)(32 * quarter) << 16) + mt * kN3;
    const int row = mt * 128 + 32 * quarter + lane - kP3Lo;
    const bool keep = row >= 0 && row < kP3Rows;
    uint32_t r[16];
    tmem_ld16(t + 16 * half, r);
    if (half == 0) {
      uint32_t q[4];
      tmem_ld4(t + 32, q);
      tmem_ld_wait();
      if (keep) {
#pragma unroll
        for (int j = 0; j < 4; ++j) P[(32 + j) * kP3Rows + row] = __uint_as_float(q[j]);
      }
    } else {
      tmem_ld_wait();
    }
    if (keep) {
#pragma unroll
      for (int j = 0; j < 16; ++j) P[(16 * half + j) * kP3Rows + row] = __uint_as_float(r[j]);
    }
  }
}

// Epilogue of a hidden layer: tanh(D + b) of this thread's cell in each M tile -> bf16 chunks.
// Warp w reads TMEM lanes 32 (w % 4) .. (its cells); warps 0-3 take channels 0-15, warps 4-7
// channels 16-31.
__device__ __forceinline__ void hidden_epilogue(uint32_t tmem, const float* __restrict__ bias,
                                                unsigned char* __restrict__ dst) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int quarter = warp & 3, half = warp >> 2;
#pragma unroll 1
  for (int mt = 0; mt < kMT; ++mt) {
    uint32_t r[16];
    tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + mt * 32 + 16 * half, r);
    tmem_ld_wait();
    const int cell = mt * 128 + 32 * quarter + lane;
    const float* b = bias + 16 * half;
    uint32_t pk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j)
      pk[j] = bf16x2(tanh_approx(__uint_as_float(r[2 * j]) + b[2 * j]),
                     tanh_approx(__uint_as_float(r[2 * j + 1]) + b[2 * j + 1]));
#pragma unroll
    for (int c = 0; c < 2; ++c)
      *reinterpret_cast<uint4*>(dst + (2 * half + c) * kChunkBytes + (kPadCells + cell) * 16) =
          make_uint4(pk[4 * c], pk[4 * c + 1], pk[4 * c + 2], pk[4 * c + 3]);
  }
}

// All CTA threads wait for the layer's MMAs; false (uniformly) if a bounded wait ran out here or
// `mine` is false in some thread.
__device__ __forceinline__ bool wait_layer(uint64_t* bar, uint32_t& phase, bool mine) {
  const bool ok = mbar_wait_bounded(bar, phase, kNetWaitNs) && mine;
  phase ^= 1u;
  tc_fence_after();
  return !__syncthreads_or(!ok);
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// The 16 input channels (12 features, 4 zeros) of patch cell `cell` -> XA chunks 0, 1 (bf16).
__device__ __forceinline__ void put_features(unsigned char* sm, int cell, const float (&f)[12]) {
  uint32_t w8[8];
#pragma unroll
  for (int j = 0; j < 6; ++j) w8[j] = bf16x2(f[2 * j], f[2 * j + 1]);
  w8[6] = w8[7] = 0u;
  *reinterpret_cast<uint4*>(sm + kSmXA + (kPadCells + cell) * 16) = make_uint4(w8[0], w8[1], w8[2], w8[3]);
  *reinterpret_cast<uint4*>(sm + kSmXA + kChunkBytes + (kPadCells + cell) * 16) =
      make_uint4(w8[4], w8[5], w8[6], w8[7]);
}

// Patch input from feature planes [batch][12][H][W] (scaled already).
__device__ __forceinline__ void load_features(unsigned char* sm, const float* __restrict__ ib, long plane, int H,
                                              int W, int ty0, int tx0) {
  for (int cell = threadIdx.x; cell < kMT * 128; cell += kNetThreads) {
    float f[12];
    if (cell < kPatch) {
      const int gy = wrap_mod(ty0 - 3 + cell / kPS, H), gx = wrap_mod(tx0 - 3 + cell % kPS, W);
      const float* p = ib + (size_t)gy * W + gx;
#pragma unroll
      for (int k = 0; k < kC0; ++k) f[k] = p[k * plane];
    } else {
#pragma unroll
      for (int k = 0; k < kC0; ++k) f[k] = 0.f;
    }
    put_features(sm, cell, f);
  }
}

// Patch input from the populations of a square grid: pull the 27 populations of each cell of
// the 24 x 24 moment grid (origin ty0 - 4, tx0 - 4), form u = J / rho and B in binary32 (layer-1
// output buffer as scratch), then the features of the 22 x 22 patch: u_x, u_y, B_x, B_y and
// their central differences (d_x, d_y of each in turn), each times 1 / in_scale.
template <typename S>
__device__ __forceinline__ void load_from_pops(unsigned char* sm, const S* __restrict__ pops, const StepGeom& g,
                                               int ty0, int tx0, const float* __restrict__ inv_s) {
  float* mom = reinterpret_cast<float*>(sm + kSmX1);
  constexpr int MM = kMS * kMS;
#pragma unroll 2
  for (int cell = threadIdx.x; cell < MM; cell += kNetThreads) {
    const int y = wrap_mod(ty0 - 4 + cell / kMS, g.ny), x = wrap_mod(tx0 - 4 + cell % kMS, g.nx);
    float v[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) {
      const int i = q % 9;
      const int sx = wrapi(x - vel_x(i), g.nx), sy = wrapi(y - vel_y(i), g.ny);
      v[q] = load_as<float>(pops[(size_t)plane_of(q) * g.plane + (size_t)sy * g.pitch + kXOff + sx]);
    }
    const float rho1 = (((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]))) + v[8];
    const float jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
    const float jy = (v[2] - v[4]) + (v[5] - v[8]) + (v[6] - v[7]);
    float bx = 0.f, by = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      bx += v[9 + i];
      by += v[18 + i];
    }
    const float r = 1.f + rho1;
    mom[cell] = jx / r;
    mom[MM + cell] = jy / r;
    mom[2 * MM + cell] = bx;
    mom[3 * MM + cell] = by;
  }
  __syncthreads();
  for (int cell = threadIdx.x; cell < kMT * 128; cell += kNetThreads) {
    float f[12];
    if (cell < kPatch) {
      const int o = (cell / kPS + 1) * kMS + cell % kPS + 1;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float* a = mom + k * MM;
        f[k] = a[o] * inv_s[k];
        f[4 + 2 * k] = 0.5f * (a[o + 1] - a[o - 1]) * inv_s[4 + 2 * k];
        f[5 + 2 * k] = 0.5f * (a[o + kMS] - a[o - kMS]) * inv_s[5 + 2 * k];
      }
    } else {
#pragma unroll
      for (int k = 0; k < kC0; ++k) f[k] = 0.f;
    }
    put_features(sm, cell, f);
  }
}

// Persistent over tiles (batch x tiles_y x tiles_x).  SRC 0: src = features [batch][12][H][W]
// fp32; SRC 1 / 2: src = binary32 / binary64 populations of the square grid g (batch 1, H = ny,
// W = nx), features formed here with in_scale.  out: [batch][4][H][W] fp32 = (network output)
// x oscale[co] (oscale NULL: 1).
template <int SRC>
__global__ void __launch_bounds__(kNetThreads, 2)
    net_tc_kernel(const void* __restrict__ src, StepGeom g, const float* __restrict__ in_scale,
                  const unsigned char* __restrict__ packed, const float* __restrict__ oscale, int batch, int H,
                  int W, float* __restrict__ out, unsigned* __restrict__ err, int skip_mma) {
  extern __shared__ __align__(128) unsigned char net_smem_raw[];
  unsigned char* sm = net_smem_raw + ((128u - (smem_u32(net_smem_raw) & 127u)) & 127u);
  const uint32_t sbase = smem_u32(sm);
  float* bias = reinterpret_cast<float*>(sm + kSmBias);
  float* inv_s = bias + kBiasFloats + 4;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + kSmBar);
  uint64_t* wbar = bar + 1;
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kSmSlot);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(wbar, 1);
    fence_barrier_init();
  }
  // zero pad cells of the 8 activation chunks (shifted reads reach kPS + 1 cells beyond 0 .. 511)
  for (int i = tid; i < 8 * 2 * kPadCells; i += kNetThreads) {
    const int ch = i / (2 * kPadCells), j = i % (2 * kPadCells);
    const int cell = j < kPadCells ? j : kMT * 128 + j;
    *reinterpret_cast<uint4*>(sm + kSmXA + ch * kChunkBytes + cell * 16) = make_uint4(0, 0, 0, 0);
  }
  // global reads start here: with a programmatic launch the previous step may still be draining
  grid_dependency_wait();
  if (tid == 0) {
    mbar_arrive_expect_tx(wbar, kWBytes);
    bulk_copy_g2s(sm + kSmW, packed, kWBytes, wbar);
  }
  for (int i = tid; i < kBiasFloats + 4 + 12; i += kNetThreads) {
    float v;
    if (i < kBiasFloats) v = reinterpret_cast<const float*>(packed + kWBytes)[i];
    else if (i < kBiasFloats + 4) v = oscale ? oscale[i - kBiasFloats] : 1.f;
    else v = SRC ? 1.f / in_scale[i - kBiasFloats - 4] : 1.f;
    bias[i] = v;
  }
  if (warp == 0) {
    tmem_alloc(slot, kTmemCols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *slot;

  const long plane = (long)H * W;
  const int tiles_x = (W + kTT - 1) / kTT, tiles_y = (H + kTT - 1) / kTT;
  const long ntiles = (long)batch * tiles_x * tiles_y;
  uint32_t phase = 0;
  bool ok = true, weights_ready = false;
  for (long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
    const int b = (int)(tile / ((long)tiles_x * tiles_y));
    const int rem = (int)(tile % ((long)tiles_x * tiles_y));
    const int ty0 = (rem / tiles_x) * kTT, tx0 = (rem % tiles_x) * kTT;
    if (SRC == 0)
      load_features(sm, static_cast<const float*>(src) + (size_t)b * kC0 * plane, plane, H, W, ty0, tx0);
    else if (SRC == 1)
      load_from_pops<float>(sm, static_cast<const float*>(src), g, ty0, tx0, inv_s);
    else
      load_from_pops<double>(sm, static_cast<const double*>(src), g, ty0, tx0, inv_s);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 1: 12 (padded to 16) -> 32
    bool mine = true;
    if (tid == 0) {
      if (!weights_ready) mine = weights_ready = mbar_wait_bounded(wbar, 0, kNetWaitNs);
      // test hook: with skip_mma the first tile's layer-1 MMAs and their commit are left out,
      // so the completion wait below runs out (nothing is in flight when TMEM is freed)
      if (mine && !(skip_mma && tile == blockIdx.x)) issue_layer<32, 1, 0, kMT>(sbase, kSmXA, kSmW, tmem, bar);
      else if (!mine) tc_commit(bar);
    }
    if (!(ok = wait_layer(bar, phase, mine))) break;
    hidden_epilogue(tmem, bias, sm + kSmX1);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 2: 32 -> 32
    if (tid == 0) issue_layer<32, 2, 0, kMT>(sbase, kSmX1, kSmW + kW1Bytes, tmem, bar);
    if (!(ok = wait_layer(bar, phase, true))) break;
    hidden_epilogue(tmem, bias + 32, sm + kSmXA);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // layer 3: 32 -> 4, one N = 48 MMA per M tile and K chunk, taps summed below
    if (tid == 0) issue_layer3(sbase, kSmXA, kSmW + kW1Bytes + kW2Bytes, tmem, bar);
    if (!(ok = wait_layer(bar, phase, true))) break;
    // the MMAs have read the activations: their buffers (XA, X1) now hold the partial products
    float* P = reinterpret_cast<float*>(sm + kSmXA);
    layer3_partials(tmem, P);
    __syncthreads();
    {  // one kept cell per thread: patch row / col 3 + tid / 16, 3 + tid % 16
      static_assert(kNetThreads == kTT * kTT, "one output cell per thread");
      const int pr = 3 + tid / kTT, pc = 3 + tid % kTT;
      const int gy = ty0 + pr - 3, gx = tx0 + pc - 3;
      if (gy < H && gx < W) {
        const int c = pr * kPS + pc - kP3Lo;
        float* ob = out + (size_t)b * kC3 * plane + (size_t)gy * W + gx;
#pragma unroll
        for (int co = 0; co < kC3; ++co) {
          float acc = 0.f;
#pragma unroll
          for (int tap = 0; tap < 9; ++tap) {
            const int shift = (tap / 3 - 1) * kPS + (tap % 3 - 1);
            acc += P[(kC3 * tap + co) * kP3Rows + c + shift];
          }
          ob[co * plane] = (acc + bias[64 + co]) * bias[kBiasFloats + co];
        }
      }
    }
    // TMEM reads and shared-memory operands of this tile are finished before the next tile
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  if (tid == 0) {
    if (!ok) {
      atomicOr(err, 1u);
      mbar_wait_bounded(bar, phase ^ 1u, kNetWaitNs);  // let outstanding MMAs drain
    }
    if (!weights_ready) mbar_wait_bounded(wbar, 0, kNetWaitNs);  // the weight copy has landed
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

int net_grid(int batch, int H, int W, int num_sms) {
  const long tiles = (long)batch * ((H + kTT - 1) / kTT) * ((W + kTT - 1) / kTT);
  const long cap = 2L * num_sms;
  return (int)(tiles < cap ? (tiles < 1 ? 1 : tiles) : cap);
}

template <int SRC>
cudaError_t set_net_attributes() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  // per device, once; handles may be driven from several host threads (setting the attribute
  // twice is harmless, a plain flag read while another thread writes it is not)
  static std::atomic<bool> attr_set[64] = {};
  if (dev < 64 && attr_set[dev].load(std::memory_order_acquire)) return cudaSuccess;
  e = cudaFuncSetAttribute(net_tc_kernel<SRC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kNetSmemBytes);
  if (e == cudaSuccess && dev < 64) attr_set[dev].store(true, std::memory_order_release);
  return e;
}

template <int SRC>
cudaError_t launch_net_impl(const void* src, const StepGeom& g, const float* in_scale, const unsigned char* packed,
                            const float* oscale, int batch, int H, int W, float* out, unsigned* err,
                            int skip_mma, cudaStream_t s) {
  cudaError_t e = set_net_attributes<SRC>();
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return launch_programmatic(net_tc_kernel<SRC>, dim3(net_grid(batch, H, W, sms)), kNetThreads, (size_t)kNetSmemBytes,
                             s, src, g, in_scale, packed, oscale, batch, H, W, out, err, skip_mma);
}

cudaError_t launch_net(const float* in, const unsigned char* packed, const float* oscale, int batch, int H,
                       int W, float* out, unsigned* err, int skip_mma, cudaStream_t s) {
  return launch_net_impl<0>(in, StepGeom{}, nullptr, packed, oscale, batch, H, W, out, err, skip_mma, s);
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
int grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  if (b > 152L * 16) b = 152L * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

int closure_num_params() { return kNumParams; }

cudaError_t prepare_closure_kernels() {
  cudaError_t e = set_net_attributes<1>();
  if (e == cudaSuccess) e = set_net_attributes<2>();
  return e;
}

// Correction planes [4][m][m] (physical units) for the current populations of a square
// binary64 / binary32 grid: one launch of the fused network kernel (pull, u and B, features,
// three tensor-core layers, output scale).
cudaError_t closure_correction(const lbmhd_closure_t* c, int precision, const void* pops, const StepGeom& g,
                               float* corr, unsigned* err, cudaStream_t s) {
  const float* sc = closure_device_scales(c);
  const unsigned char* pk = closure_device_packed(c);
  if (precision == 0) return launch_net_impl<2>(pops, g, sc, pk, sc + 12, 1, g.ny, g.nx, corr, err, 0, s);
  return launch_net_impl<1>(pops, g, sc, pk, sc + 12, 1, g.ny, g.nx, corr, err, 0, s);
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
  unsigned char* packed = nullptr;  // device: bf16 weights + fp32 biases for the tensor-core kernel
  unsigned* tc_err = nullptr;       // device: tensor-core wait timeout flag
  int test_skip_mma = 0;            // failure-detection test hook (lbmhd_closure_test_skip_mma)
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

// Refresh the tensor-core copy of the parameters (after any change of c->params).
int repack(lbmhd_closure_t* c) {
  pack_net_kernel<<<(kWBytes / 2 + kBiasFloats + 255) / 256, 256, 0, c->stream>>>(c->params, c->packed);
  CL_CUDA(c, cudaGetLastError());
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
  if (c->packed) cudaFree(c->packed);
  if (c->tc_err) cudaFree(c->tc_err);
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
  if (e == cudaSuccess) e = cudaMalloc(&c->packed, kPackedBytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->tc_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(c->tc_err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpy(c->params, params, pb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->adam_m, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(c->adam_v, 0, pb);
  if (e == cudaSuccess) e = cudaMemcpy(c->scales, c->host_scales, 16 * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    pack_net_kernel<<<(kWBytes / 2 + kBiasFloats + 255) / 256, 256, 0, c->stream>>>(c->params, c->packed);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
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
  int rc = repack(c);
  if (rc) return rc;
  CL_CUDA(c, cudaStreamSynchronize(c->stream));
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
  return repack(c);
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
    CL_CUDA(c, launch_net(x, c->packed, nullptr, batch, h, w, out, c->tc_err, c->test_skip_mma, s));
  } else {
    const int g = grid_for((long)cells);
    conv_fwd_kernel<kC0, kC1, true><<<g, kThreads, 0, s>>>(x, p1, batch, h, w, c->a1);
    conv_fwd_kernel<kC1, kC2, true><<<g, kThreads, 0, s>>>(c->a1, p2, batch, h, w, c->a2);
    conv_fwd_kernel<kC2, kC3, false><<<g, kThreads, 0, s>>>(c->a2, p3, batch, h, w, out);
  }
  CL_CUDA(c, cudaGetLastError());
  CL_CUDA(c, cudaStreamSynchronize(s));
  if (tensor_cores) {
    unsigned v = 0;
    CL_CUDA(c, cudaMemcpy(&v, c->tc_err, sizeof v, cudaMemcpyDeviceToHost));
    if (v) {
      CL_CUDA(c, cudaMemset(c->tc_err, 0, sizeof v));
      return cfail(c, LBMHD_ERR_TIMEOUT, "a tensor-core completion wait timed out");
    }
  }
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

int lbmhd_closure_test_skip_mma(lbmhd_closure_t* c, int enable) {
  if (!c) return cfail(nullptr, LBMHD_ERR_INVALID, "NULL argument");
  CL_CUDA(c, cudaStreamSynchronize(c->stream));
  c->test_skip_mma = enable ? 1 : 0;
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
const unsigned char* closure_device_packed(const lbmhd_closure_t* c) { return c->packed; }
cudaStream_t closure_stream(const lbmhd_closure_t* c) { return c->stream; }
}  // namespace lbmhd_gpu
