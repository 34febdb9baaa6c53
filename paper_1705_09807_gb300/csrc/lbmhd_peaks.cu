// Measured binary64 fused multiply-add rate of the current GPU: the ceiling that bounds the
// binary64 form of the fused step, which issues about 216 binary64 instructions per cell update
// and so reaches the arithmetic limit long before the memory one.  GB300 lists no binary64
// figure to divide by, and its binary64 rate is a small fraction of its binary32 one, so the
// library measures it: every thread of a few resident waves runs eight independent chains
// x <- x * a + b (DFMA, latency hidden by the eight chains and the other warps), and the rate
// is the number of DFMAs over the CUDA-event time of the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "lbmhd.h"
#include "lbmhd_internal.cuh"

namespace {

constexpr int kThreads = 256;

// CH independent chains x <- x a + b per thread; the store is never taken but keeps them live
template <int CH>
__global__ void __launch_bounds__(kThreads) dfma_chains_kernel(int iters, double a, double b,
                                                               double* __restrict__ sink) {
  double x[CH];
#pragma unroll
  for (int k = 0; k < CH; ++k) x[k] = 1.0 + 1e-3 * (double)(threadIdx.x + k);
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < CH; ++k) x[k] = fma(x[k], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < CH; ++k) s += x[k];
  // the chains converge to b / (1 - a) = 1
  if (s == -1.0) sink[blockIdx.x] = s;
}

int fail(int code, const char* what, cudaError_t e) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  lbmhd_gpu::set_thread_error(buf);
  return code;
}

template <int CH>
cudaError_t launch_chains(int blocks, int iters, double* sink, cudaStream_t st) {
  dfma_chains_kernel<CH><<<blocks, kThreads, 0, st>>>(iters, 0.9999999, 1e-7, sink);
  return cudaGetLastError();
}

}  // namespace

// The measurement tries three shapes -- 4, 8 and 16 chains per thread, with 16, 8 and 4 resident
// blocks of 256 threads per SM -- and reports the fastest, so that no one shape's latency or
// occupancy limit is mistaken for the arithmetic rate.
extern "C" int lbmhd_probe_fp64_fma_rate(int iters, int repeats, double* dfma_per_second) {
  if (!dfma_per_second || iters < 1 || iters > (1 << 20) || repeats < 1 || repeats > 100) {
    lbmhd_gpu::set_thread_error("lbmhd_probe_fp64_fma_rate: iters in [1, 2^20], repeats in [1, 100]");
    return LBMHD_ERR_INVALID;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(LBMHD_ERR_CUDA, "device query", e);
  const int max_blocks = sms * 16;
  double* sink = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&sink, sizeof(double) * max_blocks);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  double best = 0.0;
  const int chains[3] = {4, 8, 16}, per_sm[3] = {16, 8, 4};
  for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
    const int blocks = sms * per_sm[v];
    auto launch = [&]() {
      return chains[v] == 4 ? launch_chains<4>(blocks, iters, sink, st)
                            : (chains[v] == 8 ? launch_chains<8>(blocks, iters, sink, st)
                                              : launch_chains<16>(blocks, iters, sink, st));
    };
    e = launch();  // warm-up launch (clocks, instruction cache)
    std::vector<float> ms;
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
      e = cudaEventRecord(t0, st);
      if (e == cudaSuccess) e = launch();
      if (e == cudaSuccess) e = cudaEventRecord(t1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(t1);
      float m = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&m, t0, t1);
      if (e == cudaSuccess) ms.push_back(m);
    }
    if (e == cudaSuccess) {
      std::sort(ms.begin(), ms.end());
      const double med = ms[ms.size() / 2];  // upper median
      const double dfma = (double)blocks * kThreads * chains[v] * (double)iters;
      best = std::max(best, dfma / (med * 1e-3));
    }
  }
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (st) cudaStreamDestroy(st);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) return fail(LBMHD_ERR_CUDA, "fp64 FMA probe", e);
  *dfma_per_second = best;
  return LBMHD_OK;
}
