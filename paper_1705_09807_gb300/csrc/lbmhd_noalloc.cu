// Diagnostics of caller-provided device moment fields without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside another framework's memory
// pool or arena (every byte must come from it), code running under a strict memory budget
// that forbids new allocations after start-up, or code on a path where an allocation would
// synchronise the device.  This entry point serves them: the caller passes its device
// inputs and output, and the per-block partial sums live in a fixed, file-scope device
// array of this library instead of a buffer allocated per call.
//
// The reduction is the same as lbmhd_diagnostics' (sums, maxima and the instability flag),
// split over blocks of kCellsPerBlock consecutive cells, then combined by one block in block
// order, so the result is bitwise reproducible for a given grid.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "lbmhd.h"
#include "lbmhd_internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr long kCellsPerBlock = 4096;  // 16 cells per thread
constexpr int kMaxBlocks = 4096;       // capacity: 4096 x 4096 = 16,777,216 cells
constexpr int kSlots = LBMHD_NDIAG + 1;  // the public values plus the instability flag
constexpr int kMaxDevices = 64;

// Partial results, one record of kSlots doubles per block: 4096 x 11 x 8 B = 352 KiB held on
// every GPU that loads the library, until the process exits.  Every call overwrites the
// records it reads, so nothing has to be cleared between calls.
static __device__ __align__(256) double g_partials[kMaxBlocks * kSlots];

std::mutex g_setup_mutex;

__device__ __forceinline__ int wrap(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

__device__ __forceinline__ double iso_d(const double* a, int nx, int ny, int x, int y, int axis) {
  // isotropic lattice derivative sum_i 3 w_i c_i,axis a(x + c_i) over the D2Q9 neighbours
  const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
  const int cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  double s = 0.0;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = axis == 0 ? cx[i] : cy[i];
    if (c == 0) continue;
    const double w = i < 5 ? 1.0 / 9.0 : 1.0 / 36.0;
    s += 3.0 * w * c * a[(size_t)wrap(y + cy[i], ny) * nx + wrap(x + cx[i], nx)];
  }
  return s;
}

__global__ void partial_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                               const double* __restrict__ uy, const double* __restrict__ bx,
                               const double* __restrict__ by, int nx, int ny,
                               double* __restrict__ partials) {
  const long n = (long)nx * ny;
  const long c0 = (long)blockIdx.x * kCellsPerBlock;
  const long c1 = c0 + kCellsPerBlock < n ? c0 + kCellsPerBlock : n;
  double acc[kSlots];
#pragma unroll
  for (int k = 0; k < kSlots; ++k) acc[k] = 0.0;
  for (long c = c0 + threadIdx.x; c < c1; c += kThreads) {
    const int x = (int)(c % nx), y = (int)(c / nx);
    const double r = rho[c], u = ux[c], v = uy[c], b = bx[c], d = by[c];
    acc[0] += r;
    acc[1] += r * u;
    acc[2] += r * v;
    acc[3] += b;
    acc[4] += d;
    acc[5] += 0.5 * r * (u * u + v * v);
    acc[6] += 0.5 * (b * b + d * d);
    const double dxbx = iso_d(bx, nx, ny, x, y, 0), dybx = iso_d(bx, nx, ny, x, y, 1);
    const double dxby = iso_d(by, nx, ny, x, y, 0), dyby = iso_d(by, nx, ny, x, y, 1);
    acc[7] = fmax(acc[7], fabs(dxbx + dyby));
    const int xp = wrap(x + 1, nx), xm = wrap(x - 1, nx);
    const int yp = wrap(y + 1, ny), ym = wrap(y - 1, ny);
    const double cdiv = 0.5 * (bx[(size_t)y * nx + xp] - bx[(size_t)y * nx + xm] +
                               by[(size_t)yp * nx + x] - by[(size_t)ym * nx + x]);
    acc[8] = fmax(acc[8], fabs(cdiv));
    acc[9] = fmax(acc[9], fmax(fmax(fabs(dxbx), fabs(dybx)), fmax(fabs(dxby), fabs(dyby))));
    const bool bad = !(isfinite(r) && isfinite(u) && isfinite(v) && isfinite(b) && isfinite(d)) ||
                     !(r > 0.0) || !(u * u + v * v <= 0.16);
    if (bad) acc[10] = 1.0;
  }
  __shared__ double sh[kSlots][kThreads];
#pragma unroll
  for (int k = 0; k < kSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int k = 0; k < kSlots; ++k) {
        const double a = sh[k][threadIdx.x], b = sh[k][threadIdx.x + w];
        sh[k][threadIdx.x] = (k <= 6) ? a + b : fmax(a, b);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < kSlots) partials[(size_t)blockIdx.x * kSlots + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void final_kernel(const double* __restrict__ partials, int nblocks,
                             double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kSlots) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double v = partials[(size_t)b * kSlots + k];
    a = (k <= 6) ? a + v : fmax(a, v);
  }
  out[k] = a;
}

int set_error(int code, const char* msg) {
  lbmhd_gpu::set_thread_error(msg);
  return code;
}

// Driver calls that identify the current context, reached through the runtime's driver entry
// point (the library does not link libcuda).  cuCtxGetId gives a context an identifier that is
// unique for the life of the process, so a context that was destroyed and re-created (for
// example after cudaDeviceReset) is told apart from its predecessor even if its handle value is
// reused.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

template <typename F>
F driver_fn(const char* name, int version) {
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &f, version, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return nullptr;
  return reinterpret_cast<F>(f);
}

// Identifier of the calling thread's current context; false if it cannot be had (no current
// context yet, or a driver without cuCtxGetId), in which case the caller looks the address up
// afresh.
bool current_context_id(unsigned long long* id) {
  static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent", 4000);
  static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId", 12000);
  if (!get_current || !get_id) return false;
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  return get_id(ctx, id) == CUDA_SUCCESS;
}

struct PartialsAddr {
  double* ptr = nullptr;
  unsigned long long ctx_id = 0;
};
PartialsAddr g_partials_addr[kMaxDevices];

// Device address of g_partials in the current device's current context.  It is looked up with
// cudaGetSymbolAddress on the first call in a context (which also loads the library's module
// into that context if it is not loaded yet) and cached with the context's identifier; a call
// in another context -- a different device, or the same device after its primary context was
// reset -- looks it up again instead of using a stale address.
int partials_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_error(LBMHD_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_error(LBMHD_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long id = 0;
  const bool have_id = current_context_id(&id);
  PartialsAddr& a = g_partials_addr[dev];
  if (!(have_id && a.ptr && a.ctx_id == id)) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p) {
      char buf[256];
      snprintf(buf, sizeof buf, "cudaGetSymbolAddress of the diagnostics scratch failed: %s",
               cudaGetErrorString(e));
      return set_error(LBMHD_ERR_CUDA, buf);
    }
    a.ptr = static_cast<double*>(p);
    // the lookup above makes the primary context current if it was not yet
    a.ctx_id = current_context_id(&id) ? id : 0;
  }
  *out = a.ptr;
  return LBMHD_OK;
}

}  // namespace

extern "C" int lbmhd_diagnostics_fields_noalloc(const double* rho, const double* ux,
                                                const double* uy, const double* bx,
                                                const double* by, int nx, int ny, double* out,
                                                void* stream) {
  if (!rho || !ux || !uy || !bx || !by || !out)
    return set_error(LBMHD_ERR_INVALID, "a field or output pointer is NULL");
  if (nx < 3 || ny < 3) return set_error(LBMHD_ERR_INVALID, "grid sides must be >= 3");
  const long long ncell = (long long)nx * ny;
  if (ncell > (long long)kMaxBlocks * kCellsPerBlock) {
    char buf[256];
    snprintf(buf, sizeof buf,
             "grid %d x %d has %lld cells; the allocation-free diagnostics handle at most %lld",
             nx, ny, ncell, (long long)kMaxBlocks * kCellsPerBlock);
    return set_error(LBMHD_ERR_INVALID, buf);
  }
  double* partials = nullptr;
  int rc = partials_address(&partials);
  if (rc) return rc;
  const int nblocks = (int)((ncell + kCellsPerBlock - 1) / kCellsPerBlock);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  partial_kernel<<<nblocks, kThreads, 0, s>>>(rho, ux, uy, bx, by, nx, ny, partials);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    final_kernel<<<1, 32, 0, s>>>(partials, nblocks, out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return set_error(LBMHD_ERR_CUDA, cudaGetErrorString(e));
  return LBMHD_OK;
}
