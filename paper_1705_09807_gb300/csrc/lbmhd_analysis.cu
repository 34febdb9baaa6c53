// Analysis kernels for comparing filtered DNS with LES: the box filter with downsampling, and
// shell-summed kinetic and magnetic energy spectra.  Off the time-step path.
//
// Box filter: out(i, j) = r^-2 sum of the r x r block of `in` starting at (r i, r j) -- the
// discrete top-hat filter of width r (Sec. 1, Eq. VelFilter, with a top-hat G) sampled at
// every r-th cell.
//
// Spectra: a^(k) = n^-2 sum_x a(x) exp(-2 pi i k.x / n) by two passes of a direct DFT with a
// twiddle table (rows, then columns; O(n^3) per field), then
// E_kin(s) = 1/2 sum_{k in shell s} |u_x^(k)|^2 + |u_y^(k)|^2, E_mag(s) likewise with B, where
// shell s holds the integer wavevectors with (2s-1)^2 < 4|k|^2 < (2s+1)^2.  Each shell is summed
// by one block in a fixed order, so results are bitwise reproducible.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>

#include "lbmhd.h"
#include "lbmhd_internal.cuh"

namespace lbmhd_gpu {
namespace {

constexpr int kThreads = 256;

__global__ void block_mean_kernel(const double* __restrict__ in, int nx, int ny, int r,
                                  double* __restrict__ out) {
  const int mx = nx / r, my = ny / r;
  const long m = (long)mx * my;
  const double inv = 1.0 / ((double)r * r);
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < m; c += (long)gridDim.x * blockDim.x) {
    const int i = (int)(c % mx), j = (int)(c / mx);
    double s = 0.0;
    for (int yy = 0; yy < r; ++yy) {
      const double* row = in + (size_t)(j * r + yy) * nx + (size_t)i * r;
      for (int xx = 0; xx < r; ++xx) s += row[xx];
    }
    out[c] = s * inv;
  }
}

__global__ void twiddle_kernel(int n, double2* __restrict__ tw) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * (double)j / (double)n, &s, &c);
    tw[j] = make_double2(c, -s);  // exp(-2 pi i j / n)
  }
}

// G[y][kx] = sum_x f[y][x] exp(-2 pi i kx x / n) for the four fields at once.
__global__ void dft_rows_kernel(const double* __restrict__ f0, const double* __restrict__ f1,
                                const double* __restrict__ f2, const double* __restrict__ f3,
                                int n, const double2* __restrict__ tw, double2* __restrict__ G) {
  const long total = (long)n * n;
  const double* fs[4] = {f0, f1, f2, f3};
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < total; c += (long)gridDim.x * blockDim.x) {
    const int kx = (int)(c % n), y = (int)(c / n);
    double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
    int idx = 0;  // (kx * x) mod n
    for (int x = 0; x < n; ++x) {
      const double2 w = tw[idx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double v = fs[q][(size_t)y * n + x];
        re[q] += v * w.x;
        im[q] += v * w.y;
      }
      idx += kx;
      if (idx >= n) idx -= n;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) G[(size_t)q * total + c] = make_double2(re[q], im[q]);
  }
}

// P_kin[ky][kx] = |u_x^|^2 + |u_y^|^2 over 2, P_mag likewise, with the column DFT and n^-2.
__global__ void dft_cols_power_kernel(const double2* __restrict__ G, int n,
                                      const double2* __restrict__ tw, double* __restrict__ pk,
                                      double* __restrict__ pm) {
  const long total = (long)n * n;
  const double norm = 1.0 / ((double)n * n);
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < total; c += (long)gridDim.x * blockDim.x) {
    const int kx = (int)(c % n), ky = (int)(c / n);
    double re[4] = {0, 0, 0, 0}, im[4] = {0, 0, 0, 0};
    int idx = 0;  // (ky * y) mod n
    for (int y = 0; y < n; ++y) {
      const double2 w = tw[idx];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double2 g = G[(size_t)q * total + (size_t)y * n + kx];
        re[q] += g.x * w.x - g.y * w.y;
        im[q] += g.x * w.y + g.y * w.x;
      }
      idx += ky;
      if (idx >= n) idx -= n;
    }
    double e[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double a = re[q] * norm, b = im[q] * norm;
      e[q] = a * a + b * b;
    }
    pk[c] = 0.5 * (e[0] + e[1]);
    pm[c] = 0.5 * (e[2] + e[3]);
  }
}

// One block per shell s: rows ky in [-s, s], the kx inside (2s-1)^2 < 4(kx^2+ky^2) < (2s+1)^2.
__global__ void shell_sum_kernel(const double* __restrict__ pk, const double* __restrict__ pm,
                                 int n, double* __restrict__ ek, double* __restrict__ em) {
  const int s = blockIdx.x;
  const long lo4 = (long)(2 * s - 1) * (2 * s - 1), hi4 = (long)(2 * s + 1) * (2 * s + 1);
  // wavenumbers in FFT order: -(n/2) .. (n-1)/2 (for even n: -n/2 .. n/2-1)
  const int kneg = -(n / 2), kpos = (n - 1) / 2;
  double ak = 0.0, am = 0.0;
  for (int ky = -s + (int)threadIdx.x; ky <= s; ky += blockDim.x) {
    if (ky < kneg || ky > kpos) continue;
    const double rem_hi = (s + 0.5) * (s + 0.5) - (double)ky * ky;
    if (rem_hi <= 0.0) continue;
    const double rem_lo = (s - 0.5) * (s - 0.5) - (double)ky * ky;
    const int kmax = (int)floor(sqrt(rem_hi)) + 1;
    const int kmin = rem_lo > 0.0 ? (int)floor(sqrt(rem_lo)) - 1 : 0;
    const int row = ky < 0 ? ky + n : ky;
    for (int sgn = 0; sgn < 2; ++sgn) {
      for (int a = (kmin < 0 ? 0 : kmin); a <= kmax; ++a) {
        const int kx = sgn == 0 ? a : -a;
        if (sgn == 1 && a == 0) continue;
        if (kx < kneg || kx > kpos) continue;
        const long k4 = 4L * ((long)kx * kx + (long)ky * ky);
        if (!(k4 < hi4) || !(s == 0 || k4 > lo4)) continue;
        const size_t c = (size_t)row * n + (kx < 0 ? kx + n : kx);
        ak += pk[c];
        am += pm[c];
      }
    }
  }
  __shared__ double sk[kThreads], smg[kThreads];
  sk[threadIdx.x] = ak;
  smg[threadIdx.x] = am;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      sk[threadIdx.x] += sk[threadIdx.x + w];
      smg[threadIdx.x] += smg[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ek[s] = sk[0];
    em[s] = smg[0];
  }
}

int grid_for(long n) {
  long b = (n + kThreads - 1) / kThreads;
  if (b > 152L * 16) b = 152L * 16;
  return b < 1 ? 1 : (int)b;
}

}  // namespace

size_t spectrum_work_bytes(int n) {
  const size_t nn = (size_t)n * n;
  return ((size_t)n * sizeof(double2) + 255) / 256 * 256 + 4 * nn * sizeof(double2) + 2 * nn * sizeof(double);
}

cudaError_t launch_energy_spectrum(const double* ux, const double* uy, const double* bx,
                                   const double* by, int n, int nbins, double* ek, double* em,
                                   void* work, cudaStream_t s) {
  const size_t nn = (size_t)n * n;
  char* w = static_cast<char*>(work);
  double2* tw = reinterpret_cast<double2*>(w);
  double2* G = reinterpret_cast<double2*>(w + ((size_t)n * sizeof(double2) + 255) / 256 * 256);
  double* pk = reinterpret_cast<double*>(G + 4 * nn);
  double* pm = pk + nn;
  twiddle_kernel<<<(n + kThreads - 1) / kThreads, kThreads, 0, s>>>(n, tw);
  dft_rows_kernel<<<grid_for((long)nn), kThreads, 0, s>>>(ux, uy, bx, by, n, tw, G);
  dft_cols_power_kernel<<<grid_for((long)nn), kThreads, 0, s>>>(G, n, tw, pk, pm);
  shell_sum_kernel<<<nbins, kThreads, 0, s>>>(pk, pm, n, ek, em);
  return cudaGetLastError();
}

cudaError_t launch_block_mean(const double* in, int nx, int ny, int r, double* out, cudaStream_t s) {
  block_mean_kernel<<<grid_for((long)(nx / r) * (ny / r)), kThreads, 0, s>>>(in, nx, ny, r, out);
  return cudaGetLastError();
}

}  // namespace lbmhd_gpu

namespace {
int analysis_error(int code, const char* msg) {
  lbmhd_gpu::set_thread_error(msg);
  return code;
}
}  // namespace

extern "C" int lbmhd_block_mean_device(const double* in, int nx, int ny, int r, double* out,
                                       void* stream) {
  if (!in || !out) return analysis_error(LBMHD_ERR_INVALID, "NULL field pointer");
  if (nx < 1 || ny < 1 || r < 1 || nx % r || ny % r)
    return analysis_error(LBMHD_ERR_INVALID, "block mean: r must divide both grid sides");
  cudaError_t e = lbmhd_gpu::launch_block_mean(in, nx, ny, r, out, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return analysis_error(LBMHD_ERR_CUDA, cudaGetErrorString(e));
  return LBMHD_OK;
}

extern "C" size_t lbmhd_energy_spectrum_work_bytes(int n) {
  return n >= 1 ? lbmhd_gpu::spectrum_work_bytes(n) : 0;
}

extern "C" int lbmhd_energy_spectrum_device(const double* ux, const double* uy, const double* bx,
                                            const double* by, int n, int nbins, double* e_kin,
                                            double* e_mag, void* work, size_t work_bytes,
                                            void* stream) {
  if (!ux || !uy || !bx || !by || !e_kin || !e_mag || !work)
    return analysis_error(LBMHD_ERR_INVALID, "NULL pointer");
  if (n < 1 || n > 4096) return analysis_error(LBMHD_ERR_INVALID, "spectrum: n must be in [1, 4096]");
  if (nbins < 1 || nbins > n) return analysis_error(LBMHD_ERR_INVALID, "spectrum: nbins must be in [1, n]");
  if (work_bytes < lbmhd_gpu::spectrum_work_bytes(n))
    return analysis_error(LBMHD_ERR_INVALID, "spectrum: work buffer too small");
  cudaError_t e = lbmhd_gpu::launch_energy_spectrum(ux, uy, bx, by, n, nbins, e_kin, e_mag, work,
                                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return analysis_error(LBMHD_ERR_CUDA, cudaGetErrorString(e));
  return LBMHD_OK;
}
