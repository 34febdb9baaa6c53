// Auxiliary kernels: equilibrium initialisation, macroscopic moments, canonical population
// export and double-precision diagnostics.  None of them is on the per-step path.
#include <algorithm>
#include <type_traits>

#include "lbmhd_internal.cuh"

namespace lbmhd_gpu {
namespace {

__host__ __device__ constexpr int vx(int i) { return vel_x(i); }
__host__ __device__ constexpr int vy(int i) { return vel_y(i); }
__host__ __device__ constexpr double wt(int i) { return lattice_w(i); }

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Stored (post-collision) populations whose pull gives the equilibria of the fields:
// stored f*_i(x) = f_i^eq(fields(x + c_i)), so that f_i(x) = f*_i(x - c_i) = f_i^eq(x).
// Eq. feq, written as the deviation f_i^eq - w_i; Eq. geq.  Ghost columns written too.
// REL (relative binary16 storage, LBMHD_FP16_REL): the cell's velocity reference U is its own
// initial u rounded to binary16 (planes kQ, kQ + 1), and each stored f value is taken relative
// to w_i (1 + 3 c_i . U).  The equilibria are evaluated in the storage's arithmetic type A:
// binary64 for binary64 storage, binary32 otherwise (the stored value is rounded to binary32 or
// binary16 anyway, and GB300's binary64 rate is about 1/60 of its binary32 rate).
//
// One block per strip of kInitCols columns and band of kInitRows rows.  The fields of rows
// y - 1, y, y + 1 sit in a ring of three shared-memory rows (columns x0 - 1 .. x0 + kInitCols,
// periodic), each value read and converted to A once, with |u|^2 and |B|^2 formed once per cell:
// the nine equilibria of a cell then read only shared memory.  Only the two halo rows of each
// band are read twice, so the input arrays may be page-locked host memory read over the host
// link.  (Converting every binary64 input nine times, once per direction, took 0.45 ms at 2048^2
// on GB300's binary64 conversion rate.)
constexpr int kInitCols = 128, kInitRows = 32;

template <typename T, bool REL = false>
__global__ void __launch_bounds__(kInitCols)
    init_eq_kernel(T* __restrict__ pops, StepGeom g, const double* __restrict__ rho,
                   const double* __restrict__ ux, const double* __restrict__ uy,
                   const double* __restrict__ bx, const double* __restrict__ by) {
  using A = typename std::conditional<sizeof(T) == 8, double, float>::type;
  constexpr int W = kInitCols + 2;
  constexpr int NV = REL ? 9 : 7;  // rho, ux, uy, bx, by, |u|^2, |B|^2 (REL: U_x, U_y in binary16)
  __shared__ A ring[3][NV][W];
  const int x0 = blockIdx.x * kInitCols;
  const int cols = min(kInitCols, g.nx - x0);
  const int nbands = (g.ny + kInitRows - 1) / kInitRows;
  for (int band = blockIdx.y; band < nbands; band += gridDim.y) {
    const int y0 = band * kInitRows, y1 = min(y0 + kInitRows, g.ny);
    // field row yy (in [-1, ny], periodic) into ring slot (yy + 3) mod 3
    auto load_row = [&](int yy) {
      const int slot = (yy + 3) % 3;
      const size_t row = (size_t)wrapi(yy, g.ny) * g.nx;
      for (int j = threadIdx.x; j < cols + 2; j += blockDim.x) {
        const size_t c = row + wrapi(x0 - 1 + j, g.nx);
        const double du = ux[c], dv = uy[c];
        const A r = (A)rho[c], u = (A)du, v = (A)dv, bb = (A)bx[c], d = (A)by[c];
        A* e = &ring[slot][0][j];
        e[0 * W] = r;
        e[1 * W] = u;
        e[2 * W] = v;
        e[3 * W] = bb;
        e[4 * W] = d;
        e[5 * W] = u * u + v * v;
        e[6 * W] = bb * bb + d * d;
        if constexpr (REL) {
          e[7 * W] = (A)__half2float(__double2half(du));
          e[8 * W] = (A)__half2float(__double2half(dv));
        }
      }
    };
    // (the previous band ended with a block barrier: its readers of the ring are done)
    load_row(y0 - 1);
    load_row(y0);
    for (int y = y0; y < y1; ++y) {
      load_row(y + 1);
      __syncthreads();
      const int jx = threadIdx.x + 1;
      const int x = x0 + threadIdx.x;
      if (threadIdx.x < cols) {
        const size_t o = (size_t)y * g.pitch + kXOff + x;
        A Ux = A(0), Uy = A(0);
        if constexpr (REL) {
          const A* e = &ring[y % 3][0][jx];
          Ux = e[7 * W];
          Uy = e[8 * W];
          const T u2[2] = {store_as<T>(Ux), store_as<T>(Uy)};  // exact: Ux, Uy are binary16 values
#pragma unroll
          for (int comp = 0; comp < 2; ++comp) {
            T* pl = pops + (size_t)(kQ + comp) * g.plane + o;
            pl[0] = u2[comp];
            if (x < 2) pl[g.nx] = u2[comp];
            if (x >= g.nx - 2) pl[-g.nx] = u2[comp];
          }
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const A* e = &ring[(y + vy(i) + 3) % 3][0][jx + vx(i)];
          const A r = e[0 * W], u = e[1 * W], v = e[2 * W], b = e[3 * W], d = e[4 * W];
          const A usq = e[5 * W], bsq = e[6 * W];
          const A cu = vx(i) * u + vy(i) * v;
          const A cb = vx(i) * b + vy(i) * d;
          const A csq = (A)(vx(i) * vx(i) + vy(i) * vy(i));
          const A w = (A)wt(i);
          A fdev = w * (r - A(1)) + w * r * (A(3) * cu + A(4.5) * cu * cu - A(1.5) * usq) +
                   A(4.5) * w * (A(0.5) * bsq * csq - cb * cb);
          if (REL) fdev -= A(3) * w * (vx(i) * Ux + vy(i) * Uy);
          const A gx = w * (b + A(3) * (cu * b - cb * u));
          const A gy = w * (d + A(3) * (cu * d - cb * v));
          const T vals[3] = {store_as<T>(fdev), store_as<T>(gx), store_as<T>(gy)};
#pragma unroll
          for (int comp = 0; comp < 3; ++comp) {
            T* pl = pops + (size_t)plane_of(9 * comp + i) * g.plane + o;
            pl[0] = vals[comp];
            if (x < 2) pl[g.nx] = vals[comp];          // ghosts of columns 0, 1 at nx, nx + 1
            if (x >= g.nx - 2) pl[-g.nx] = vals[comp];  // ghosts of columns nx-2, nx-1 at -2, -1
          }
        }
      }
      __syncthreads();
    }
  }
}

// Pull the 27 current populations of cell (x, y) in binary64, f as deviations (for REL, each f
// value plus 3 w_i c_i . U of the source cell that stored it).
template <typename T, bool REL = false>
__device__ __forceinline__ void pull_cell(const T* __restrict__ pops, const StepGeom& g, int x,
                                          int y, double v[27]) {
#pragma unroll
  for (int q = 0; q < 27; ++q) {
    const int i = q % 9;
    const int sx = wrapi(x - vx(i), g.nx), sy = wrapi(y - vy(i), g.ny);
    const size_t src = (size_t)sy * g.pitch + kXOff + sx;
    v[q] = load_as<double>(pops[(size_t)plane_of(q) * g.plane + src]);
    if (REL && q >= 1 && q < 9) {
      const double Ux = load_as<double>(pops[(size_t)kQ * g.plane + src]);
      const double Uy = load_as<double>(pops[(size_t)(kQ + 1) * g.plane + src]);
      v[q] += 3.0 * wt(i) * (vx(i) * Ux + vy(i) * Uy);
    }
  }
}

// Sum of binary32 values kept exactly as the unevaluated pair hi + lo (Knuth's TwoSum: the
// rounding error of each binary32 addition is itself a binary32 value).  Nine stored binary32 or
// binary16 values sum to the binary64 result up to one rounding of lo, with binary32 arithmetic
// only: GB300's binary64 rate (about 1/60 of binary32) made the binary64 sums of the moments
// read-out take 0.55 ms at 2048^2, four times the kernel's memory time.
struct PairSum {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float s = hi + v, bv = s - hi;
    lo += (hi - (s - bv)) + (v - bv);
    hi = s;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

template <typename T, bool REL = false>
__global__ void moments_kernel(const T* __restrict__ pops, StepGeom g, double* __restrict__ rho,
                               double* __restrict__ ux, double* __restrict__ uy,
                               double* __restrict__ bx, double* __restrict__ by) {
  const long n = (long)g.nx * g.ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double rr, jx, jy, sbx, sby;
    if constexpr (sizeof(T) == 8 || REL) {  // binary64 sums (REL: the decoded values are binary64)
      double v[27];
      pull_cell<T, REL>(pops, g, x, y, v);
      double r = 0;
      jx = jy = sbx = sby = 0;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        r += v[i];
        jx += vx(i) * v[i];
        jy += vy(i) * v[i];
        sbx += v[9 + i];
        sby += v[18 + i];
      }
      rr = 1.0 + r;
    } else {  // binary32 / binary16 storage: exact binary32 pair sums of the pulled values
      PairSum r, px, py, qx, qy;
#pragma unroll
      for (int q = 0; q < 27; ++q) {
        const int i = q % 9;
        const int sx = wrapi(x - vx(i), g.nx), sy = wrapi(y - vy(i), g.ny);
        const float v = load_as<float>(pops[(size_t)plane_of(q) * g.plane + (size_t)sy * g.pitch + kXOff + sx]);
        if (q < 9) {
          r.add(v);
          if (vx(i)) px.add(vx(i) > 0 ? v : -v);
          if (vy(i)) py.add(vy(i) > 0 ? v : -v);
        } else if (q < 18) {
          qx.add(v);
        } else {
          qy.add(v);
        }
      }
      rr = 1.0 + r.value();
      jx = px.value();
      jy = py.value();
      sbx = qx.value();
      sby = qy.value();
    }
    rho[c] = rr;
    if (sizeof(T) == 8) {
      ux[c] = jx / rr;
      uy[c] = jy / rr;
    } else {  // binary32 / binary16 storage: a binary32 division (GB300's binary64 divide is slow)
      const float ir = 1.f / (float)rr;
      ux[c] = (double)((float)jx * ir);
      uy[c] = (double)((float)jy * ir);
    }
    bx[c] = sbx;
    by[c] = sby;
  }
}

template <typename T, bool REL = false>
__global__ void populations_kernel(const T* __restrict__ pops, StepGeom g, double* __restrict__ out) {
  const long n = (long)g.nx * g.ny;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx), y = (int)(c / g.nx);
    double v[27];
    pull_cell<T, REL>(pops, g, x, y, v);
#pragma unroll
    for (int q = 0; q < 27; ++q) out[(size_t)q * n + c] = q < 9 ? v[q] + wt(q) : v[q];
  }
}

// ---- diagnostics ----------------------------------------------------------------------
constexpr int kDiagThreads = 256;

__device__ __forceinline__ double iso_d(const double* a, int nx, int ny, int x, int y, int axis) {
  double s = 0.0;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = axis == 0 ? vx(i) : vy(i);
    if (c == 0) continue;
    s += 3.0 * wt(i) * c * a[(size_t)wrapi(y + vy(i), ny) * nx + wrapi(x + vx(i), nx)];
  }
  return s;
}

// Slots: 0 sum rho, 1 sum Jx, 2 sum Jy, 3 sum Bx, 4 sum By, 5 sum rho|u|^2/2, 6 sum |B|^2/2,
// 7 max|div B| isotropic, 8 max|div B| central, 9 max|dB| isotropic, 10 instability flag.
__global__ void diag_partial_kernel(const double* __restrict__ f, int nx, int ny,
                                    double* __restrict__ partials) {
  const long n = (long)nx * ny;
  const double* rho = f;
  const double* ux = f + n;
  const double* uy = f + 2 * n;
  const double* bx = f + 3 * n;
  const double* by = f + 4 * n;
  double acc[kDiagSlots];
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) acc[k] = 0.0;
  for (long c = blockIdx.x * (long)blockDim.x + threadIdx.x; c < n; c += (long)gridDim.x * blockDim.x) {
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
    const int xp = x + 1 == nx ? 0 : x + 1, xm = x == 0 ? nx - 1 : x - 1;
    const int yp = y + 1 == ny ? 0 : y + 1, ym = y == 0 ? ny - 1 : y - 1;
    const double cdiv = 0.5 * (bx[(size_t)y * nx + xp] - bx[(size_t)y * nx + xm] +
                               by[(size_t)yp * nx + x] - by[(size_t)ym * nx + x]);
    acc[8] = fmax(acc[8], fabs(cdiv));
    acc[9] = fmax(acc[9], fmax(fmax(fabs(dxbx), fabs(dybx)), fmax(fabs(dxby), fabs(dyby))));
    const bool bad = !(isfinite(r) && isfinite(u) && isfinite(v) && isfinite(b) && isfinite(d)) ||
                     !(r > 0.0) || !(u * u + v * v <= 0.16);
    if (bad) acc[10] = 1.0;
  }
  __shared__ double sh[kDiagSlots][kDiagThreads];
#pragma unroll
  for (int k = 0; k < kDiagSlots; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = kDiagThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
#pragma unroll
      for (int k = 0; k < kDiagSlots; ++k) {
        const double a = sh[k][threadIdx.x], b = sh[k][threadIdx.x + w];
        sh[k][threadIdx.x] = (k <= 6) ? a + b : fmax(a, b);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < kDiagSlots) partials[(size_t)blockIdx.x * kDiagSlots + threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void diag_final_kernel(const double* __restrict__ partials, int nblocks,
                                  double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= kDiagSlots) return;
  double a = 0.0;
  for (int b = 0; b < nblocks; ++b) {
    const double v = partials[(size_t)b * kDiagSlots + k];
    a = (k <= 6) ? a + v : fmax(a, v);
  }
  out[k] = a;
}

int grid_for(long n, int threads) {
  long b = (n + threads - 1) / threads;
  if (b > 152L * 16) b = 152L * 16;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_init_eq(int precision, void* pops, const StepGeom& g, const double* rho,
                           const double* ux, const double* uy, const double* bx, const double* by,
                           cudaStream_t s) {
  const dim3 grid((g.nx + kInitCols - 1) / kInitCols,
                  (unsigned)std::min((g.ny + kInitRows - 1) / kInitRows, 65535));
  if (precision == 0)
    init_eq_kernel<double><<<grid, kInitCols, 0, s>>>((double*)pops, g, rho, ux, uy, bx, by);
  else if (precision == 1)
    init_eq_kernel<float><<<grid, kInitCols, 0, s>>>((float*)pops, g, rho, ux, uy, bx, by);
  else if (precision == LBMHD_FP16)
    init_eq_kernel<__half><<<grid, kInitCols, 0, s>>>((__half*)pops, g, rho, ux, uy, bx, by);
  else
    init_eq_kernel<__half, true><<<grid, kInitCols, 0, s>>>((__half*)pops, g, rho, ux, uy, bx, by);
  return cudaGetLastError();
}

// Zero the row padding of both population copies: physical columns [0, kXOff - 2) and
// [nx + kXOff + 2, plane) of every plane row.  One thread per padding element; a warp covers a
// row's contiguous run.  (cudaMemset2DAsync over the same 110,592 row pieces at 2048^2 took
// 0.12 ms.)
template <typename W>
__global__ void zero_pads_kernel(W* __restrict__ p0, W* __restrict__ p1, StepGeom g, long rows) {
  const int left = kXOff - 2, right0 = g.nx + kXOff + 2, padw = left + (g.plane - right0);
  const long n = 2 * rows * padw;
  for (long k = blockIdx.x * (long)blockDim.x + threadIdx.x; k < n; k += (long)gridDim.x * blockDim.x) {
    const long rr = k / padw;
    const int j = (int)(k - rr * padw);
    const long row = rr < rows ? rr : rr - rows;
    W* base = rr < rows ? p0 : p1;
    base[(size_t)row * g.plane + (j < left ? j : right0 + (j - left))] = W(0);
  }
}

cudaError_t launch_zero_pads(void* pops0, void* pops1, const StepGeom& g, int nplanes, size_t elem,
                             cudaStream_t s) {
  const long rows = (long)nplanes * g.ny;
  const long n = 2 * rows * (kXOff - 2 + g.plane - (g.nx + kXOff + 2));
  const int grid = grid_for(n, 256);
  if (elem == 8)
    zero_pads_kernel<unsigned long long><<<grid, 256, 0, s>>>((unsigned long long*)pops0,
                                                             (unsigned long long*)pops1, g, rows);
  else if (elem == 4)
    zero_pads_kernel<unsigned><<<grid, 256, 0, s>>>((unsigned*)pops0, (unsigned*)pops1, g, rows);
  else
    zero_pads_kernel<unsigned short><<<grid, 256, 0, s>>>((unsigned short*)pops0,
                                                         (unsigned short*)pops1, g, rows);
  return cudaGetLastError();
}

cudaError_t launch_moments(int precision, const void* pops, const StepGeom& g, double* rho,
                           double* ux, double* uy, double* bx, double* by, cudaStream_t s) {
  const int grid = grid_for((long)g.nx * g.ny, 256);
  if (precision == 0)
    moments_kernel<double><<<grid, 256, 0, s>>>((const double*)pops, g, rho, ux, uy, bx, by);
  else if (precision == 1)
    moments_kernel<float><<<grid, 256, 0, s>>>((const float*)pops, g, rho, ux, uy, bx, by);
  else if (precision == LBMHD_FP16)
    moments_kernel<__half><<<grid, 256, 0, s>>>((const __half*)pops, g, rho, ux, uy, bx, by);
  else
    moments_kernel<__half, true><<<grid, 256, 0, s>>>((const __half*)pops, g, rho, ux, uy, bx, by);
  return cudaGetLastError();
}

cudaError_t launch_populations(int precision, const void* pops, const StepGeom& g, double* out,
                               cudaStream_t s) {
  const int grid = grid_for((long)g.nx * g.ny, 256);
  if (precision == 0)
    populations_kernel<double><<<grid, 256, 0, s>>>((const double*)pops, g, out);
  else if (precision == 1)
    populations_kernel<float><<<grid, 256, 0, s>>>((const float*)pops, g, out);
  else if (precision == LBMHD_FP16)
    populations_kernel<__half><<<grid, 256, 0, s>>>((const __half*)pops, g, out);
  else
    populations_kernel<__half, true><<<grid, 256, 0, s>>>((const __half*)pops, g, out);
  return cudaGetLastError();
}

cudaError_t launch_diagnostics(const double* fields, int nx, int ny, double* partials, double* out,
                               cudaStream_t s) {
  diag_partial_kernel<<<kDiagBlocks, kDiagThreads, 0, s>>>(fields, nx, ny, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  diag_final_kernel<<<1, 32, 0, s>>>(partials, kDiagBlocks, out);
  return cudaGetLastError();
}

}  // namespace lbmhd_gpu
