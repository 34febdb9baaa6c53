// Fused time step of the filtered LES lattice Boltzmann MHD model (Flint & Vahala,
// arXiv:1705.09807): one launch per step, all of
//   pull-stream -> moments -> gradients -> filtered equilibria -> relax -> store
// on the GPU with each population read once from HBM and written once.
//
// Work decomposition.  A block of kStepThreads threads owns a strip of that many adjacent
// columns and a band of `band` rows; each thread owns one column and walks the band from
// top to bottom.  For row y it
//   1. pulls the 27 populations of row y+1 (f_i(x) = f*_i(x - c_i), periodic) into registers
//      and forms their moments, writing J and B of row y+1 to a 4-row shared-memory ring;
//   2. after one barrier, takes the x-differences of J, B from the ring (and, for the
//      isotropic stencil, the diagonal neighbours from the rows above and below), and the
//      y-differences from the moments it holds in registers for rows y-1 and y+1;
//   3. collides row y (pulled one iteration earlier, still in registers) and stores it.
// The moments of the two columns just outside the strip and of row band_start-1 are
// recomputed by the block (halo), so no intermediate ever goes to HBM.  Rows are pitched to
// 32 elements, so each warp-wide load or store of one plane touches whole 128-byte lines
// (the +-1 column shifts of the pull straddle two lines; the neighbour warp's reads hit L1/L2).
//
// Collision (Sec. 2, Eqs. LBKinEqn, LBMagEqn, Transformation).  Fluid, MRT in moment space:
//   f* = f - T^{-1} S (T f - Mbar^eq);  T^{-1} = T^T diag(1/|T_j|^2) since T's rows are
// orthogonal, and only rows j = 3..8 are non-conserved, so the transform is done with the
// sparse integer rows of Eq. FluidTMatrix.  Magnetic, SRT: in moment space
//   N* = N - s_m (N - Nbar^eq)  is the same as  g* = g - s_m (g - T_m^{-1} Nbar^eq),
// and T_m^{-1} Nbar^eq is Eq. geq with the electric term E = (J x B)/rho replaced by its
// filtered value, so the magnetic collision is done in distribution space.  Both rewrites
// are exact algebra; only the rounding order differs from the moment-space statement.
//
// Filtered equilibria (Sec. 2.1 with Sec. 3's simplification, density gradients dropped):
//   J_a J_b / rho -> (J_a J_b + k G_ab)/rho,  B_a B_b -> B_a B_b + k H_ab,
//   E -> (J_x B_y - J_y B_x + k (K_xy - K_yx))/rho,   k = Delta^2/12,
//   G_ab = d_b'J_a d_b'J_b, H_ab = d_b'B_a d_b'B_b, K_ab = d_b'J_a d_b'B_b (sum over b').
#include "lbmhd_internal.cuh"

namespace lbmhd_gpu {
namespace {

// Paper's D2Q9 velocity order (Sec. 2): c_x = {0,1,0,-1,0,1,-1,-1,1}, c_y = {0,0,1,0,-1,1,1,-1,-1}.
__host__ __device__ constexpr int vel_x(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int vel_y(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}

template <typename T>
struct KCoef {
  T r3, r4, r5, r6, r7, r8, sm, kq;
};

template <typename T>
__device__ __forceinline__ T ld(const T* p) {
  return __ldg(p);
}

// Pull the populations of one cell.  cols[0..2] = columns x-1, x, x+1; rows[0..2] = row
// offsets (row * pitch) of y-1, y, y+1.  Population i comes from (x - c_ix, y - c_iy).
template <typename T, bool WITH_REST>
__device__ __forceinline__ void pull27(const T* __restrict__ src, size_t plane, const int cols[3],
                                       const size_t rows[3], T v[kQ]) {
#pragma unroll
  for (int q = 0; q < kQ; ++q) {
    const int i = q % 9;
    if (!WITH_REST && q == 0) {  // the rest population f_0 enters neither J nor B
      v[q] = T(0);
      continue;
    }
    const int col = cols[1 - vel_x(i)];
    const size_t row = rows[1 - vel_y(i)];
    v[q] = ld(src + (size_t)q * plane + row + col);
  }
}

template <typename T>
__device__ __forceinline__ void moments_jb(const T v[kQ], T& jx, T& jy, T& bx, T& by) {
  jx = (v[1] - v[3]) + (v[5] - v[6]) + (v[8] - v[7]);
  jy = (v[2] - v[4]) + (v[5] - v[8]) + (v[6] - v[7]);
  bx = ((v[9] + v[10]) + (v[11] + v[12])) + ((v[13] + v[14]) + (v[15] + v[16])) + v[17];
  by = ((v[18] + v[19]) + (v[20] + v[21])) + ((v[22] + v[23]) + (v[24] + v[25])) + v[26];
}

template <typename T>
__device__ __forceinline__ T moment_rho_dev(const T v[kQ]) {
  return ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7])) + v[8];
}

// Collision of one cell; p[] holds the pulled (current) populations with f as deviations
// f_i - w_i, and receives the post-collision values.  rho1 = rho - 1.  dJ = undivided
// differences {dx Jx, dy Jx, dx Jy, dy Jy}, dB likewise; c.kq folds in their scale.
template <typename T>
__device__ __forceinline__ void collide(T p[kQ], T rho1, T jx, T jy, T bx, T by, const T dJ[4],
                                        const T dB[4], const KCoef<T>& c) {
  const T ir = T(1) / (T(1) + rho1);
  const T k = c.kq;
  // gradient products
  const T Gxx = dJ[0] * dJ[0] + dJ[1] * dJ[1];
  const T Gyy = dJ[2] * dJ[2] + dJ[3] * dJ[3];
  const T Gxy = dJ[0] * dJ[2] + dJ[1] * dJ[3];
  const T Hxx = dB[0] * dB[0] + dB[1] * dB[1];
  const T Hyy = dB[2] * dB[2] + dB[3] * dB[3];
  const T Hxy = dB[0] * dB[2] + dB[1] * dB[3];
  const T Kxy = dJ[0] * dB[2] + dJ[1] * dB[3];  // d J_x . d B_y
  const T Kyx = dJ[2] * dB[0] + dJ[3] * dB[1];  // d J_y . d B_x
  // filtered quadratic terms of the equilibria
  const T Qxx = (jx * jx + k * Gxx) * ir;
  const T Qyy = (jy * jy + k * Gyy) * ir;
  const T Qxy = (jx * jy + k * Gxy) * ir;
  const T Rxx = bx * bx + k * Hxx;
  const T Ryy = by * by + k * Hyy;
  const T Rxy = bx * by + k * Hxy;
  const T E = (jx * by - jy * bx + k * (Kxy - Kyx)) * ir;

  // ---- fluid: non-equilibrium parts of moments 3..8 (rows of Eq. FluidTMatrix) ----
  const T a13 = p[1] + p[3], a24 = p[2] + p[4], a57 = p[5] + p[7], a68 = p[6] + p[8];
  const T qq = Qxx + Qyy;
  const T n3 = (a57 - a68) - (Qxy - Rxy);
  const T n4 = (a13 - a24) - ((Qxx - Qyy) - (Rxx - Ryy));
  const T n5 = T(2) * (p[3] - p[1]) + ((p[5] - p[6]) + (p[8] - p[7])) + jx;
  const T n6 = T(2) * (p[4] - p[2]) + ((p[5] - p[8]) + (p[6] - p[7])) + jy;
  const T n7 = T(4) * p[0] - T(5) * (a13 + a24) + T(4) * (a57 + a68) + T(3) * qq;
  // M_8 of the deviations plus T_8 . w = 5/3 minus M_8^eq = 5/3 rho - 3 qq
  const T n8 = T(4) * p[0] - (a57 + a68) - T(5.0 / 3.0) * rho1 + T(3) * qq;
  const T d3 = c.r3 * n3, d4 = c.r4 * n4, d5 = c.r5 * n5, d6 = c.r6 * n6, d7 = c.r7 * n7,
          d8 = c.r8 * n8;
  // f* = f - T^T (d): columns of T for each population
  const T e78 = d8 - T(4) * d7;
  p[0] -= T(4) * (d7 + d8);
  p[1] += (T(5) * d7 - d4) + T(2) * d5;
  p[2] += (T(5) * d7 + d4) + T(2) * d6;
  p[3] += (T(5) * d7 - d4) - T(2) * d5;
  p[4] += (T(5) * d7 + d4) - T(2) * d6;
  p[5] += e78 - (d3 + d5 + d6);
  p[6] += e78 + (d3 + d5 - d6);
  p[7] += e78 + (d5 + d6 - d3);
  p[8] += e78 + (d3 + d6 - d5);

  // ---- magnetic: SRT toward Eq. geq with the filtered E ----
  // g^eq_x,i = w_i (B_x - 3 c_iy E),  g^eq_y,i = w_i (B_y + 3 c_ix E).  The rest population takes
  // B minus the other eight, so the equilibria sum to B exactly up to one rounding even where
  // the weights are not representable (binary32): no systematic drift of the magnetic flux.
  // The update g* = g + s_m (g^eq - g) rounds the small non-equilibrium part, not g itself.
  const T sm = c.sm;
  const T e3 = T(3) * E;
  const T wa = T(1.0 / 9.0), wd = T(1.0 / 36.0);
  {
    // x component: c_iy = {0,0,1,0,-1,1,1,-1,-1}
    const T ea = wa * bx, em = wa * (bx - e3), ep = wa * (bx + e3);
    const T dm = wd * (bx - e3), dp = wd * (bx + e3);
    const T e0 = bx - (((ea + ea) + (em + ep)) + ((dm + dm) + (dp + dp)));
    p[9] += sm * (e0 - p[9]);
    p[10] += sm * (ea - p[10]);
    p[11] += sm * (em - p[11]);
    p[12] += sm * (ea - p[12]);
    p[13] += sm * (ep - p[13]);
    p[14] += sm * (dm - p[14]);
    p[15] += sm * (dm - p[15]);
    p[16] += sm * (dp - p[16]);
    p[17] += sm * (dp - p[17]);
  }
  {
    // y component: c_ix = {0,1,0,-1,0,1,-1,-1,1}
    const T ea = wa * by, ep = wa * (by + e3), em = wa * (by - e3);
    const T dp = wd * (by + e3), dm = wd * (by - e3);
    const T e0 = by - (((ea + ea) + (em + ep)) + ((dm + dm) + (dp + dp)));
    p[18] += sm * (e0 - p[18]);
    p[19] += sm * (ep - p[19]);
    p[20] += sm * (ea - p[20]);
    p[21] += sm * (em - p[21]);
    p[22] += sm * (ea - p[22]);
    p[23] += sm * (dp - p[23]);
    p[24] += sm * (dm - p[24]);
    p[25] += sm * (dm - p[25]);
    p[26] += sm * (dp - p[26]);
  }
}

template <typename T>
struct StepSmem {
  T m[kRing][4][kStepThreads + 2];  // J_x, J_y, B_x, B_y of 4 rows, strip plus 1-column halo
};

template <typename T, int ISO, int MINB>
__global__ void __launch_bounds__(kStepThreads, MINB)
    fused_step_kernel(const T* __restrict__ src, T* __restrict__ dst, StepGeom g, KCoef<T> c) {
  __shared__ StepSmem<T> sh;
  const int t = threadIdx.x;
  const int nx = g.nx, ny = g.ny;
  const int x0 = blockIdx.x * kStepThreads;
  const int ncol = min(kStepThreads, nx - x0);
  const bool active = t < ncol;
  const int y0 = blockIdx.y * g.band;
  const int y1 = min(y0 + g.band, ny);
  if (y0 >= ny) return;  // uniform per block

  const int x = x0 + t;
  int cols[3];
  cols[1] = active ? x : x0;
  cols[0] = cols[1] == 0 ? nx - 1 : cols[1] - 1;
  cols[2] = cols[1] == nx - 1 ? 0 : cols[1] + 1;
  // halo duties: thread 0 -> column left of the strip, thread ncol-1 -> column right of it
  const bool hleft = (t == 0);
  const bool hright = (t == ncol - 1);
  int hcl[3], hcr[3];
  hcl[1] = x0 == 0 ? nx - 1 : x0 - 1;
  hcl[0] = hcl[1] == 0 ? nx - 1 : hcl[1] - 1;
  hcl[2] = hcl[1] == nx - 1 ? 0 : hcl[1] + 1;
  hcr[1] = (x0 + ncol == nx) ? 0 : x0 + ncol;
  hcr[0] = hcr[1] == 0 ? nx - 1 : hcr[1] - 1;
  hcr[2] = hcr[1] == nx - 1 ? 0 : hcr[1] + 1;
  const int si = t + 1;        // shared-memory slot of this column
  const int sr = ncol + 1;     // slot of the right halo column
  const size_t pitch = (size_t)g.pitch;

  auto row_offsets = [&](int y, size_t r[3]) {
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    r[0] = (size_t)ym * pitch;
    r[1] = (size_t)y * pitch;
    r[2] = (size_t)yp * pitch;
  };
  // moments of the halo columns of row y into ring slot `slot`
  auto halo = [&](int y, int slot) {
    if (hleft || hright) {
      size_t r[3];
      row_offsets(y, r);
      T v[kQ], jx, jy, bx, by;
      if (hleft) {
        pull27<T, false>(src, g.plane, hcl, r, v);
        moments_jb(v, jx, jy, bx, by);
        sh.m[slot][0][0] = jx;
        sh.m[slot][1][0] = jy;
        sh.m[slot][2][0] = bx;
        sh.m[slot][3][0] = by;
      }
      if (hright) {
        pull27<T, false>(src, g.plane, hcr, r, v);
        moments_jb(v, jx, jy, bx, by);
        sh.m[slot][0][sr] = jx;
        sh.m[slot][1][sr] = jy;
        sh.m[slot][2][sr] = bx;
        sh.m[slot][3][sr] = by;
      }
    }
  };

  // ---- prologue: row y0-1 (moments only) and row y0 (populations kept) ----
  T jxm = 0, jym = 0, bxm = 0, bym = 0;        // row y-1
  T rho1c = 0, jxc = 0, jyc = 0, bxc = 0, byc = 0;  // row y
  T p[kQ];
  {
    const int ym = y0 == 0 ? ny - 1 : y0 - 1;
    size_t r[3];
    if (active) {
      row_offsets(ym, r);
      pull27<T, false>(src, g.plane, cols, r, p);
      moments_jb(p, jxm, jym, bxm, bym);
      sh.m[0][0][si] = jxm;
      sh.m[0][1][si] = jym;
      sh.m[0][2][si] = bxm;
      sh.m[0][3][si] = bym;
    }
    halo(ym, 0);
    if (active) {
      row_offsets(y0, r);
      pull27<T, true>(src, g.plane, cols, r, p);
      moments_jb(p, jxc, jyc, bxc, byc);
      rho1c = moment_rho_dev(p);
      sh.m[1][0][si] = jxc;
      sh.m[1][1][si] = jyc;
      sh.m[1][2][si] = bxc;
      sh.m[1][3][si] = byc;
    }
    halo(y0, 1);
  }

  // ---- march down the band ----
  int it = 1;  // ring index of row y is it & 3
  for (int y = y0; y < y1; ++y, ++it) {
    const int yn = y == ny - 1 ? 0 : y + 1;
    const int sn = (it + 1) & (kRing - 1);
    const int sc = it & (kRing - 1);
    const int sp = (it - 1) & (kRing - 1);
    T q[kQ];
    T rho1n = 0, jxn = 0, jyn = 0, bxn = 0, byn = 0;
    if (active) {
      size_t r[3];
      row_offsets(yn, r);
      pull27<T, true>(src, g.plane, cols, r, q);
      moments_jb(q, jxn, jyn, bxn, byn);
      rho1n = moment_rho_dev(q);
      sh.m[sn][0][si] = jxn;
      sh.m[sn][1][si] = jyn;
      sh.m[sn][2][si] = bxn;
      sh.m[sn][3][si] = byn;
    }
    halo(yn, sn);
    __syncthreads();
    if (active) {
      T dJ[4], dB[4];
      if (ISO) {
        // undivided isotropic differences: 4 (a_E - a_W) + (a_NE - a_NW) + (a_SE - a_SW)
        // and 4 (a_N - a_S) + (a_NE - a_SE) + (a_NW - a_SW); their scale 1/12 is in kq
        T dx[4], dy[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const T e = sh.m[sc][f][si + 1], w = sh.m[sc][f][si - 1];
          const T ne = sh.m[sn][f][si + 1], nw = sh.m[sn][f][si - 1], nn = sh.m[sn][f][si];
          const T se = sh.m[sp][f][si + 1], sw = sh.m[sp][f][si - 1], ss = sh.m[sp][f][si];
          dx[f] = T(4) * (e - w) + ((ne - nw) + (se - sw));
          dy[f] = T(4) * (nn - ss) + ((ne - se) + (nw - sw));
        }
        dJ[0] = dx[0]; dJ[1] = dy[0]; dJ[2] = dx[1]; dJ[3] = dy[1];
        dB[0] = dx[2]; dB[1] = dy[2]; dB[2] = dx[3]; dB[3] = dy[3];
      } else {
        // undivided central differences a(+1) - a(-1); their scale 1/2 is in kq
        dJ[0] = sh.m[sc][0][si + 1] - sh.m[sc][0][si - 1];
        dJ[1] = jxn - jxm;
        dJ[2] = sh.m[sc][1][si + 1] - sh.m[sc][1][si - 1];
        dJ[3] = jyn - jym;
        dB[0] = sh.m[sc][2][si + 1] - sh.m[sc][2][si - 1];
        dB[1] = bxn - bxm;
        dB[2] = sh.m[sc][3][si + 1] - sh.m[sc][3][si - 1];
        dB[3] = byn - bym;
      }
      collide(p, rho1c, jxc, jyc, bxc, byc, dJ, dB, c);
      T* o = dst + (size_t)y * pitch + x;
#pragma unroll
      for (int qq = 0; qq < kQ; ++qq) o[(size_t)qq * g.plane] = p[qq];
      // rotate the row window
#pragma unroll
      for (int qq = 0; qq < kQ; ++qq) p[qq] = q[qq];
      jxm = jxc; jym = jyc; bxm = bxc; bym = byc;
      rho1c = rho1n; jxc = jxn; jyc = jyn; bxc = bxn; byc = byn;
    }
  }
}

template <typename T>
KCoef<T> cast_coef(const StepCoef& c) {
  KCoef<T> k;
  k.r3 = (T)c.r[3];
  k.r4 = (T)c.r[4];
  k.r5 = (T)c.r[5];
  k.r6 = (T)c.r[6];
  k.r7 = (T)c.r[7];
  k.r8 = (T)c.r[8];
  k.sm = (T)c.s_m;
  k.kq = (T)c.kq;
  return k;
}

template <typename T, int MINB>
cudaError_t launch_step(const T* src, T* dst, const StepGeom& g, const StepCoef& c, int stencil,
                        cudaStream_t s) {
  dim3 grid((g.nx + kStepThreads - 1) / kStepThreads, (g.ny + g.band - 1) / g.band);
  KCoef<T> k = cast_coef<T>(c);
  if (stencil == 1)
    fused_step_kernel<T, 1, MINB><<<grid, kStepThreads, 0, s>>>(src, dst, g, k);
  else
    fused_step_kernel<T, 0, MINB><<<grid, kStepThreads, 0, s>>>(src, dst, g, k);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_f64(const double* src, double* dst, const StepGeom& g, const StepCoef& c,
                            int stencil, cudaStream_t s) {
  return launch_step<double, 1>(src, dst, g, c, stencil, s);
}

cudaError_t launch_step_f32(const float* src, float* dst, const StepGeom& g, const StepCoef& c,
                            int stencil, cudaStream_t s) {
  return launch_step<float, 3>(src, dst, g, c, stencil, s);
}

// Rows per block: long bands amortise the two recomputed halo rows, short bands give enough
// blocks to fill 152 SMs several times over.
int step_band_rows(int nx, int ny, int precision, int num_sms) {
  const int strips = (nx + kStepThreads - 1) / kStepThreads;
  const int per_sm = precision == 0 ? 1 : 3;  // resident blocks per SM (launch bounds)
  const long target_blocks = (long)num_sms * per_sm * 4;  // about four waves
  long band = ((long)strips * ny + target_blocks - 1) / target_blocks;
  if (band < 4) band = 4;
  if (band > 64) band = 64;
  if (band > ny) band = ny;
  return (int)band;
}

}  // namespace lbmhd_gpu
