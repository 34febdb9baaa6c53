// Internal declarations shared by the translation units of liblbmhd.so.
//
// HBM layout of the population state (one copy; the handle holds two for ping-pong):
//   ny rows, each holding the row segment of all 27 planes one after the other ([y][plane][x],
//   x fastest; a row of one plane is `plane` elements, a row of all planes `pitch` = 27 plane
//   elements), so the data a row of the step needs lies together in memory (measured 1.6%
//   faster at 4096^2 binary32 than whole planes one after another).  Logical column x (0..nx-1) sits at
//   physical column x + kXOff, so every row's interior starts on a 128-byte (binary32) or
//   256-byte (binary64) boundary; physical kXOff-2, kXOff-1 and nx+kXOff, nx+kXOff+1 are ghost
//   copies of logical columns nx-2, nx-1 and 0, 1, kept up to date by every writer, so a row
//   segment read in one piece already contains the periodic x-neighbours two deep (the pull of
//   a halo column reaches two columns outside the strip).  plane = roundup(nx + kXOff + 2, 32).
//   Plane order groups the populations by c_y (the row they are pulled from):
//     planes 0..8   c_y = +1: f_2 f_5 f_6, g_x,2 g_x,5 g_x,6, g_y,2 g_y,5 g_y,6
//     planes 9..17  c_y =  0: f_0 f_1 f_3, g_x,0 g_x,1 g_x,3, g_y,0 g_y,1 g_y,3
//     planes 18..26 c_y = -1: f_4 f_7 f_8, g_x,4 g_x,7 g_x,8, g_y,4 g_y,7 g_y,8
//   so the pulled row y of all 27 populations is three boxes: rows y-1, y, y+1 of one
//   9-plane group each.
//   The stored values are the POST-COLLISION populations f*_i(x), g*_i(x) of the last step;
//   the current (post-stream) populations are pulled: f_i(x) = f*_i(x - c_i), periodic.
//   f is stored as the deviation f_i - w_i from the rest state (rho = 1, u = 0), g as is.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>

#include "lbmhd.h"
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbmhd_gpu {

constexpr int kQ = 27;             // populations per cell: 9 (f) + 2 x 9 (g)
constexpr int kStepThreads = 128;  // threads (= columns) per block of the fused step
constexpr int kRing = 4;           // rows of moments kept in shared memory
constexpr int kXOff = 32;          // physical column of logical x = 0
// Staged row segment of a strip: it starts `box_lead` columns left of the strip (so its first
// byte is 16-byte aligned for the tensor copy) and spans the strip plus a lead on each side.
__host__ __device__ constexpr int box_lead(int elem_bytes) { return elem_bytes == 2 ? 8 : 4; }
__host__ __device__ constexpr int box_width(int elem_bytes) {
  return kStepThreads + 2 * box_lead(elem_bytes);
}

// Paper's D2Q9 velocity order (Sec. 2): c_x = {0,1,0,-1,0,1,-1,-1,1}, c_y = {0,0,1,0,-1,1,1,-1,-1}.
__host__ __device__ constexpr int vel_x(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int vel_y(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
// group of velocity i (0: c_y = +1, 1: c_y = 0, 2: c_y = -1) and its index inside the group
__host__ __device__ constexpr int group_of(int i) { return vel_y(i) == 1 ? 0 : (vel_y(i) == 0 ? 1 : 2); }
__host__ __device__ constexpr int index_in_group(int i) {
  return (i == 2 || i == 0 || i == 4) ? 0 : ((i == 5 || i == 1 || i == 7) ? 1 : 2);
}
// storage plane of canonical population q (0..8 f_i, 9..17 g_x,i, 18..26 g_y,i)
__host__ __device__ constexpr int plane_of(int q) {
  return 9 * group_of(q % 9) + 3 * (q / 9) + index_in_group(q % 9);
}
// Inverse of plane_of: the population index q stored in plane pl.
__host__ __device__ constexpr int q_of_plane(int pl) {
  int q = 0;
  while (plane_of(q) != pl) ++q;
  return q;
}
__host__ __device__ constexpr double lattice_w(int i) {
  return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
}

// Conversions between the storage type S of the populations and the arithmetic type C.
template <typename C, typename S>
__device__ __forceinline__ C load_as(S v) { return static_cast<C>(v); }
template <>
__device__ __forceinline__ float load_as<float, __half>(__half v) { return __half2float(v); }
template <>
__device__ __forceinline__ double load_as<double, __half>(__half v) { return (double)__half2float(v); }
template <typename S, typename C>
__device__ __forceinline__ S store_as(C v) { return static_cast<S>(v); }
template <>
__device__ __forceinline__ __half store_as<__half, float>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __half store_as<__half, double>(double v) { return __double2half(v); }

// Per-launch constants of the fused step, computed on the host in binary64.
struct StepCoef {
  double r[9];   // r[j] = s_j / |T_j|^2 for j = 3..8 (relaxation scaled by T T^T's diagonal)
  double s_m;    // magnetic rate
  double kq;     // Delta^2/12 times the squared scale of the undivided stencil differences
};

struct StepGeom {
  int nx, ny, pitch;  // grid; elements from one row to the next (all 27 planes of a row)
  size_t plane;       // elements from one plane to the next within a row
  int band;           // rows per block
  int skip_copy;      // test hook: 1 = block (0, 0) never issues its third row copy, so its
                      // bounded wait runs out and the step reports a timeout (no fault)
};

// Fused step launchers (lbmhd_step.cu).  `src` is a 3-D tensor map {plane, 27, ny} of the
// source copy (box {box_width(elem), 1, 9}); dst is the other copy.  *err receives 1 if a pipeline wait
// timed out (the kernel then stops early; the state is not valid).  corr (may be NULL): four
// binary32 planes [4][ny][nx] added to the subgrid terms of the collision (xy stress, normal
// stress difference, trace, electric field); not offered for binary16 storage.  flip (0 / 1)
// reverses the bands' marching directions; callers pass the source copy's index so that the
// direction alternates from step to step (results do not depend on it).
cudaError_t launch_step_f64(const CUtensorMap& src, double* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, const float* corr,
                            int flip, cudaStream_t s);
cudaError_t launch_step_f32(const CUtensorMap& src, float* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, const float* corr,
                            int flip, cudaStream_t s);
cudaError_t launch_step_f16(const CUtensorMap& src, __half* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, const float* corr,
                            int flip, cudaStream_t s);
// Relative binary16 storage (LBMHD_FP16_REL): the 27 planes hold f_i - w_i (1 + 3 c_i . U) and g_i,
// and two more planes per row (kQ, kQ + 1) the velocity reference U_x, U_y of the cell that wrote
// them (binary16); usrc is a tensor map over the same copy with boxes {box_width(2), 2, 1}.
constexpr int kQRel = kQ + 2;
cudaError_t launch_step_f16rel(const CUtensorMap& src, const CUtensorMap& usrc, __half* dst, const StepGeom& g,
                               const StepCoef& c, int stencil, unsigned* err, cudaStream_t s);
// Rows per block for the grid and precision (one wave of resident blocks when possible).
int step_band_rows(int nx, int ny, int precision, int num_sms);
// Opt the step kernels in to their dynamic shared memory (once per process and device).
cudaError_t prepare_step_kernels();
#ifdef LBMHD_BOUNDS_CHECK
// Bounds-checking build: the step kernels' failed-check bits since the last call (cleared).
unsigned bounds_check_flags();
#endif

// Ensemble step (lbmhd_step.cu): the member table is packed on the host into
// ensemble_member_bytes(precision) * n bytes and copied to the device; work[i] = {member,
// strip x0, band start y0, band index}; queue == nullptr takes tiles by a static stride,
// otherwise from the zeroed atomic counter *queue.
size_t ensemble_member_bytes(int precision);
void pack_ensemble_members(int precision, int n, const CUtensorMap* maps, void* const* pops,
                           const StepGeom* geoms, const StepCoef* coefs, void* host_out);
cudaError_t launch_ensemble_step(int precision, int stencil, const void* members, const int4* work,
                                 int nwork, int parity, unsigned long long* queue, int grid,
                                 unsigned* err, cudaStream_t s);
int resident_step_blocks(int precision, int num_sms);

// Auxiliary kernels (lbmhd_aux.cu).  `precision` selects double / float / half storage (and the
// relative binary16 form, LBMHD_FP16_REL).
cudaError_t launch_init_eq(int precision, void* pops, const StepGeom& g, const double* rho,
                           const double* ux, const double* uy, const double* bx, const double* by,
                           cudaStream_t s);
cudaError_t launch_moments(int precision, const void* pops, const StepGeom& g, double* rho,
                           double* ux, double* uy, double* bx, double* by, cudaStream_t s);
cudaError_t launch_populations(int precision, const void* pops, const StepGeom& g, double* out,
                               cudaStream_t s);
// Diagnostics over the five moment fields (rho, ux, uy, bx, by, each nx*ny, contiguous):
// block partials into `partials` (kDiagBlocks x kDiagSlots doubles), then a single-block
// fixed-order reduction into out[kDiagSlots] (device).
constexpr int kDiagBlocks = 304;
constexpr int kDiagSlots = 11;  // 10 public values + instability flag
cudaError_t launch_diagnostics(const double* fields, int nx, int ny, double* partials,
                               double* out, cudaStream_t s);

// Analysis kernels (lbmhd_analysis.cu): r x r block mean, and the shell-summed energy spectra
// of a square n x n field set into device outputs e_kin[nbins], e_mag[nbins], using `work` of
// spectrum_work_bytes(n) bytes.
cudaError_t launch_block_mean(const double* in, int nx, int ny, int r, double* out, cudaStream_t s);
size_t spectrum_work_bytes(int n);
cudaError_t launch_energy_spectrum(const double* ux, const double* uy, const double* bx,
                                   const double* by, int n, int nbins, double* ek, double* em,
                                   void* work, cudaStream_t s);

// Learned closure (lbmhd_closure.cu): correction planes corr [4][ny][nx] (physical units) for
// the current populations of a square binary64 (precision 0) or binary32 (1) grid, in one launch
// of the fused tensor-core network kernel; *err is set if one of its waits times out.
int closure_num_params();
cudaError_t closure_correction(const lbmhd_closure_t* c, int precision, const void* pops, const StepGeom& g,
                               float* corr, unsigned* err, cudaStream_t s);
// Kernel attributes of the network kernels (shared-memory size); call outside stream capture.
cudaError_t prepare_closure_kernels();

const float* closure_device_params(const lbmhd_closure_t* c);
const float* closure_device_scales(const lbmhd_closure_t* c);
const unsigned char* closure_device_packed(const lbmhd_closure_t* c);
cudaStream_t closure_stream(const lbmhd_closure_t* c);

// Store a message for lbmhd_last_error(NULL) on the calling thread (lbmhd_api.cu).
void set_thread_error(const char* msg);

// Launch `kernel` with programmatic stream serialisation: its blocks may be scheduled while the
// previous kernel in the stream drains (dependants are released at that kernel's block exit);
// the kernel must wait (griddepcontrol.wait) before its first global-memory access.  After a
// copy or a memset the launch is ordered as usual.
template <typename K, typename... A>
cudaError_t launch_programmatic(K kernel, dim3 grid, int threads, size_t smem, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lbmhd_gpu
