// Internal declarations shared by the translation units of liblbmhd.so.
//
// HBM layout of the population state (one copy; the handle holds two for ping-pong):
//   27 planes q = 0..8 (f_i), 9..17 (g_x,i), 18..26 (g_y,i), velocity order of the paper,
//   each plane ny rows of `pitch` elements (pitch = nx rounded up to 32 elements, so every row
//   starts on a 128-byte boundary for binary32 and 256-byte for binary64), x fastest.
//   The stored values are the POST-COLLISION populations f*_i(x), g*_i(x) of the last step;
//   the current (post-stream) populations are pulled: f_i(x) = f*_i(x - c_i), periodic.
//   f is stored as the deviation f_i - w_i from the rest state (rho = 1, u = 0), g as is.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace lbmhd_gpu {

constexpr int kQ = 27;           // populations per cell: 9 (f) + 2 x 9 (g)
constexpr int kStepThreads = 128;  // threads (= columns) per block of the fused step
constexpr int kRing = 4;         // rows of moments kept in shared memory

// Per-launch constants of the fused step, computed on the host in binary64.
struct StepCoef {
  double r[9];   // r[j] = s_j / |T_j|^2 for j = 3..8 (relaxation scaled by T T^T's diagonal)
  double s_m;    // magnetic rate
  double kq;     // Delta^2/12 times the squared scale of the undivided stencil differences
};

struct StepGeom {
  int nx, ny, pitch;  // grid and row pitch (elements)
  size_t plane;       // elements per plane = pitch * ny
  int band;           // rows per block
};

// Fused step launchers (lbmhd_step.cu).  src/dst are distinct population copies.
cudaError_t launch_step_f64(const double* src, double* dst, const StepGeom& g, const StepCoef& c,
                            int stencil, cudaStream_t s);
cudaError_t launch_step_f32(const float* src, float* dst, const StepGeom& g, const StepCoef& c,
                            int stencil, cudaStream_t s);
int step_band_rows(int nx, int ny, int precision, int num_sms);

// Auxiliary kernels (lbmhd_aux.cu).  `precision` selects double / float storage.
cudaError_t launch_init_eq(int precision, void* pops, const StepGeom& g, const double* rho,
                           const double* ux, const double* uy, const double* bx, const double* by,
                           cudaStream_t s);
cudaError_t launch_moments(int precision, const void* pops, const StepGeom& g, double* rho,
                           double* ux, double* uy, double* bx, double* by, cudaStream_t s);
cudaError_t launch_populations(int precision, const void* pops, const StepGeom& g, double* out,
                               cudaStream_t s);
// Diagnostics over the five moment fields (rho, ux, uy, bx, by, each nx*ny, contiguous):
// block partials into `partials` (nblocks x kDiagSlots doubles), then a single-block fixed-order
// reduction into out[kDiagSlots] (device).  Returns the number of blocks used via *nblocks.
constexpr int kDiagBlocks = 304;
constexpr int kDiagSlots = 11;  // 10 public values + instability flag
cudaError_t launch_diagnostics(const double* fields, int nx, int ny, double* partials,
                               double* out, cudaStream_t s);

// Store a message for lbmhd_last_error(NULL) on the calling thread (lbmhd_api.cu).
void set_thread_error(const char* msg);

}  // namespace lbmhd_gpu
