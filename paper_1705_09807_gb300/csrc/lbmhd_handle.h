// The handle behind lbmhd_t (internal; shared by the host translation units).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>

#include "lbmhd.h"
#include "lbmhd_internal.cuh"

struct lbmhd {
  bool in_ensemble = false;       // stepped by an ensemble: lbmhd_step on it is refused
  lbmhd_params p{};
  int precision = 0;
  int device = 0;
  lbmhd_gpu::StepGeom geom{};
  lbmhd_gpu::StepCoef coef{};
  size_t elem = 8;         // bytes per stored population value
  int nplanes = 27;        // planes per row: 27 populations (+ 2 velocity-reference planes for
                           // LBMHD_FP16_REL)
  size_t state_bytes = 0;  // one population copy
  void* pops[2] = {nullptr, nullptr};
  int cur = 0;             // copy holding the current state
  double* fields = nullptr;    // 5 x nx*ny moment fields (moments / diagnostics)
  double* partials = nullptr;  // diagnostics block partials
  double* diag_out = nullptr;  // kDiagSlots results
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;  // ordering with the legacy default stream
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  long graph_launches = 0;  // kernel launches in one captured graph
  CUtensorMap tmap[2];             // 3-D TMA descriptors of the two copies
  CUtensorMap umap[2];             // LBMHD_FP16_REL: the same copies, boxes over the U planes
  unsigned* err_flag = nullptr;    // device word: set by the step kernel on a pipeline timeout
  void* spec_work = nullptr;       // spectrum work buffer and outputs (allocated on first use)
  const float* corr_static = nullptr;    // caller's correction planes [4][ny][nx] (not owned)
  struct lbmhd_closure* closure = nullptr;  // attached learned closure (not owned)
  float* cl_buf = nullptr;         // closure correction planes [4][ny][nx]
  uint64_t launches = 0;
  int64_t steps = 0;
  std::string err;
};

namespace lbmhd_gpu {
// Implemented in lbmhd_aux.cu: zero the row padding (columns outside the interior and the two
// ghost columns on each side) of both population copies, elements of `elem` bytes.
cudaError_t launch_zero_pads(void* pops0, void* pops1, const StepGeom& g, int nplanes, size_t elem,
                             cudaStream_t s);
// Implemented in lbmhd_api.cu.
int create_handle(lbmhd_t** out, const lbmhd_params* p);  // allocations, no initial state
void destroy_handle(lbmhd_t* h);
int handle_fail(lbmhd_t* h, int code, const char* fmt, ...);
}  // namespace lbmhd_gpu
