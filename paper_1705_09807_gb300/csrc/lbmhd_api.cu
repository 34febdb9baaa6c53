// Host side of the C ABI declared in include/lbmhd.h: argument checks, device memory,
// stream and graph management, and the launches.  Every function returns a status code;
// nothing throws across the ABI.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "lbmhd.h"
#include "lbmhd_handle.h"
#include "lbmhd_internal.cuh"

using namespace lbmhd_gpu;

namespace {

constexpr int kGraphSteps = 32;  // steps per captured graph (even: returns to the same buffer)

thread_local std::string g_tls_error;

}  // namespace

void lbmhd_gpu::set_thread_error(const char* msg) { g_tls_error = msg ? msg : ""; }


namespace {

int fail(lbmhd_t* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (h)
    h->err = buf;
  else
    g_tls_error = buf;
  return code;
}

int cuda_fail(lbmhd_t* h, cudaError_t e, const char* what) {
  return fail(h, e == cudaErrorMemoryAllocation ? LBMHD_ERR_OOM : LBMHD_ERR_CUDA, "%s: %s (%s)",
              what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define LB_CUDA(h, call)                              \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

int check_params(const lbmhd_params* p) {
  if (!p) return fail(nullptr, LBMHD_ERR_INVALID, "params is NULL");
  if (p->nx < 3 || p->ny < 3)
    return fail(nullptr, LBMHD_ERR_INVALID, "grid %d x %d: both sides must be >= 3", p->nx, p->ny);
  if ((long long)p->nx * p->ny > (1LL << 31))
    return fail(nullptr, LBMHD_ERR_INVALID, "grid %d x %d exceeds 2^31 cells", p->nx, p->ny);
  // the row stride (all 27 planes of one row -- 29 for LBMHD_FP16_REL -- ghost and pad columns
  // included) is an int
  const int planes = p->precision == LBMHD_FP16_REL ? kQRel : kQ;
  if ((long long)planes * (((long long)p->nx + kXOff + 2 + 31) / 32 * 32) > INT_MAX)
    return fail(nullptr, LBMHD_ERR_INVALID, "grid width %d too large: a row of all %d planes must "
                "hold fewer than 2^31 elements", p->nx, planes);
  for (int j = 3; j < 9; ++j)
    if (!(p->s[j] > 0.0 && p->s[j] < 2.0))
      return fail(nullptr, LBMHD_ERR_INVALID, "s[%d] = %g outside (0, 2)", j, p->s[j]);
  if (!(p->s_m > 0.0 && p->s_m < 2.0))
    return fail(nullptr, LBMHD_ERR_INVALID, "s_m = %g outside (0, 2)", p->s_m);
  if (!(p->delta >= 0.0) || !std::isfinite(p->delta))
    return fail(nullptr, LBMHD_ERR_INVALID, "delta = %g must be finite and >= 0", p->delta);
  if (p->precision != LBMHD_FP64 && p->precision != LBMHD_FP32 && p->precision != LBMHD_FP16 &&
      p->precision != LBMHD_FP16_REL)
    return fail(nullptr, LBMHD_ERR_INVALID, "unknown precision %d", p->precision);
  if (p->grad_stencil != LBMHD_GRAD_CENTRAL && p->grad_stencil != LBMHD_GRAD_ISOTROPIC)
    return fail(nullptr, LBMHD_ERR_INVALID, "unknown grad_stencil %d", p->grad_stencil);
  return LBMHD_OK;
}

void free_all(lbmhd_t* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) cudaGraphExecDestroy(h->graph[i]);
  for (int i = 0; i < 2; ++i)
    if (h->pops[i]) cudaFree(h->pops[i]);
  if (h->fields) cudaFree(h->fields);
  if (h->partials) cudaFree(h->partials);
  if (h->diag_out) cudaFree(h->diag_out);
  if (h->err_flag) cudaFree(h->err_flag);
  if (h->spec_work) cudaFree(h->spec_work);
  if (h->cl_buf) cudaFree(h->cl_buf);
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

// When the handle runs on its own stream, device arrays of the caller are ordered with the
// legacy default stream (where a caller without streams puts its work) at entry and exit.
int order_in(lbmhd_t* h) {
  if (!h->own_stream) return LBMHD_OK;
  LB_CUDA(h, cudaEventRecord(h->ev_a, cudaStreamLegacy));
  LB_CUDA(h, cudaStreamWaitEvent(h->stream, h->ev_a, 0));
  return LBMHD_OK;
}
int order_out(lbmhd_t* h) {
  if (!h->own_stream) return LBMHD_OK;
  LB_CUDA(h, cudaEventRecord(h->ev_b, h->stream));
  LB_CUDA(h, cudaStreamWaitEvent(cudaStreamLegacy, h->ev_b, 0));
  return LBMHD_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  });
  return fn;
}

// 3-D map {columns, 27 planes (29 for LBMHD_FP16_REL), ny rows} over one population copy,
// boxes of {box_width, box_planes, 1}: one row of one 9-plane group (the strip plus box_lead
// columns on each side), or of the two velocity-reference planes of the relative form.
int make_tensor_map(lbmhd_t* h, void* base, CUtensorMap* map, int box_planes = 9) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(nullptr, LBMHD_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t e = h->elem;
  cuuint64_t dims[3] = {(cuuint64_t)h->geom.plane, (cuuint64_t)h->nplanes, (cuuint64_t)h->geom.ny};
  cuuint64_t strides[2] = {(cuuint64_t)h->geom.plane * e, (cuuint64_t)h->geom.pitch * e};
  cuuint32_t box[3] = {(cuuint32_t)box_width((int)e), (cuuint32_t)box_planes, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  const CUtensorMapDataType dt = e == 8   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                 : e == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
  CUresult r = enc(map, dt, 3,
                   base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(nullptr, LBMHD_ERR_CUDA, "cuTensorMapEncodeTiled failed (CUresult %d)", (int)r);
  return LBMHD_OK;
}

// Device address of a host array of `bytes` bytes that kernels may write directly: the array
// lies entirely inside one page-locked allocation (cudaHostAlloc, cudaMallocHost,
// cudaHostRegister) that the current device maps.  nullptr otherwise -- pageable memory, or an
// extent that cannot be had -- and the caller stages through device memory instead.
void* mapped_host_array(const void* ptr, size_t bytes) {
  using PointerGetAttributeFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);
  static const PointerGetAttributeFn get = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &f, 4000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return static_cast<PointerGetAttributeFn>(nullptr);
    return reinterpret_cast<PointerGetAttributeFn>(f);
  }();
  if (!get || !ptr) return nullptr;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  const CUdeviceptr d = (CUdeviceptr)(uintptr_t)a.devicePointer;
  CUdeviceptr start = 0;
  size_t size = 0;
  if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, d) != CUDA_SUCCESS ||
      get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, d) != CUDA_SUCCESS)
    return nullptr;
  if (d < start || d - start > size || size - (d - start) < bytes) return nullptr;
  return a.devicePointer;
}

// The device moment-field buffer (5 x nx*ny binary64), allocated on the first call that stages
// through it: page-locked host arrays and the device entry points never need it.
int ensure_fields(lbmhd_t* h) {
  if (!h->fields) {
    cudaError_t e = cudaMalloc(&h->fields, 5 * (size_t)h->p.nx * h->p.ny * sizeof(double));
    if (e != cudaSuccess) {
      h->fields = nullptr;
      return cuda_fail(h, e, "allocating the moment-field buffer");
    }
  }
  return LBMHD_OK;
}

// Status of the step kernels' pipeline waits (call after synchronising the stream).
int check_step_status(lbmhd_t* h) {
  unsigned v = 0;
  LB_CUDA(h, cudaMemcpy(&v, h->err_flag, sizeof v, cudaMemcpyDeviceToHost));
  if (v) return fail(h, LBMHD_ERR_TIMEOUT, "a fused-step pipeline wait timed out; the state is invalid");
#ifdef LBMHD_BOUNDS_CHECK
  if (const unsigned bf = bounds_check_flags())
    return fail(h, LBMHD_ERR_INVALID, "bounds check failed in a step kernel (flags 0x%x)", bf);
#endif
  return LBMHD_OK;
}

// Handle with its device memory and tensor maps (no initial state).
int create(lbmhd_t** out, const lbmhd_params* p) {
  if (!out) return fail(nullptr, LBMHD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int rc = check_params(p);
  if (rc) return rc;
  lbmhd_t* h = new (std::nothrow) lbmhd();
  if (!h) return fail(nullptr, LBMHD_ERR_OOM, "host allocation failed");
  h->p = *p;
  h->precision = p->precision;
  h->elem = p->precision == LBMHD_FP64 ? 8 : (p->precision == LBMHD_FP32 ? 4 : 2);
  h->nplanes = p->precision == LBMHD_FP16_REL ? kQRel : kQ;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(nullptr, e, "cudaGetDevice");
  }
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  StepGeom& g = h->geom;
  g.nx = p->nx;
  g.ny = p->ny;
  g.plane = (p->nx + kXOff + 2 + 31) / 32 * 32;  // one row of one plane
  g.pitch = (int)(h->nplanes * g.plane);          // one row of all 27 (29) planes
  g.band = step_band_rows(p->nx, p->ny, p->precision, sms);
  // rates scaled by the diagonal of T T^T = (9, 6, 6, 4, 4, 12, 12, 180, 20) (Eq. FluidTMatrix)
  const double norm[9] = {9, 6, 6, 4, 4, 12, 12, 180, 20};
  for (int j = 0; j < 9; ++j) h->coef.r[j] = j < 3 ? 0.0 : p->s[j] / norm[j];
  h->coef.s_m = p->s_m;
  const double kd = p->delta * p->delta / 12.0;
  // undivided differences: central a(+1)-a(-1) = 2 d; isotropic 12 d
  h->coef.kq = p->grad_stencil == LBMHD_GRAD_ISOTROPIC ? kd / 144.0 : kd / 4.0;
  h->state_bytes = (size_t)g.pitch * p->ny * h->elem;
#define LB_INIT(call)                 \
  do {                                \
    cudaError_t e_ = (call);          \
    if (e_ != cudaSuccess) {          \
      int rc_ = cuda_fail(nullptr, e_, #call); \
      free_all(h);                    \
      return rc_;                     \
    }                                 \
  } while (0)
  if (p->cuda_stream) {
    h->stream = (cudaStream_t)p->cuda_stream;
  } else {
    LB_INIT(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  LB_INIT(cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming));
  LB_INIT(cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming));
  for (int i = 0; i < 2; ++i) LB_INIT(cudaMalloc(&h->pops[i], h->state_bytes));
  LB_INIT(cudaMalloc(&h->partials, (size_t)kDiagBlocks * kDiagSlots * sizeof(double)));
  LB_INIT(cudaMalloc(&h->diag_out, kDiagSlots * sizeof(double)));
  LB_INIT(cudaMalloc(&h->err_flag, sizeof(unsigned)));
  LB_INIT(cudaMemsetAsync(h->err_flag, 0, sizeof(unsigned), h->stream));
  LB_INIT(prepare_step_kernels());
  for (int i = 0; i < 2; ++i) {
    int rc_map = make_tensor_map(h, h->pops[i], &h->tmap[i]);
    if (!rc_map && h->precision == LBMHD_FP16_REL) rc_map = make_tensor_map(h, h->pops[i], &h->umap[i], 2);
    if (rc_map) {
      free_all(h);
      return rc_map;
    }
  }
  // zero the row padding once so checkpoints are deterministic (the interior and the ghost
  // columns are written by the initialisation in copy 0 and by the first step in copy 1)
  LB_INIT(launch_zero_pads(h->pops[0], h->pops[1], g, h->nplanes, h->elem, h->stream));
#undef LB_INIT
  *out = h;
  return LBMHD_OK;
}

// One fused step from copy `from` into copy `to` (with the subgrid correction planes `corr`,
// or none).  The bands' marching direction alternates with `from` (binary64 / binary32), so each
// band starts a step on the rows it wrote last, still in L2: at 2048^2 binary32 that cut the DRAM
// reads of a step from 471 MB to 427 MB (ncu without its L2 flush) and the time by 0.5%; the
// binary16 form, bound by latency rather than memory, ran 0.7% slower with it and keeps a fixed
// direction.
cudaError_t launch_one(lbmhd_t* h, int from, int to, const float* corr = nullptr) {
  switch (h->precision) {
    case LBMHD_FP64:
      return launch_step_f64(h->tmap[from], (double*)h->pops[to], h->geom, h->coef,
                             h->p.grad_stencil, h->err_flag, corr, from, h->stream);
    case LBMHD_FP32:
      return launch_step_f32(h->tmap[from], (float*)h->pops[to], h->geom, h->coef,
                             h->p.grad_stencil, h->err_flag, corr, from, h->stream);
    case LBMHD_FP16:
      return launch_step_f16(h->tmap[from], (__half*)h->pops[to], h->geom, h->coef,
                             h->p.grad_stencil, h->err_flag, corr, 0, h->stream);
    default:  // LBMHD_FP16_REL (no correction: refused when it is attached)
      return launch_step_f16rel(h->tmap[from], h->umap[from], (__half*)h->pops[to], h->geom, h->coef,
                                h->p.grad_stencil, h->err_flag, h->stream);
  }
}

// The launches of one step from copy `from` into copy `to`: with an attached learned closure,
// its network (correction of the current state) and the corrected step; with static correction
// planes, the corrected step; else the plain step.  *nlaunch receives the number of launches.
cudaError_t launch_step_seq(lbmhd_t* h, int from, int to, int* nlaunch) {
  *nlaunch = 1;
  if (h->closure) {
    cudaError_t e = closure_correction(h->closure, h->precision, h->pops[from], h->geom, h->cl_buf, h->err_flag,
                                       h->stream);
    if (e != cudaSuccess) return e;
    *nlaunch = 2;
    return launch_one(h, from, to, h->cl_buf);
  }
  return launch_one(h, from, to, h->corr_static);
}

// Captured graphs hold kernel arguments (geometry, correction planes, closure): drop them when
// any of those changes.
void drop_graphs(lbmhd_t* h) {
  for (int i = 0; i < 2; ++i)
    if (h->graph[i]) {
      cudaGraphExecDestroy(h->graph[i]);
      h->graph[i] = nullptr;
    }
}

int build_graph(lbmhd_t* h, int parity) {
  cudaGraph_t graph = nullptr;
  LB_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  int cur = parity;
  cudaError_t le = cudaSuccess;
  int per_step = 1;
  for (int n = 0; n < kGraphSteps && le == cudaSuccess; ++n) {
    const int nxt = cur ^ 1;
    le = launch_step_seq(h, cur, nxt, &per_step);
    cur = nxt;
  }
  h->graph_launches = kGraphSteps * per_step;
  cudaError_t ce = cudaStreamEndCapture(h->stream, &graph);
  if (le != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return cuda_fail(h, le, "capturing the step graph");
  }
  if (ce != cudaSuccess) return cuda_fail(h, ce, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(&h->graph[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    h->graph[parity] = nullptr;
    return cuda_fail(h, ie, "cudaGraphInstantiate");
  }
  return LBMHD_OK;
}

int one_step(lbmhd_t* h) {
  const int nxt = h->cur ^ 1;
  int nl = 1;
  cudaError_t e = launch_step_seq(h, h->cur, nxt, &nl);
  if (e != cudaSuccess) return cuda_fail(h, e, "fused step launch");
  h->cur = nxt;
  h->launches += nl;
  h->steps += 1;
  return LBMHD_OK;
}

int check_fields(const double* a, const double* b, const double* c, const double* d,
                 const double* e) {
  return a && b && c && d && e;
}

}  // namespace

int lbmhd_gpu::create_handle(lbmhd_t** out, const lbmhd_params* p) { return create(out, p); }
void lbmhd_gpu::destroy_handle(lbmhd_t* h) { free_all(h); }
int lbmhd_gpu::handle_fail(lbmhd_t* h, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  return fail(h, code, "%s", buf);
}

extern "C" {

int lbmhd_params_srt(lbmhd_params* p, int nx, int ny, double nu, double eta, double delta,
                     int precision) {
  if (!p) return fail(nullptr, LBMHD_ERR_INVALID, "params is NULL");
  if (!(nu > 0.0) || !(eta > 0.0))
    return fail(nullptr, LBMHD_ERR_INVALID, "nu = %g and eta = %g must be > 0", nu, eta);
  std::memset(p, 0, sizeof *p);
  p->nx = nx;
  p->ny = ny;
  const double s = 1.0 / (3.0 * nu + 0.5);
  for (int j = 0; j < 9; ++j) p->s[j] = s;
  p->s_m = 1.0 / (3.0 * eta + 0.5);
  p->delta = delta;
  p->precision = precision;
  p->grad_stencil = LBMHD_GRAD_CENTRAL;
  p->cuda_stream = nullptr;
  return LBMHD_OK;
}

int lbmhd_init(lbmhd_t** out, const lbmhd_params* p, const double* rho, const double* ux,
               const double* uy, const double* bx, const double* by) {
  if (!out) return fail(nullptr, LBMHD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!check_fields(rho, ux, uy, bx, by))
    return fail(nullptr, LBMHD_ERR_INVALID, "a field pointer is NULL");
  lbmhd_t* h = nullptr;
  int rc = create(&h, p);
  if (rc) return rc;
  const size_t ncell = (size_t)p->nx * p->ny;
  const double* src[5] = {rho, ux, uy, bx, by};
  const double* in[5];
  bool mapped = true;
  for (int k = 0; k < 5; ++k) {
    in[k] = static_cast<const double*>(mapped_host_array(src[k], ncell * sizeof(double)));
    mapped = mapped && in[k];
  }
  if (!mapped) {  // pageable fields: through the device field buffer; page-locked ones are read
                  // by the initialisation kernel directly over the host link
    rc = ensure_fields(h);
    if (rc) {
      g_tls_error = h->err;
      free_all(h);
      return rc;
    }
    for (int k = 0; k < 5; ++k) {
      in[k] = h->fields + k * ncell;
      cudaError_t e = cudaMemcpyAsync(h->fields + k * ncell, src[k], ncell * sizeof(double),
                                      cudaMemcpyHostToDevice, h->stream);
      if (e != cudaSuccess) {
        rc = cuda_fail(nullptr, e, "copying the initial fields to the device");
        free_all(h);
        return rc;
      }
    }
  }
  cudaError_t e = launch_init_eq(h->precision, h->pops[0], h->geom, in[0], in[1], in[2], in[3],
                                 in[4], h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    rc = cuda_fail(nullptr, e, "equilibrium initialisation");
    free_all(h);
    return rc;
  }
  h->launches += 1;
  *out = h;
  return LBMHD_OK;
}

int lbmhd_init_device(lbmhd_t** out, const lbmhd_params* p, const double* rho,
                      const double* ux, const double* uy, const double* bx, const double* by) {
  if (!out) return fail(nullptr, LBMHD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!check_fields(rho, ux, uy, bx, by))
    return fail(nullptr, LBMHD_ERR_INVALID, "a field pointer is NULL");
  lbmhd_t* h = nullptr;
  int rc = create(&h, p);
  if (rc) return rc;
  rc = order_in(h);
  cudaError_t e = cudaSuccess;
  if (!rc) e = launch_init_eq(h->precision, h->pops[0], h->geom, rho, ux, uy, bx, by, h->stream);
  if (!rc && e != cudaSuccess) rc = cuda_fail(h, e, "equilibrium initialisation");
  if (!rc) rc = order_out(h);
  if (rc) {
    g_tls_error = h->err;
    free_all(h);
    return rc;
  }
  h->launches += 1;
  *out = h;
  return LBMHD_OK;
}

int lbmhd_step(lbmhd_t* h, int nsteps) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (h->in_ensemble)
    return fail(h, LBMHD_ERR_INVALID, "this handle is an ensemble member: step the ensemble");
  if (nsteps < 0) return fail(h, LBMHD_ERR_INVALID, "nsteps = %d < 0", nsteps);
  int n = nsteps;
  // whole graphs of kGraphSteps steps when the handle owns its stream
  if (h->own_stream && n >= kGraphSteps) {
    if (!h->graph[h->cur]) {
      int rc = build_graph(h, h->cur);
      if (rc) return rc;
    }
    while (n >= kGraphSteps) {
      LB_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
      h->launches += h->graph_launches;
      h->steps += kGraphSteps;
      n -= kGraphSteps;  // kGraphSteps is even: h->cur is unchanged
    }
  }
  for (; n > 0; --n) {
    int rc = one_step(h);
    if (rc) return rc;
  }
  return LBMHD_OK;
}

int lbmhd_moments_device(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx,
                         double* by) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!check_fields(rho, ux, uy, bx, by)) return fail(h, LBMHD_ERR_INVALID, "a field pointer is NULL");
  int rc = order_in(h);
  if (rc) return rc;
  LB_CUDA(h, launch_moments(h->precision, h->pops[h->cur], h->geom, rho, ux, uy, bx, by, h->stream));
  h->launches += 1;
  return order_out(h);
}

int lbmhd_moments(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx, double* by) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!check_fields(rho, ux, uy, bx, by)) return fail(h, LBMHD_ERR_INVALID, "a field pointer is NULL");
  const size_t ncell = (size_t)h->p.nx * h->p.ny;
  double* dst[5] = {rho, ux, uy, bx, by};
  double* direct[5];
  bool mapped = true;
  for (int k = 0; k < 5; ++k) {
    direct[k] = static_cast<double*>(mapped_host_array(dst[k], ncell * sizeof(double)));
    mapped = mapped && direct[k];
  }
  if (mapped) {  // page-locked outputs: the read-out kernel writes them over the host link
    LB_CUDA(h, launch_moments(h->precision, h->pops[h->cur], h->geom, direct[0], direct[1],
                              direct[2], direct[3], direct[4], h->stream));
    h->launches += 1;
  } else {  // pageable outputs: through the device field buffer
    int rc = ensure_fields(h);
    if (rc) return rc;
    double* f = h->fields;
    LB_CUDA(h, launch_moments(h->precision, h->pops[h->cur], h->geom, f, f + ncell, f + 2 * ncell,
                              f + 3 * ncell, f + 4 * ncell, h->stream));
    h->launches += 1;
    for (int k = 0; k < 5; ++k)
      LB_CUDA(h, cudaMemcpyAsync(dst[k], f + k * ncell, ncell * sizeof(double),
                                 cudaMemcpyDeviceToHost, h->stream));
  }
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_step_status(h);
}

int lbmhd_get_populations(lbmhd_t* h, double* pops) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!pops) return fail(h, LBMHD_ERR_INVALID, "pops is NULL");
  const size_t n = (size_t)kQ * h->p.nx * h->p.ny;
  double* tmp = nullptr;
  LB_CUDA(h, cudaMallocAsync((void**)&tmp, n * sizeof(double), h->stream));
  cudaError_t e = launch_populations(h->precision, h->pops[h->cur], h->geom, tmp, h->stream);
  if (e == cudaSuccess) {
    h->launches += 1;
    e = cudaMemcpyAsync(pops, tmp, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
  }
  cudaError_t fe = cudaFreeAsync(tmp, h->stream);
  if (e == cudaSuccess) e = fe;
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "exporting populations");
  return check_step_status(h);
}

int lbmhd_diagnostics(lbmhd_t* h, double* out) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!out) return fail(h, LBMHD_ERR_INVALID, "out is NULL");
  const size_t ncell = (size_t)h->p.nx * h->p.ny;
  int frc = ensure_fields(h);
  if (frc) return frc;
  double* f = h->fields;
  LB_CUDA(h, launch_moments(h->precision, h->pops[h->cur], h->geom, f, f + ncell, f + 2 * ncell,
                            f + 3 * ncell, f + 4 * ncell, h->stream));
  LB_CUDA(h, launch_diagnostics(f, h->p.nx, h->p.ny, h->partials, h->diag_out, h->stream));
  h->launches += 3;
  double res[kDiagSlots];
  LB_CUDA(h, cudaMemcpyAsync(res, h->diag_out, sizeof res, cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  for (int k = 0; k < LBMHD_NDIAG; ++k) out[k] = res[k];
  int st = check_step_status(h);
  if (st) return st;
  if (res[LBMHD_NDIAG] != 0.0)
    return fail(h, LBMHD_ERR_UNSTABLE, "unstable state: NaN/Inf, rho <= 0 or |u| > 0.4 after %lld steps",
                (long long)h->steps);
  return LBMHD_OK;
}

int lbmhd_energy_spectrum(lbmhd_t* h, int nbins, double* e_kin, double* e_mag) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!e_kin || !e_mag) return fail(h, LBMHD_ERR_INVALID, "output pointer is NULL");
  const int n = h->p.nx;
  if (h->p.ny != n) return fail(h, LBMHD_ERR_INVALID, "spectra need a square grid");
  if (n > 4096) return fail(h, LBMHD_ERR_INVALID, "spectra are limited to n <= 4096");
  if (nbins < 1 || nbins > n) return fail(h, LBMHD_ERR_INVALID, "nbins must be in [1, n]");
  const size_t wb = spectrum_work_bytes(n);
  if (!h->spec_work) LB_CUDA(h, cudaMalloc(&h->spec_work, wb + 2 * (size_t)n * sizeof(double)));
  double* dk = reinterpret_cast<double*>(static_cast<char*>(h->spec_work) + wb);
  double* dm = dk + n;
  const size_t ncell = (size_t)n * n;
  int frc = ensure_fields(h);
  if (frc) return frc;
  double* f = h->fields;
  LB_CUDA(h, launch_moments(h->precision, h->pops[h->cur], h->geom, f, f + ncell, f + 2 * ncell,
                            f + 3 * ncell, f + 4 * ncell, h->stream));
  LB_CUDA(h, launch_energy_spectrum(f + ncell, f + 2 * ncell, f + 3 * ncell, f + 4 * ncell, n, nbins,
                                    dk, dm, h->spec_work, h->stream));
  h->launches += 5;
  LB_CUDA(h, cudaMemcpyAsync(e_kin, dk, nbins * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaMemcpyAsync(e_mag, dm, nbins * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_step_status(h);
}

int lbmhd_test_skip_row_copy(lbmhd_t* h, int enable) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (h->in_ensemble) return fail(h, LBMHD_ERR_INVALID, "not for ensemble members");
  h->geom.skip_copy = enable ? 1 : 0;
  drop_graphs(h);
  return LBMHD_OK;
}

int lbmhd_set_correction_device(lbmhd_t* h, const float* corr) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (corr && (h->precision == LBMHD_FP16 || h->precision == LBMHD_FP16_REL))
    return fail(h, LBMHD_ERR_INVALID, "the subgrid correction needs binary64 or binary32 storage");
  if (corr && h->closure) return fail(h, LBMHD_ERR_INVALID, "detach the learned closure first");
  h->corr_static = corr;
  drop_graphs(h);
  return LBMHD_OK;
}

int lbmhd_set_closure(lbmhd_t* h, lbmhd_closure_t* c) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (c) {
    if (h->precision == LBMHD_FP16 || h->precision == LBMHD_FP16_REL)
      return fail(h, LBMHD_ERR_INVALID, "the learned closure needs binary64 or binary32 storage");
    if (h->p.nx != h->p.ny) return fail(h, LBMHD_ERR_INVALID, "the learned closure needs a square grid");
    if (h->corr_static) return fail(h, LBMHD_ERR_INVALID, "detach the static correction first");
    if (!h->cl_buf) {
      const size_t mm = (size_t)h->p.nx * h->p.ny;
      LB_CUDA(h, cudaMalloc(&h->cl_buf, 4 * mm * sizeof(float)));
    }
    // the closure's parameters must be in place before this handle's stream reads them
    LB_CUDA(h, cudaStreamSynchronize(closure_stream(c)));
    LB_CUDA(h, prepare_closure_kernels());  // before any graph capture
  }
  h->closure = c;
  drop_graphs(h);
  return LBMHD_OK;
}

int lbmhd_closure_correction_device(lbmhd_t* h, float* corr) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!h->closure) return fail(h, LBMHD_ERR_INVALID, "no learned closure is attached");
  if (!corr) return fail(h, LBMHD_ERR_INVALID, "corr is NULL");
  int rc = order_in(h);
  if (rc) return rc;
  LB_CUDA(h, closure_correction(h->closure, h->precision, h->pops[h->cur], h->geom, corr, h->err_flag, h->stream));
  h->launches += 1;
  return order_out(h);
}

size_t lbmhd_state_bytes(const lbmhd_t* h) { return h ? h->state_bytes : 0; }

int lbmhd_get_state(lbmhd_t* h, void* host_buf, size_t bytes) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!host_buf || bytes != h->state_bytes)
    return fail(h, LBMHD_ERR_INVALID, "state buffer must be %zu bytes", h->state_bytes);
  LB_CUDA(h, cudaMemcpyAsync(host_buf, h->pops[h->cur], bytes, cudaMemcpyDeviceToHost, h->stream));
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  return check_step_status(h);
}

int lbmhd_set_state(lbmhd_t* h, const void* host_buf, size_t bytes) {
  if (!h) return fail(nullptr, LBMHD_ERR_INVALID, "handle is NULL");
  if (!host_buf || bytes != h->state_bytes)
    return fail(h, LBMHD_ERR_INVALID, "state buffer must be %zu bytes", h->state_bytes);
  LB_CUDA(h, cudaMemcpyAsync(h->pops[h->cur], host_buf, bytes, cudaMemcpyHostToDevice, h->stream));
  // a restored state is valid again: clear a pipeline-timeout status
  LB_CUDA(h, cudaMemsetAsync(h->err_flag, 0, sizeof(unsigned), h->stream));
  LB_CUDA(h, cudaStreamSynchronize(h->stream));
  h->steps = 0;
  return LBMHD_OK;
}

void* lbmhd_get_stream(const lbmhd_t* h) { return h ? (void*)h->stream : nullptr; }

uint64_t lbmhd_launch_count(const lbmhd_t* h) { return h ? h->launches : 0; }

int64_t lbmhd_step_count(const lbmhd_t* h) { return h ? h->steps : 0; }

const char* lbmhd_last_error(const lbmhd_t* h) {
  if (h) return h->err.c_str();
  return g_tls_error.c_str();
}

void lbmhd_free(lbmhd_t* h) {
  if (h && h->in_ensemble) return;  // owned by its ensemble
  free_all(h);
}

}  // extern "C"
