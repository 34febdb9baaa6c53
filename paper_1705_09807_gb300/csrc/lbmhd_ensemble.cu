// Ensembles of independent runs advanced together: one kernel launch per time step covers every
// member (grids of any size), tile by tile from a work list; K steps are captured in a CUDA
// graph.  An autotuner picks the tile height and the scheduling (one block per tile, or
// persistent blocks taking tiles from an atomic counter) by timing candidate schedules.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbmhd.h"
#include "lbmhd_handle.h"
#include "lbmhd_internal.cuh"

using namespace lbmhd_gpu;

namespace {
constexpr int kEnsGraphSteps = 32;  // even: the parity returns to its start
thread_local std::string g_ens_tls_error;
}  // namespace

struct lbmhd_ensemble {
  int n = 0;
  int precision = 0;
  int stencil = 0;
  int num_sms = 152;
  std::vector<lbmhd_t*> members;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* d_members = nullptr;       // packed member table
  int4* d_work = nullptr;          // work list
  int work_capacity = 0;
  int nwork = 0;
  int rows_per_tile = 0;           // 0: each member's one-wave band
  int persistent = 0;
  int grid = 0;
  unsigned long long* d_queue = nullptr;
  unsigned* d_err = nullptr;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  uint64_t launches = 0;
  int64_t steps = 0;
  std::string err;
};

namespace {

int efail(lbmhd_ensemble_t* e, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (e)
    e->err = buf;
  else
    g_ens_tls_error = buf;
  return code;
}

#define ENS_CUDA(e, call)                                                                    \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return efail(e, e_ == cudaErrorMemoryAllocation ? LBMHD_ERR_OOM : LBMHD_ERR_CUDA, "%s: %s", \
                   #call, cudaGetErrorString(e_));                                           \
  } while (0)

void drop_graphs(lbmhd_ensemble_t* e) {
  for (int i = 0; i < 2; ++i)
    if (e->graph[i]) {
      cudaGraphExecDestroy(e->graph[i]);
      e->graph[i] = nullptr;
    }
}

void destroy(lbmhd_ensemble_t* e) {
  if (!e) return;
  if (e->stream) cudaStreamSynchronize(e->stream);
  drop_graphs(e);
  for (lbmhd_t* m : e->members) {
    if (!m) continue;
    m->in_ensemble = false;
    destroy_handle(m);
  }
  if (e->d_members) cudaFree(e->d_members);
  if (e->d_work) cudaFree(e->d_work);
  if (e->d_queue) cudaFree(e->d_queue);
  if (e->d_err) cudaFree(e->d_err);
  if (e->own_stream && e->stream) cudaStreamDestroy(e->stream);
  delete e;
}

// Work list for a schedule: tiles of every member, largest members first, band by band.
int build_work(lbmhd_ensemble_t* e, int rows_per_tile, int persistent) {
  std::vector<int> order(e->n);
  for (int i = 0; i < e->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (long)e->members[a]->p.nx * e->members[a]->p.ny > (long)e->members[b]->p.nx * e->members[b]->p.ny;
  });
  std::vector<int4> work;
  std::vector<StepGeom> geoms(e->n);
  for (int i : order) {
    StepGeom g = e->members[i]->geom;
    g.skip_copy = 0;
    g.band = rows_per_tile > 0 ? std::min(rows_per_tile, g.ny)
                               : step_band_rows(g.nx, g.ny, e->precision, e->num_sms);
    if (g.band < 1) g.band = 1;
    geoms[i] = g;
    for (int y0 = 0, b = 0; y0 < g.ny; y0 += g.band, ++b)
      for (int x0 = 0; x0 < g.nx; x0 += kStepThreads) work.push_back(make_int4(i, x0, y0, b));
  }
  // the member table carries each member's band
  std::vector<CUtensorMap> maps(2 * e->n);
  std::vector<void*> pops(2 * e->n);
  std::vector<StepCoef> coefs(e->n);
  for (int i = 0; i < e->n; ++i) {
    maps[2 * i] = e->members[i]->tmap[0];
    maps[2 * i + 1] = e->members[i]->tmap[1];
    pops[2 * i] = e->members[i]->pops[0];
    pops[2 * i + 1] = e->members[i]->pops[1];
    coefs[i] = e->members[i]->coef;
  }
  const size_t mbytes = ensemble_member_bytes(e->precision) * e->n;
  std::vector<unsigned char> host(mbytes + 64);
  void* aligned = host.data() + ((64 - (reinterpret_cast<uintptr_t>(host.data()) & 63)) & 63);
  pack_ensemble_members(e->precision, e->n, maps.data(), pops.data(), geoms.data(), coefs.data(),
                        aligned);
  if (!e->d_members) ENS_CUDA(e, cudaMalloc(&e->d_members, mbytes));
  ENS_CUDA(e, cudaMemcpyAsync(e->d_members, aligned, mbytes, cudaMemcpyHostToDevice, e->stream));
  if ((int)work.size() > e->work_capacity) {
    if (e->d_work) ENS_CUDA(e, cudaFree(e->d_work));
    e->d_work = nullptr;
    ENS_CUDA(e, cudaMalloc(&e->d_work, work.size() * sizeof(int4)));
    e->work_capacity = (int)work.size();
  }
  ENS_CUDA(e, cudaMemcpyAsync(e->d_work, work.data(), work.size() * sizeof(int4),
                              cudaMemcpyHostToDevice, e->stream));
  ENS_CUDA(e, cudaStreamSynchronize(e->stream));  // host vectors go out of scope
  e->nwork = (int)work.size();
  e->rows_per_tile = rows_per_tile;
  e->persistent = persistent;
  const int resident = resident_step_blocks(e->precision, e->num_sms);
  e->grid = persistent ? std::min(e->nwork, resident) : e->nwork;
  drop_graphs(e);
  return LBMHD_OK;
}

int launch_one(lbmhd_ensemble_t* e, int parity) {
  if (e->persistent) ENS_CUDA(e, cudaMemsetAsync(e->d_queue, 0, sizeof(unsigned long long), e->stream));
  ENS_CUDA(e, launch_ensemble_step(e->precision, e->stencil, e->d_members, e->d_work, e->nwork, parity,
                                   e->persistent ? e->d_queue : nullptr, e->grid, e->d_err, e->stream));
  return LBMHD_OK;
}

int build_graph(lbmhd_ensemble_t* e, int parity) {
  cudaGraph_t graph = nullptr;
  ENS_CUDA(e, cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal));
  int rc = LBMHD_OK;
  for (int k = 0; k < kEnsGraphSteps && rc == LBMHD_OK; ++k) rc = launch_one(e, parity ^ (k & 1));
  cudaError_t ce = cudaStreamEndCapture(e->stream, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (ce != cudaSuccess) return efail(e, LBMHD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ce));
  cudaError_t ie = cudaGraphInstantiate(&e->graph[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    e->graph[parity] = nullptr;
    return efail(e, LBMHD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ie));
  }
  return LBMHD_OK;
}

void advance_members(lbmhd_ensemble_t* e, int nsteps) {
  for (lbmhd_t* m : e->members) {
    if (nsteps & 1) m->cur ^= 1;
    m->steps += nsteps;
  }
  e->steps += nsteps;
}

int step_impl(lbmhd_ensemble_t* e, int nsteps) {
  const int parity0 = e->members[0]->cur;
  for (lbmhd_t* m : e->members)
    if (m->cur != parity0)
      return efail(e, LBMHD_ERR_INVALID, "ensemble members are out of step (a member was stepped alone?)");
  int n = nsteps;
  if (e->own_stream && n >= kEnsGraphSteps) {
    if (!e->graph[parity0]) {
      int rc = build_graph(e, parity0);
      if (rc) return rc;
    }
    while (n >= kEnsGraphSteps) {
      ENS_CUDA(e, cudaGraphLaunch(e->graph[parity0], e->stream));
      e->launches += kEnsGraphSteps;
      n -= kEnsGraphSteps;
    }
  }
  int parity = parity0;
  for (; n > 0; --n) {
    int rc = launch_one(e, parity);
    if (rc) return rc;
    e->launches += 1;
    parity ^= 1;
  }
  advance_members(e, nsteps);
  return LBMHD_OK;
}

}  // namespace

extern "C" {

int lbmhd_ensemble_create(lbmhd_ensemble_t** out, int n, const lbmhd_params* params,
                          const double* const* fields, void* cuda_stream) {
  if (!out) return efail(nullptr, LBMHD_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (n < 1 || !params || !fields) return efail(nullptr, LBMHD_ERR_INVALID, "need n >= 1 members");
  for (int i = 0; i < n; ++i) {
    if (params[i].precision != params[0].precision || params[i].grad_stencil != params[0].grad_stencil)
      return efail(nullptr, LBMHD_ERR_INVALID, "members must share precision and gradient stencil");
    if (params[i].precision == LBMHD_FP16_REL)
      return efail(nullptr, LBMHD_ERR_INVALID, "ensembles take LBMHD_FP64, LBMHD_FP32 or LBMHD_FP16 members");
    for (int k = 0; k < 5; ++k)
      if (!fields[5 * i + k]) return efail(nullptr, LBMHD_ERR_INVALID, "member %d: field pointer NULL", i);
  }
  lbmhd_ensemble_t* e = new (std::nothrow) lbmhd_ensemble();
  if (!e) return efail(nullptr, LBMHD_ERR_OOM, "host allocation failed");
  e->n = n;
  e->precision = params[0].precision;
  e->stencil = params[0].grad_stencil;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t ce;
  if (cuda_stream) {
    e->stream = static_cast<cudaStream_t>(cuda_stream);
  } else if ((ce = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking)) != cudaSuccess) {
    delete e;
    return efail(nullptr, LBMHD_ERR_CUDA, "stream: %s", cudaGetErrorString(ce));
  } else {
    e->own_stream = true;
  }
  for (int i = 0; i < n; ++i) {
    lbmhd_params p = params[i];
    p.cuda_stream = e->stream;
    lbmhd_t* h = nullptr;
    int rc = lbmhd_init(&h, &p, fields[5 * i], fields[5 * i + 1], fields[5 * i + 2], fields[5 * i + 3],
                        fields[5 * i + 4]);
    if (rc) {
      int r2 = efail(nullptr, rc, "member %d: %s", i, lbmhd_last_error(nullptr));
      destroy(e);
      return r2;
    }
    h->in_ensemble = true;
    e->members.push_back(h);
  }
  int rc = LBMHD_OK;
  if ((ce = cudaMalloc(&e->d_queue, sizeof(unsigned long long))) != cudaSuccess ||
      (ce = cudaMalloc(&e->d_err, sizeof(unsigned))) != cudaSuccess ||
      (ce = cudaMemsetAsync(e->d_err, 0, sizeof(unsigned), e->stream)) != cudaSuccess)
    rc = efail(nullptr, LBMHD_ERR_CUDA, "ensemble buffers: %s", cudaGetErrorString(ce));
  if (!rc) rc = build_work(e, 0, 0);
  if (rc) {
    if (!e->err.empty()) g_ens_tls_error = e->err;
    destroy(e);
    return rc;
  }
  *out = e;
  return LBMHD_OK;
}

int lbmhd_ensemble_set_schedule(lbmhd_ensemble_t* e, int rows_per_tile, int persistent) {
  if (!e) return efail(nullptr, LBMHD_ERR_INVALID, "ensemble is NULL");
  if (rows_per_tile < 0) return efail(e, LBMHD_ERR_INVALID, "rows_per_tile must be >= 0");
  return build_work(e, rows_per_tile, persistent ? 1 : 0);
}

int lbmhd_ensemble_get_schedule(const lbmhd_ensemble_t* e, int* rows_per_tile, int* persistent,
                                int* nwork, int* grid) {
  if (!e) return efail(nullptr, LBMHD_ERR_INVALID, "ensemble is NULL");
  if (rows_per_tile) *rows_per_tile = e->rows_per_tile;
  if (persistent) *persistent = e->persistent;
  if (nwork) *nwork = e->nwork;
  if (grid) *grid = e->grid;
  return LBMHD_OK;
}

int lbmhd_ensemble_step(lbmhd_ensemble_t* e, int nsteps) {
  if (!e) return efail(nullptr, LBMHD_ERR_INVALID, "ensemble is NULL");
  if (nsteps < 0) return efail(e, LBMHD_ERR_INVALID, "nsteps < 0");
  return step_impl(e, nsteps);
}

int lbmhd_ensemble_autotune(lbmhd_ensemble_t* e, int trial_steps, double* best_ms) {
  if (!e) return efail(nullptr, LBMHD_ERR_INVALID, "ensemble is NULL");
  if (trial_steps < 1) return efail(e, LBMHD_ERR_INVALID, "trial_steps must be >= 1");
  // keep every member's state: copy the current buffers aside, restore them afterwards
  std::vector<void*> backup(e->n, nullptr);
  int rc = LBMHD_OK;
  for (int i = 0; i < e->n && !rc; ++i) {
    lbmhd_t* m = e->members[i];
    cudaError_t ce = cudaMallocAsync(&backup[i], m->state_bytes, e->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(backup[i], m->pops[m->cur], m->state_bytes, cudaMemcpyDeviceToDevice, e->stream);
    if (ce != cudaSuccess) rc = efail(e, LBMHD_ERR_CUDA, "autotune backup: %s", cudaGetErrorString(ce));
  }
  const int parity0 = e->members[0]->cur;
  const int64_t steps0 = e->steps;
  std::vector<int64_t> msteps(e->n);
  for (int i = 0; i < e->n; ++i) msteps[i] = e->members[i]->steps;
  const int candidates_rows[] = {0, 8, 16, 32, 64, 128, 256};
  double best = 1e300;
  int best_rows = 0, best_pers = 0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (!rc && (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess))
    rc = efail(e, LBMHD_ERR_CUDA, "events");
  for (int rows : candidates_rows) {
    for (int pers = 0; pers < 2 && !rc; ++pers) {
      rc = build_work(e, rows, pers);
      if (!rc) rc = step_impl(e, 2);  // warm-up
      if (rc) break;
      cudaEventRecord(a, e->stream);
      rc = step_impl(e, trial_steps);
      cudaEventRecord(b, e->stream);
      if (rc) break;
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) {
        best = ms;
        best_rows = rows;
        best_pers = pers;
      }
    }
    if (rc) break;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  // restore the states, the parity and the counters
  for (int i = 0; i < e->n; ++i) {
    lbmhd_t* m = e->members[i];
    m->cur = parity0;
    m->steps = msteps[i];
    if (backup[i]) {
      cudaMemcpyAsync(m->pops[parity0], backup[i], m->state_bytes, cudaMemcpyDeviceToDevice, e->stream);
      cudaFreeAsync(backup[i], e->stream);
    }
  }
  e->steps = steps0;
  if (!rc) rc = build_work(e, best_rows, best_pers);
  if (!rc) ENS_CUDA(e, cudaStreamSynchronize(e->stream));
  unsigned errv = 0;
  if (!rc) ENS_CUDA(e, cudaMemcpy(&errv, e->d_err, sizeof errv, cudaMemcpyDeviceToHost));
  if (!rc && errv) rc = efail(e, LBMHD_ERR_TIMEOUT, "a pipeline wait timed out during tuning");
  if (!rc && best_ms) *best_ms = best / trial_steps;
  return rc;
}

int lbmhd_ensemble_sync(lbmhd_ensemble_t* e) {
  if (!e) return efail(nullptr, LBMHD_ERR_INVALID, "ensemble is NULL");
  ENS_CUDA(e, cudaStreamSynchronize(e->stream));
  unsigned errv = 0;
  ENS_CUDA(e, cudaMemcpy(&errv, e->d_err, sizeof errv, cudaMemcpyDeviceToHost));
  if (errv) return efail(e, LBMHD_ERR_TIMEOUT, "a pipeline wait timed out; the states are invalid");
#ifdef LBMHD_BOUNDS_CHECK
  if (const unsigned bf = bounds_check_flags())
    return efail(e, LBMHD_ERR_INVALID, "bounds check failed in a step kernel (flags 0x%x)", bf);
#endif
  return LBMHD_OK;
}

lbmhd_t* lbmhd_ensemble_member(lbmhd_ensemble_t* e, int i) {
  if (!e || i < 0 || i >= e->n) return nullptr;
  return e->members[i];
}

int lbmhd_ensemble_size(const lbmhd_ensemble_t* e) { return e ? e->n : 0; }

void* lbmhd_ensemble_get_stream(const lbmhd_ensemble_t* e) { return e ? (void*)e->stream : nullptr; }

uint64_t lbmhd_ensemble_launch_count(const lbmhd_ensemble_t* e) { return e ? e->launches : 0; }

const char* lbmhd_ensemble_last_error(const lbmhd_ensemble_t* e) {
  return e ? e->err.c_str() : g_ens_tls_error.c_str();
}

void lbmhd_ensemble_free(lbmhd_ensemble_t* e) { destroy(e); }

}  // extern "C"
