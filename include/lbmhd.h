/*
 * lbmhd.h - C ABI of the GB300 (sm_103a) fused time step of the filtered (large eddy)
 * lattice Boltzmann MHD model of Flint & Vahala, "A large eddy lattice Boltzmann
 * simulation of magnetohydrodynamic turbulence", arXiv:1705.09807.
 *
 * The model (Sec. 2, Eqs. LBKinEqn and LBMagEqn): a scalar D2Q9 distribution f_i carries
 * density and momentum, a vector D2Q9 distribution g_i (two components) carries the magnetic
 * field.  Moments rho = sum f_i, J = rho u = sum f_i c_i, B = sum g_i (Sec. 2).  One time step
 * collides in moment space (Eq. Transformation with the matrices T, T_m of Eqs. FluidTMatrix
 * and MagTMatrix) toward the filtered equilibrium moments of Sec. 2.1 / Sec. 3: the printed
 * tables Eq. KinMomentEq / MagMomentEq with every nonlinear product expanded to O(Delta^2)
 * by Eqs. FilterExampleSmall / FilterExampleLarge, filtered density gradients dropped (Sec. 3),
 * and then streams on a periodic nx x ny grid.  The gradients d_beta J, d_beta B the Delta^2
 * terms need are finite differences of the current moments.
 *
 * Conventions for every function:
 *  - Return 0 on success or a negative LBMHD_ERR_* code; no C++ exception crosses the ABI.
 *    lbmhd_last_error() gives a message.
 *  - Host arrays are owned by the caller and only read or written during the call.
 *    Device arrays (the *_device variants) are owned by the caller; the call enqueues work
 *    on the handle's stream and returns without synchronising.
 *  - Fields are row-major [ny][nx] arrays of double, x fastest.  Populations in canonical
 *    layout are [q][ny][nx] with q = 0..8 for f_i, 9..17 for g_x,i and 18..26 for g_y,i,
 *    in the paper's velocity order c_x = {0,1,0,-1,0,1,-1,-1,1}, c_y = {0,0,1,0,-1,1,1,-1,-1}.
 *  - The handle owns all its device memory; lbmhd_free releases it.  A handle may be used
 *    from one host thread at a time.
 */
#ifndef LBMHD_H
#define LBMHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBMHD_OK 0
#define LBMHD_ERR_INVALID (-1)  /* bad argument (checked on the host before any GPU work);
                                   in the bounds-checking build (liblbmhd_check.so, compiled
                                   with -DLBMHD_BOUNDS_CHECK) also a failed index check in a
                                   step kernel, reported by the next synchronising call */
#define LBMHD_ERR_CUDA (-2)     /* a CUDA runtime call failed (message has the CUDA error) */
#define LBMHD_ERR_OOM (-3)      /* device memory allocation failed */
#define LBMHD_ERR_UNSTABLE (-4) /* diagnostics found NaN/Inf, rho <= 0 or |u| > 0.4 */
#define LBMHD_ERR_TIMEOUT (-5)  /* a step kernel's pipeline wait ran out (reported by the next
                                   synchronising call; the state is then invalid) */

/* Storage / arithmetic forms of the populations. */
#define LBMHD_FP64 0 /* populations stored in binary64, collision in binary64 */
#define LBMHD_FP32 1 /* f_i - w_i and g_i stored in binary32, collision in binary32 */
#define LBMHD_FP16 2 /* f_i - w_i and g_i stored in binary16, collision in binary32 */
#define LBMHD_FP16_REL 3 /* binary16 storage relative to the local velocity: f_i - w_i (1 + 3 c_i . U)
                            and g_i, where U is the velocity of the cell that stored the value,
                            itself stored in binary16 in two more planes (116 instead of 108 bytes
                            per cell update); collision in binary32.  Removing the O(u) part of
                            f_i before rounding resolves the density fluctuation that LBMHD_FP16
                            rounds away.  Single grids only: ensembles, static corrections and
                            the learned closure take the other forms. */

/* Finite-difference stencils for d_beta (the paper leaves the discretisation open). */
#define LBMHD_GRAD_CENTRAL 0   /* (a(x+e_beta) - a(x-e_beta)) / 2 */
#define LBMHD_GRAD_ISOTROPIC 1 /* sum_i 3 w_i c_i,beta a(x + c_i) over the D2Q9 neighbours */

#define LBMHD_NDIAG 10

typedef struct lbmhd lbmhd_t; /* opaque handle */

/* Problem statement, as the paper states it (Sec. 2 and Sec. 3). */
typedef struct {
  int nx, ny;        /* periodic grid, each >= 3; nx * ny <= 2^31 and nx <= 79,536,382 (a row
                        of all 27 planes, 34 ghost/offset columns and padding to 32 included,
                        must hold fewer than 2^31 elements; 74,051,102 for the 29 planes of
                        LBMHD_FP16_REL); otherwise LBMHD_ERR_INVALID */
  double s[9];       /* fluid MRT rates s_j for the rows j of T (Eq. LBKinEqn); s[0..2] act
                        on conserved moments and are ignored; s[3..8] must lie in (0, 2).
                        nu = 1/(3 s_3) - 1/6 = 1/(3 s_4) - 1/6 and
                        xi = -1/9 - 1/(9 s_4) - 1/(15 s_7) + 2/(5 s_8) (Sec. 2).
                        The paper's runs are SRT: all s_j = 1/(3 nu + 1/2) (Sec. 3). */
  double s_m;        /* magnetic SRT rate (Eq. LBMagEqn), in (0, 2); eta = 1/(3 s_m) - 1/6 */
  double delta;      /* filter width Delta in lattice units, >= 0; the Delta^2/12 terms of
                        Sec. 2.1; 0 gives plain (DNS) LB-MHD */
  int precision;     /* LBMHD_FP64, LBMHD_FP32, LBMHD_FP16 or LBMHD_FP16_REL */
  int grad_stencil;  /* LBMHD_GRAD_CENTRAL or LBMHD_GRAD_ISOTROPIC */
  void* cuda_stream; /* cudaStream_t to run on; NULL: the handle creates its own stream */
} lbmhd_params;

/* Fill *p for the paper's SRT runs (Sec. 3): every s_j = 1/(3 nu + 1/2), s_m = 1/(3 eta + 1/2),
 * central gradients, no stream.  Returns LBMHD_ERR_INVALID for nu, eta <= 0 or a NULL p. */
int lbmhd_params_srt(lbmhd_params* p, int nx, int ny, double nu, double eta, double delta,
                     int precision);

/* Create a handle and set the populations to the equilibria Eq. feq and Eq. geq of the
 * given fields (rho, u = (ux, uy), B = (bx, by)), without Delta terms.  Host input arrays
 * [ny][nx], read before the call returns (the caller may reuse them afterwards); synchronises.
 * Arrays that lie wholly inside page-locked allocations (cudaHostAlloc, cudaMallocHost,
 * cudaHostRegister) are read by the initialisation kernel directly over the host link;
 * pageable ones are copied through a device buffer (5 x nx*ny doubles, allocated then and kept
 * by the handle).  The state is the same either way.  On error *out is NULL. */
int lbmhd_init(lbmhd_t** out, const lbmhd_params* p, const double* rho, const double* ux,
               const double* uy, const double* bx, const double* by);

/* Same as lbmhd_init with device input arrays [ny][nx] (e.g. torch tensors); the
 * equilibrium kernel runs on the handle's stream, ordered after earlier work on it. */
int lbmhd_init_device(lbmhd_t** out, const lbmhd_params* p, const double* rho,
                      const double* ux, const double* uy, const double* bx, const double* by);

/* Advance nsteps >= 0 time steps (one step = collide, then stream; Sec. 3).  Each step is one
 * launch of the fused kernel: pull-stream the 27 populations, form rho, J, B and their
 * gradients, build the filtered equilibria, relax (Eq. LBKinEqn / LBMagEqn in moment space),
 * store.  Enqueued on the handle's stream; returns without synchronising.  The step kernels
 * are programmatic dependent launches: their blocks may be scheduled while the previous kernel
 * on the stream finishes, but they touch no global memory before it has completed, so the
 * stream's order holds for all work before and after them.  A wait that runs out in a step
 * (2 s) is reported as LBMHD_ERR_TIMEOUT by the next synchronising call. */
int lbmhd_step(lbmhd_t* h, int nsteps);

/* Macroscopic fields of the current (post-stream, pre-collision) populations: rho,
 * u = J/rho, B.  Host output arrays [ny][nx]; synchronises.  Arrays that lie wholly inside
 * page-locked allocations are written by the read-out kernel directly over the host link;
 * otherwise the fields go through a device buffer (allocated on first use, kept by the handle)
 * and a copy.  The values are the same either way.  For FP32 / FP16 handles the sums are exact
 * binary32 pair sums (rho and B to binary64 rounding) and u takes one binary32 division. */
int lbmhd_moments(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx, double* by);

/* Same as lbmhd_moments into device arrays [ny][nx]; asynchronous on the handle's stream. */
int lbmhd_moments_device(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx,
                         double* by);

/* Current populations in canonical layout [27][ny][nx] (binary64), host array of
 * 27*nx*ny doubles; synchronises.  For FP32 / FP16 handles the stored values are widened. */
int lbmhd_get_populations(lbmhd_t* h, double* pops);

/* Double-precision diagnostics of the current state (host array of LBMHD_NDIAG):
 * [0] sum rho  [1] sum J_x  [2] sum J_y  [3] sum B_x  [4] sum B_y
 * [5] sum rho |u|^2 / 2  [6] sum |B|^2 / 2  [7] max |div B| (isotropic stencil)
 * [8] max |div B| (central stencil)  [9] max |d_beta B_alpha| (isotropic stencil).
 * Sums are reduced in a fixed order (bitwise reproducible).  Synchronises; the moment fields
 * go through the handle's device buffer (allocated on first use).  Returns
 * LBMHD_ERR_UNSTABLE (with out[] filled) if any cell has a NaN/Inf, rho <= 0 or |u| > 0.4. */
int lbmhd_diagnostics(lbmhd_t* h, double* out);

/* ---- Filtered-DNS vs LES comparison tools (off the time-step path) ---------------------
 *
 * Box filter: out = the r x r block means of `in` (a device [ny][nx] array; r divides nx and
 * ny; out is [ny/r][nx/r]) -- the top-hat filter of width r (Sec. 1, Eq. VelFilter, whose second
 * moment is the Delta^2/12 of Sec. 2.1 with Delta = r) followed by downsampling.  Asynchronous
 * on `stream` (NULL: legacy default stream).  LBMHD_ERR_INVALID if r does not divide the grid. */
int lbmhd_block_mean_device(const double* in, int nx, int ny, int r, double* out, void* stream);

/* Shell-summed energy spectra of square n x n device fields (u_x, u_y, B_x, B_y):
 *   a^(k) = n^-2 sum_x a(x) exp(-2 pi i k.x/n),  E_kin(s) = 1/2 sum_{k in s} |u_x^|^2 + |u_y^|^2,
 *   E_mag(s) likewise with B; shell s = the integer wavevectors with (2s-1)^2 < 4|k|^2 < (2s+1)^2.
 * e_kin, e_mag: device arrays of nbins (1 <= nbins <= n); n <= 4096.  `work` is a caller device
 * buffer of at least lbmhd_energy_spectrum_work_bytes(n) bytes.  Bitwise reproducible;
 * asynchronous on `stream`. */
size_t lbmhd_energy_spectrum_work_bytes(int n);
int lbmhd_energy_spectrum_device(const double* ux, const double* uy, const double* bx,
                                 const double* by, int n, int nbins, double* e_kin, double* e_mag,
                                 void* work, size_t work_bytes, void* stream);

/* The same spectra of a handle's current state (square grid), into host arrays of nbins;
 * allocates its work buffer on first use; synchronises. */
int lbmhd_energy_spectrum(lbmhd_t* h, int nbins, double* e_kin, double* e_mag);

/* ---- Ensembles: many independent runs, one launch per time step -------------------------
 *
 * An ensemble owns n member runs (each its own grid size, rates and filter width; all with the
 * same precision and gradient stencil) and advances all of them with ONE kernel launch per time
 * step: the launch walks a work list of tiles (member, 128-column strip, band of rows), either
 * one block per tile or persistent blocks taking tiles from an atomic counter.  With an
 * ensemble-owned stream, whole groups of 32 steps are replayed from a captured CUDA graph.
 * Members are ordinary handles for every read-out call (moments, populations, diagnostics,
 * spectra, checkpoints); lbmhd_step on a member is refused and lbmhd_free on it is a no-op.
 *
 * fields: 5*n host pointers, rho, ux, uy, bx, by of member 0, then member 1, ... ([ny][nx] each,
 * copied).  cuda_stream: NULL = the ensemble creates its own stream (and uses graphs). */
typedef struct lbmhd_ensemble lbmhd_ensemble_t;
int lbmhd_ensemble_create(lbmhd_ensemble_t** out, int n, const lbmhd_params* params,
                          const double* const* fields, void* cuda_stream);
/* Advance every member by nsteps (asynchronous on the ensemble's stream). */
int lbmhd_ensemble_step(lbmhd_ensemble_t* e, int nsteps);
/* Tile schedule: rows_per_tile = 0 gives each member its one-wave band height; persistent = 1
 * launches one resident wave of blocks that take tiles from an atomic counter. */
int lbmhd_ensemble_set_schedule(lbmhd_ensemble_t* e, int rows_per_tile, int persistent);
int lbmhd_ensemble_get_schedule(const lbmhd_ensemble_t* e, int* rows_per_tile, int* persistent,
                                int* nwork, int* grid);
/* Autotuner: times trial_steps steps of each candidate schedule (rows per tile in {one-wave,
 * 8, 16, 32, 64, 128, 256} x {one block per tile, persistent}), keeps the fastest, and restores
 * every member's state and step count.  *best_ms (may be NULL) receives its time per step. */
int lbmhd_ensemble_autotune(lbmhd_ensemble_t* e, int trial_steps, double* best_ms);
/* Wait for the ensemble's stream; LBMHD_ERR_TIMEOUT if a pipeline wait ran out. */
int lbmhd_ensemble_sync(lbmhd_ensemble_t* e);
/* Member i as a handle for read-out calls (borrowed; valid until lbmhd_ensemble_free). */
lbmhd_t* lbmhd_ensemble_member(lbmhd_ensemble_t* e, int i);
int lbmhd_ensemble_size(const lbmhd_ensemble_t* e);
void* lbmhd_ensemble_get_stream(const lbmhd_ensemble_t* e);
uint64_t lbmhd_ensemble_launch_count(const lbmhd_ensemble_t* e);
const char* lbmhd_ensemble_last_error(const lbmhd_ensemble_t* e);
void lbmhd_ensemble_free(lbmhd_ensemble_t* e);

/* ---- Subgrid correction and the learned closure ------------------------------------------
 *
 * The collision's filtered equilibria carry four subgrid terms (Sec. 2.1 / Sec. 3): the xy
 * stress in M_3 (c0), the normal-stress difference in M_4 (c1), the trace in M_7 and M_8 (c2,
 * entering as -3 c2) and the electric field E of N^eq (c3).  The analytic closure gives each as
 * Delta^2/12 times gradient products; a correction adds c0..c3 per cell on top of it.
 *
 * lbmhd_set_correction_device: a static correction, binary32 device planes corr[4][ny][nx]
 * (caller-owned, read at every step; NULL detaches).  Binary64 / binary32 storage only. */
int lbmhd_set_correction_device(lbmhd_t* h, const float* corr);

/* The learned closure: a periodic 3x3 convolutional network 12 -> 32 -> 32 -> 4 channels (tanh
 * after the first two layers; 13,892 binary32 parameters: per layer W[co][ci][dy+1][dx+1] then
 * b[co]) mapping 12 features of the state -- u_x, u_y, B_x, B_y and their central differences
 * d_x, d_y, each divided by in_scale[k] -- to the residual of the four subgrid terms with
 * respect to the analytic closure, divided by out_scale[k].  Trained on box-filtered fine runs
 * by the library's own binary32 forward / back-propagation / Adam kernels; applied with bf16
 * operands on the tensor cores (binary32 accumulation). */
typedef struct lbmhd_closure lbmhd_closure_t;
int lbmhd_closure_num_params(void);
int lbmhd_closure_create(lbmhd_closure_t** out, const float* params, const float* in_scale,
                         const float* out_scale);
int lbmhd_closure_get_params(lbmhd_closure_t* c, float* params);
int lbmhd_closure_set_params(lbmhd_closure_t* c, const float* params);
/* Training pair from a fine state: fine = device binary64 planes rho, ux, uy, bx, by [n][n];
 * box filter r (r | n); x = features [12][n/r][n/r], t = targets [4][n/r][n/r] (device
 * binary32): t = (exact filtered subgrid term - analytic closure with filter width delta, in
 * coarse lattice units) / out_scale.  work: device buffer of 9 (n/r)^2 doubles. Synchronises. */
int lbmhd_closure_training_pair(lbmhd_closure_t* c, const double* fine, int n, int r, double delta,
                                float* x, float* t, double* work);
/* Features (and optionally the analytic closure, 4 planes, physical units) of a coarse state
 * given as device binary64 planes rho, ux, uy, bx, by [m][m].  Synchronises. */
int lbmhd_closure_features(lbmhd_closure_t* c, const double* state, int m, double delta, float* x,
                           float* analytic);
/* x: device [batch][12][h][w]; t: [batch][4][h][w]; mean-squared-error loss / 2.
 * gradient: loss and the flat parameter gradient (host, may be NULL); train_step: one Adam step
 * (beta1 0.9, beta2 0.999, eps 1e-8) with learning rate lr.  Both synchronise. */
int lbmhd_closure_gradient(lbmhd_closure_t* c, const float* x, const float* t, int batch, int h,
                           int w, float* grad, double* loss);
int lbmhd_closure_train_step(lbmhd_closure_t* c, const float* x, const float* t, int batch, int h,
                             int w, float lr, double* loss);
/* Network output (scaled units) for device features x into out [batch][4][h][w]:
 * tensor_cores = 1 runs the fused bf16 tcgen05 kernel (all three layers in one launch, fp32
 * accumulation in tensor memory), 0 the binary32 layer-by-layer kernels.  Synchronises;
 * LBMHD_ERR_TIMEOUT if a tensor-core completion wait of the fused kernel ran out (2 s). */
int lbmhd_closure_forward(lbmhd_closure_t* c, const float* x, int batch, int h, int w, float* out,
                          int tensor_cores);
/* Failure-detection test hook of the tensor-core forward pass.  With enable = 1, every
 * following lbmhd_closure_forward(..., tensor_cores = 1) leaves out the first tile's layer-1
 * MMAs and their commit in each CTA, so the time-bounded completion wait (2 s) runs out: the
 * kernel stops without a GPU fault, frees its tensor memory and the call returns
 * LBMHD_ERR_TIMEOUT (its output is then invalid).  enable = 0 restores normal calls; steps of
 * handles the closure is attached to are not affected.  For tests of the error path only. */
int lbmhd_closure_test_skip_mma(lbmhd_closure_t* c, int enable);
const char* lbmhd_closure_last_error(const lbmhd_closure_t* c);
void lbmhd_closure_free(lbmhd_closure_t* c);
/* Attach a closure to a square binary64 / binary32 handle (NULL detaches): every step then runs
 * two launches, the fused network kernel (pull of the populations, u and B and the features in
 * binary32, the three tcgen05 layers, output scale -> correction planes) and the corrected fused
 * step; on the handle's own stream whole groups of 32 steps run as one CUDA graph.  The closure
 * must outlive the attachment and must not be trained while attached. */
int lbmhd_set_closure(lbmhd_t* h, lbmhd_closure_t* c);

/* The correction planes that the attached closure gives the CURRENT state (what the next step
 * would add: the fused network kernel of lbmhd_set_closure, run on its own), into the caller's
 * device array corr [4][ny][nx] binary32 (xy stress, normal-stress difference, trace, electric
 * field; physical units).  For inspecting or testing the learned correction; the state does not
 * change.  Enqueued on the handle's stream (ordered with the legacy default stream when the
 * handle owns its stream); LBMHD_ERR_INVALID without an attached closure or with corr NULL.  A
 * wait that runs out in the network kernel is reported by the next synchronising call. */
int lbmhd_closure_correction_device(lbmhd_t* h, float* corr);

/* Failure-detection test hook.  With enable = 1, the first block of every following step
 * leaves out one of its staged-row copies, so its time-bounded wait (2 s) runs out: the block
 * records a timeout, drains its other copies and stops, no GPU fault occurs, and the next
 * synchronising call returns LBMHD_ERR_TIMEOUT.  enable = 0 restores normal steps;
 * lbmhd_set_state clears the timeout status.  For tests of the error path only. */
int lbmhd_test_skip_row_copy(lbmhd_t* h, int enable);

/* Size in bytes of a checkpoint of this handle's state. */
size_t lbmhd_state_bytes(const lbmhd_t* h);

/* Copy the raw population state to / from a host buffer of exactly lbmhd_state_bytes(h)
 * bytes (checkpoint / resume; restoring and stepping reproduces the run bitwise).  The
 * format is the handle's storage (precision, row pitch); restore only into a handle made
 * with the same nx, ny and precision.  Both synchronise; set_state also clears a pipeline-timeout
 * status (LBMHD_ERR_TIMEOUT), since the restored state is valid. */
int lbmhd_get_state(lbmhd_t* h, void* host_buf, size_t bytes);
int lbmhd_set_state(lbmhd_t* h, const void* host_buf, size_t bytes);

/* The CUDA stream the handle enqueues its work on (the caller's, or the one it created), as a
 * cudaStream_t cast to void*; lets a caller record events on it or order other work after it.
 * NULL for a NULL handle. */
void* lbmhd_get_stream(const lbmhd_t* h);

/* Number of GPU kernels this handle has launched so far (all kinds). */
uint64_t lbmhd_launch_count(const lbmhd_t* h);

/* Number of time steps taken since init (or since the last set_state). */
int64_t lbmhd_step_count(const lbmhd_t* h);

/* Diagnostics of moment fields that the caller already holds on the device, for callers that
 * cannot allocate device memory: code that must take every byte from another framework's pool
 * or arena, code under a fixed memory budget that forbids allocations after start-up, or code
 * on a path where an allocation would synchronise the device.  The paper has no counterpart;
 * this is an interface convenience of this library.
 *
 * Inputs: rho, ux, uy, bx, by, device arrays [ny][nx] (e.g. from lbmhd_moments_device).
 * Output: out, a device array of LBMHD_NDIAG + 1 doubles: the LBMHD_NDIAG values of
 * lbmhd_diagnostics, then 1.0 if any cell has NaN/Inf, rho <= 0 or |u| > 0.4, else 0.0.
 * Enqueued on `stream` (a cudaStream_t; NULL = the legacy default stream); no synchronisation.
 *
 * It calls no cudaMalloc/cudaFree or other allocating routine: its scratch (one partial record
 * per 4096 cells) is a fixed 352 KiB device array of the library, resident on every GPU that
 * loads the library until the process exits.  Hence at most 4096 x 4096 = 16,777,216 cells;
 * larger grids, sides < 3 and NULL pointers return LBMHD_ERR_INVALID (see lbmhd_last_error(NULL)).
 * The first call in a device's context looks up that array's device address (with the device
 * current) and keeps it for that context; make that first call before any stream capture.  A
 * call in a new context of the same device (after cudaDeviceReset, say) looks it up again,
 * so the first call after such a reset must also come before any capture.  All calls share the one
 * array, so calls that overlap on the GPU (different streams, no ordering) race and may return
 * wrong values; each call overwrites every record it reads, so nothing needs clearing. */
int lbmhd_diagnostics_fields_noalloc(const double* rho, const double* ux, const double* uy,
                                     const double* bx, const double* by, int nx, int ny,
                                     double* out, void* stream);

/* Measured binary64 FMA rate of the current device, the arithmetic ceiling of the LBMHD_FP64
 * step (about 216 binary64 instructions per cell update; the paper states no precision or
 * hardware, so this is a property of the GPU that runs it, not of the method).  Three shapes --
 * 4, 8 and 16 independent chains x <- x a + b per thread, (SMs x 16, 8, 4) blocks of 256
 * threads, `iters` iterations -- each one warm-up launch and `repeats` timed launches;
 * *dfma_per_second = the fastest shape's DFMAs per launch / its median CUDA-event time (one
 * DFMA = 2 flops).  Allocates a small device buffer and a stream
 * for the call and frees them; synchronises.  iters in [1, 2^20], repeats in [1, 100], else
 * LBMHD_ERR_INVALID; CUDA failures return LBMHD_ERR_CUDA (message: lbmhd_last_error(NULL)). */
int lbmhd_probe_fp64_fma_rate(int iters, int repeats, double* dfma_per_second);

/* Message for the last error on h, or for the calling thread's last handle-less call when
 * h is NULL.  Never NULL; valid until the next call on the same handle / thread. */
const char* lbmhd_last_error(const lbmhd_t* h);

/* Release the handle and its device memory (waits for its stream).  NULL is a no-op. */
void lbmhd_free(lbmhd_t* h);

#ifdef __cplusplus
}
#endif

#endif /* LBMHD_H */
