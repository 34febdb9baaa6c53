// Fused time step of the filtered LES lattice Boltzmann MHD model (Flint & Vahala,
// arXiv:1705.09807): one launch per step, all of
//   pull-stream -> moments -> gradients -> filtered equilibria -> relax -> store
// on the GPU with each population read once from HBM and written once.
//
// Work decomposition.  A block owns a strip of kStepThreads adjacent columns and a band of
// rows; each thread owns one column (binary16 storage: two adjacent columns, whose arithmetic
// runs in packed binary32 pairs, see run_tile_pair) and the block marches through the band row
// by row (adjacent bands march in opposite directions, so the two rows a band shares with its
// neighbour are fetched by both at about the same time and the second fetch hits L2).
// Rows are staged in shared memory by the tensor-memory accelerator: one elected thread
// issues, per pulled row r, three 3-D box copies (cp.async.bulk.tensor) of 9 planes x the strip
// columns each -- source rows r-1, r, r+1 of the three plane groups (planes are grouped by
// c_y, see lbmhd_internal.cuh) -- completing on the row's mbarrier, NST-2 rows ahead of the
// row whose moments are being formed.  For row r the block then
//   A. waits for row r+1, forms its moments (cell and the two halo columns) into a 4-row
//      ring of J, B in shared memory;
//   B. one CTA barrier; the elected thread refills the stage freed by row r-1;
//   C. takes x- and y-differences of J, B from the ring, collides row r from its stage and
//      stores 27 coalesced values (plus the ghost columns at the grid's x edges).
// Every mbarrier wait is bounded in time; on a timeout the block reports through *err,
// drains its outstanding copies (bounded) and stops.
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
#include <cstdlib>
#include <mutex>

#include "lbmhd_internal.cuh"
#include "lbmhd_ptx.cuh"

namespace lbmhd_gpu {
namespace {

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s per mbarrier wait

// Index checks of the bounds-checking build (-DLBMHD_BOUNDS_CHECK, a stand-in for a memory
// checker): LB_IN(cond, bit) is true in the normal build; in the checking build a false cond sets
// `bit` in g_bounds_flags (0: staged-row column, 1: moment-ring extent, 2: global store, 3: copy
// coordinates) and the caller skips the access.  The bits of g_bounds_force (environment
// variable LBMHD_BOUNDS_FORCE, read when the kernels are prepared) fail their checks whatever
// cond says, so that a test can see the skip-and-report path work.
#ifdef LBMHD_BOUNDS_CHECK
__device__ unsigned g_bounds_flags;
__device__ unsigned g_bounds_force;
#define LB_IN(cond, bit) \
  (((cond) && !((g_bounds_force >> (bit)) & 1u)) || (atomicOr(&g_bounds_flags, 1u << (bit)), false))
#else
#define LB_IN(cond, bit) true
#endif

template <typename T>
struct KCoef {
  T r3, r4, r5, r6, r7, r8, sm, kq;
};

// Collision of one cell; p[] holds the pulled (current) populations with f as deviations
// f_i - w_i, and receives the post-collision values.  rho1 = rho - 1.  dJ = undivided
// differences {dx Jx, dy Jx, dx Jy, dy Jy}, dB likewise; c.kq folds in their scale.
template <typename T, bool CORR = false>
__device__ __forceinline__ void collide(T p[kQ], T rho1, T jx, T jy, T bx, T by, const T dJ[4],
                                        const T dB[4], const KCoef<T>& c, const T* cq = nullptr) {
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
  T E = (jx * by - jy * bx + k * (Kxy - Kyx)) * ir;
  // optional additive correction of the four subgrid terms (xy stress, normal-stress
  // difference, trace, electric field), e.g. from the learned closure
  T c0 = T(0), c1 = T(0), c2 = T(0);
  if (CORR) {
    c0 = cq[0];
    c1 = cq[1];
    c2 = cq[2];
    E += cq[3];
  }

  // ---- fluid: non-equilibrium parts of moments 3..8 (rows of Eq. FluidTMatrix) ----
  const T a13 = p[1] + p[3], a24 = p[2] + p[4], a57 = p[5] + p[7], a68 = p[6] + p[8];
  const T qq = CORR ? (Qxx + Qyy) + c2 : Qxx + Qyy;
  const T n3 = CORR ? (a57 - a68) - ((Qxy - Rxy) + c0) : (a57 - a68) - (Qxy - Rxy);
  const T n4 = CORR ? (a13 - a24) - (((Qxx - Qyy) - (Rxx - Ryy)) + c1)
                    : (a13 - a24) - ((Qxx - Qyy) - (Rxx - Ryy));
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


// ---- packed binary32 pairs (two cells per thread, binary16 storage) ---------------------------
// Blackwell executes add / sub / mul / fma on two binary32 lanes held in a 64-bit register pair
// as one instruction (PTX .f32x2, round to nearest on each lane).  F2 holds (cell a, cell b).
struct F2 {
  uint64_t v;
};
__device__ __forceinline__ F2 f2(float a, float b) {
  F2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r.v) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ F2 f2(float a) { return f2(a, a); }
__device__ __forceinline__ float lo(F2 x) { return __uint_as_float((uint32_t)x.v); }
__device__ __forceinline__ float hi(F2 x) { return __uint_as_float((uint32_t)(x.v >> 32)); }
__device__ __forceinline__ F2 operator+(F2 a, F2 b) {
  F2 r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator-(F2 a, F2 b) {
  F2 r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
__device__ __forceinline__ F2 operator*(F2 a, F2 b) {
  F2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r.v) : "l"(a.v), "l"(b.v));
  return r;
}
// a * b + c, one rounding per lane
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) {
  F2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r.v) : "l"(a.v), "l"(b.v), "l"(c.v));
  return r;
}

struct KCoef2 {
  F2 r3, r4, r5, r6, r7, r8, sm, kq;
};
__device__ __forceinline__ KCoef2 pair_coef(const KCoef<float>& c) {
  return {f2(c.r3), f2(c.r4), f2(c.r5), f2(c.r6), f2(c.r7), f2(c.r8), f2(c.sm), f2(c.kq)};
}

// `collide` for two cells at once (same equations and operation order per lane, with the
// products that the scalar form leaves to the compiler's contraction written as fma).
__device__ __forceinline__ void collide_pair(F2 p[kQ], F2 rho1, F2 jx, F2 jy, F2 bx, F2 by, const F2 dJ[4],
                                             const F2 dB[4], const KCoef2& c, F2* ir_out = nullptr) {
  const F2 one = f2(1.f), two = f2(2.f), three = f2(3.f), four = f2(4.f), five = f2(5.f);
  const F2 r = one + rho1;
  const F2 ir = f2(1.f / lo(r), 1.f / hi(r));
  if (ir_out) *ir_out = ir;
  const F2 k = c.kq;
  const F2 Gxx = fma2(dJ[1], dJ[1], dJ[0] * dJ[0]);
  const F2 Gyy = fma2(dJ[3], dJ[3], dJ[2] * dJ[2]);
  const F2 Gxy = fma2(dJ[1], dJ[3], dJ[0] * dJ[2]);
  const F2 Hxx = fma2(dB[1], dB[1], dB[0] * dB[0]);
  const F2 Hyy = fma2(dB[3], dB[3], dB[2] * dB[2]);
  const F2 Hxy = fma2(dB[1], dB[3], dB[0] * dB[2]);
  const F2 Kxy = fma2(dJ[1], dB[3], dJ[0] * dB[2]);
  const F2 Kyx = fma2(dJ[3], dB[1], dJ[2] * dB[0]);
  const F2 Qxx = fma2(k, Gxx, jx * jx) * ir;
  const F2 Qyy = fma2(k, Gyy, jy * jy) * ir;
  const F2 Qxy = fma2(k, Gxy, jx * jy) * ir;
  const F2 Rxx = fma2(k, Hxx, bx * bx);
  const F2 Ryy = fma2(k, Hyy, by * by);
  const F2 Rxy = fma2(k, Hxy, bx * by);
  const F2 E = fma2(k, Kxy - Kyx, jx * by - jy * bx) * ir;

  const F2 a13 = p[1] + p[3], a24 = p[2] + p[4], a57 = p[5] + p[7], a68 = p[6] + p[8];
  const F2 qq = Qxx + Qyy;
  const F2 n3 = (a57 - a68) - (Qxy - Rxy);
  const F2 n4 = (a13 - a24) - ((Qxx - Qyy) - (Rxx - Ryy));
  const F2 n5 = fma2(two, p[3] - p[1], (p[5] - p[6]) + (p[8] - p[7])) + jx;
  const F2 n6 = fma2(two, p[4] - p[2], (p[5] - p[8]) + (p[6] - p[7])) + jy;
  const F2 n7 = fma2(three, qq, fma2(four, a57 + a68, fma2(four, p[0], f2(-5.f) * (a13 + a24))));
  const F2 n8 = fma2(three, qq, fma2(f2(-5.f / 3.f), rho1, four * p[0] - (a57 + a68)));
  const F2 d3 = c.r3 * n3, d4 = c.r4 * n4, d5 = c.r5 * n5, d6 = c.r6 * n6, d7 = c.r7 * n7, d8 = c.r8 * n8;
  const F2 e78 = fma2(f2(-4.f), d7, d8);
  p[0] = fma2(f2(-4.f), d7 + d8, p[0]);
  const F2 u = five * d7 - d4, w = fma2(five, d7, d4);
  p[1] = p[1] + fma2(two, d5, u);
  p[3] = p[3] + fma2(f2(-2.f), d5, u);
  p[2] = p[2] + fma2(two, d6, w);
  p[4] = p[4] + fma2(f2(-2.f), d6, w);
  p[5] = p[5] + (e78 - ((d3 + d5) + d6));
  p[6] = p[6] + (e78 + ((d3 + d5) - d6));
  p[7] = p[7] + (e78 + ((d5 + d6) - d3));
  p[8] = p[8] + (e78 + ((d3 + d6) - d5));

  const F2 sm = c.sm;
  const F2 e3 = three * E;
  const F2 wa = f2(1.f / 9.f), wd = f2(1.f / 36.f);
  {
    const F2 bm = bx - e3, bp = bx + e3;
    const F2 ea = wa * bx, em = wa * bm, ep = wa * bp, dm = wd * bm, dp = wd * bp;
    const F2 e0 = bx - (((ea + ea) + (em + ep)) + ((dm + dm) + (dp + dp)));
    p[9] = fma2(sm, e0 - p[9], p[9]);
    p[10] = fma2(sm, ea - p[10], p[10]);
    p[11] = fma2(sm, em - p[11], p[11]);
    p[12] = fma2(sm, ea - p[12], p[12]);
    p[13] = fma2(sm, ep - p[13], p[13]);
    p[14] = fma2(sm, dm - p[14], p[14]);
    p[15] = fma2(sm, dm - p[15], p[15]);
    p[16] = fma2(sm, dp - p[16], p[16]);
    p[17] = fma2(sm, dp - p[17], p[17]);
  }
  {
    const F2 bp = by + e3, bm = by - e3;
    const F2 ea = wa * by, ep = wa * bp, em = wa * bm, dp = wd * bp, dm = wd * bm;
    const F2 e0 = by - (((ea + ea) + (em + ep)) + ((dm + dm) + (dp + dp)));
    p[18] = fma2(sm, e0 - p[18], p[18]);
    p[19] = fma2(sm, ep - p[19], p[19]);
    p[20] = fma2(sm, ea - p[20], p[20]);
    p[21] = fma2(sm, em - p[21], p[21]);
    p[22] = fma2(sm, ea - p[22], p[22]);
    p[23] = fma2(sm, dp - p[23], p[23]);
    p[24] = fma2(sm, dm - p[24], p[24]);
    p[25] = fma2(sm, dm - p[25], p[25]);
    p[26] = fma2(sm, dp - p[26], p[26]);
  }
}

// Arithmetic type for each storage type: binary16 populations are collided in binary32.
template <typename S> struct ArithOf { using type = S; };
template <> struct ArithOf<__half> { using type = float; };

// Binary16 storage relative to the local velocity (LBMHD_FP16_REL): the velocity references
// U_x, U_y of kURing staged source rows ([row][component][box column]), indexed by march index.
// Rows in use at once: the collision of row m reads m-1 .. m+1, the moments of row m+1 read
// m .. m+2, and the copy issued in the same iteration brings m+3 (NST = 3): five, so six slots.
// Each ring row is the destination of one tensor copy ({BW columns, 2 planes}: U_x at [0, BW),
// U_y at [BW, 2 BW)), which must start on a 128-byte boundary in shared memory, so rows are
// padded to a multiple of 128 bytes (576 -> 640 B at BW = 144).
constexpr int kURing = 6;
__host__ __device__ constexpr int urow_elems(int bw) { return (2 * bw * 2 + 127) / 128 * 128 / 2; }
template <bool REL, int BW> struct URingSmem {};
template <int BW> struct URingSmem<true, BW> {
  static_assert(urow_elems(BW) * 2 % 128 == 0 && urow_elems(BW) >= 2 * BW, "U rows on 128-byte boundaries");
  __half uring[kURing][urow_elems(BW)];  // 3840 B at BW = 144
};

// Shared memory of one block: NST row stages, the moment ring, the stage barriers (and, for the
// relative binary16 form, the U ring, first: 3840 B, a multiple of 128, so the stages stay
// 128-byte aligned).
template <typename S, int NST, bool REL = false>
struct StepSmem : URingSmem<REL, box_width((int)sizeof(S))> {
  using C = typename ArithOf<S>::type;
  static constexpr int kNst = NST;
  static constexpr int kLead = box_lead((int)sizeof(S));
  static constexpr int kBoxW = box_width((int)sizeof(S));
  static constexpr int kGroupElems = ((9 * kBoxW * (int)sizeof(S) + 127) / 128 * 128) / (int)sizeof(S);
  static constexpr int kStageElems = 3 * kGroupElems;
  static constexpr uint32_t kTxBytes = 3u * 9u * kBoxW * sizeof(S);  // bytes landing per stage
  // moment ring row: the strip's columns plus one halo column each side; binary16 (two cells
  // per thread) keeps the strip at an even offset (column c at c + 2) so a cell pair is 8-byte
  // aligned
  static constexpr int kRingW = sizeof(S) == 2 ? kStepThreads + 4 : kStepThreads + 2;
  static constexpr int kRingOff = sizeof(S) == 2 ? 2 : 1;  // ring index of strip column 0
  S stage[NST][kStageElems];
  C ring[kRing][4][kRingW];
  uint64_t full[NST];
  int abort_flag[2];
};

// Store the 27 post-collision values of one cell, planes in address order through one advancing
// pointer (fewer address instructions than 27 independent 64-bit plane offsets).
template <typename S, typename T, int PL>
__device__ __forceinline__ void store_planes(S* op, const T* p, size_t plane, const S* lo, const S* hi) {
  if constexpr (PL < kQ) {
    constexpr int q = q_of_plane(PL);
    if (LB_IN(op >= lo && op < hi, 2)) *op = store_as<S>(p[q]);
    store_planes<S, T, PL + 1>(op + plane, p, plane, lo, hi);
  }
}

// Pulled population q of the cell at box column `col` of a staged row.
template <typename C, typename S, int BW>
__device__ __forceinline__ C staged(const S* st, int ge, int q, int col) {
  const int i = q % 9;
  const int c = col - vel_x(i);
  if (!LB_IN(c >= 0 && c < BW, 0)) return C(0);
  return load_as<C>(st[group_of(i) * ge + (3 * (q / 9) + index_in_group(i)) * BW + c]);
}

template <typename C, typename S, int BW>
__device__ __forceinline__ void moments_from(const S* st, int ge, int col, C& rho1, C& jx, C& jy,
                                             C& bx, C& by) {
  auto v = [&](int q) -> C { return staged<C, S, BW>(st, ge, q, col); };
  const C f0 = v(0), f1 = v(1), f2 = v(2), f3 = v(3), f4 = v(4), f5 = v(5), f6 = v(6), f7 = v(7),
          f8 = v(8);
  rho1 = ((f0 + f1) + (f2 + f3)) + ((f4 + f5) + (f6 + f7)) + f8;
  jx = (f1 - f3) + (f5 - f6) + (f8 - f7);
  jy = (f2 - f4) + (f5 - f8) + (f6 - f7);
  bx = ((v(9) + v(10)) + (v(11) + v(12))) + ((v(13) + v(14)) + (v(15) + v(16))) + v(17);
  by = ((v(18) + v(19)) + (v(20) + v(21))) + ((v(22) + v(23)) + (v(24) + v(25))) + v(26);
}

// Dynamic shared memory of a step block, rounded up to the 128-byte alignment TMA needs.
template <typename S, int NST, bool REL = false>
__device__ __forceinline__ StepSmem<S, NST, REL>& step_smem() {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  return *reinterpret_cast<StepSmem<S, NST, REL>*>(smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u));
}

template <typename SM>
__device__ __forceinline__ void init_stage_barriers(SM& S_, const CUtensorMap* prefetch,
                                                    const CUtensorMap* prefetch2 = nullptr) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < SM::kNst; ++s) mbar_init(&S_.full[s], 1);
    fence_barrier_init();
    if (prefetch) prefetch_tmap(prefetch);
    if (prefetch2) prefetch_tmap(prefetch2);
  }
}

// The three boxes of staged row r (groups c_y = +1, 0, -1 from rows ra, r, rc) into one stage.
// The first two rows a band stages are also the first two of the neighbouring band that marches
// the other way: `keep` asks L2 to keep their lines (evict_last) for that second reader.
// Measured: 2048^2 binary32 1.6% and binary16 0.8% less time per step (DRAM reads of a warm
// binary32 step 1% lower), 4096^2, binary64 and 256^2 unchanged; the same hint on the last two
// rows instead helped less (binary32 1.0%, binary16 none), and streaming (evict_first) the
// other rows made every form slower (binary32 15% more time, DRAM reads 470 -> 518 MB per step:
// neighbouring strips then re-read their overlapping box columns from DRAM).
template <typename S>
__device__ __forceinline__ void copy_row_boxes(S* stage, int ge, const CUtensorMap* srcp, int cx, int ra, int r, int rc,
                                               uint64_t* bar, bool keep) {
  if (keep) {
    const uint64_t pol = l2_policy_evict_last();
    tma_load_3d_hint(stage, srcp, cx, 0, ra, bar, pol);
    tma_load_3d_hint(stage + ge, srcp, cx, 9, r, bar, pol);
    tma_load_3d_hint(stage + 2 * ge, srcp, cx, 18, rc, bar, pol);
  } else {
    tma_load_3d(stage, srcp, cx, 0, ra, bar);
    tma_load_3d(stage + ge, srcp, cx, 9, r, bar);
    tma_load_3d(stage + 2 * ge, srcp, cx, 18, rc, bar);
  }
}

// One tile: the strip of kStepThreads columns starting at x0 and the band of rows [y0, y0 + band)
// of one grid, marched in direction +1 (band_parity even) or -1 (odd).  `kbase` counts the rows
// this block has staged before this tile, so stage slots and mbarrier phases continue across
// tiles.  Returns false if a wait timed out (the block must stop; *err is set).
template <typename S, int ISO, int NST, bool CORR = false>
__device__ __forceinline__ bool run_tile(const CUtensorMap* srcp, S* __restrict__ dst, const StepGeom& g,
                                         const KCoef<typename ArithOf<S>::type>& c, int x0, int y0,
                                         int band_parity, uint32_t& kbase, unsigned* __restrict__ err,
                                         const float* __restrict__ corr = nullptr) {
  using SM = StepSmem<S, NST>;
  using T = typename SM::C;
  constexpr int GE = SM::kGroupElems;
  constexpr int LEAD = SM::kLead;
  constexpr int BW = SM::kBoxW;
  SM& S_ = step_smem<S, NST>();

  static_assert(SM::kRingOff == 1, "one cell per thread: strip column c at ring index c + 1");
  const int t = threadIdx.x;
  const int nx = g.nx, ny = g.ny;
  const int ncol = min(kStepThreads, nx - x0);
  const bool active = t < ncol;
  // the ring holds columns -1 .. ncol at indices 0 .. ncol + 1 (uniform over the block)
  if (!LB_IN(ncol >= 1 && ncol + 1 < SM::kRingW, 1)) return true;
  const int y1 = min(y0 + g.band, ny);
  const int L = (y1 - y0) + 2;  // rows staged: the band and one on each side
  const int dir = (band_parity & 1) ? -1 : 1;
  const uint32_t kb = kbase;
  // k-th row in march order (k = 0 and L-1 are the neighbours' rows)
  auto row_of = [&](int k) -> int {
    int r = dir > 0 ? y0 - 1 + k : y1 - k;
    if (r < 0) r += ny;
    if (r >= ny) r -= ny;
    return r;
  };
  auto issue = [&](int k) {
    if (g.skip_copy && k == 2 && blockIdx.x == 0 && blockIdx.y == 0) return;  // test hook
    const uint32_t K = kb + (uint32_t)k;
    const int s = (int)(K % NST);
    const int r = row_of(k);
    const int ra = r == 0 ? ny - 1 : r - 1;  // c_y = +1 group is pulled from row r - 1
    const int rc = r == ny - 1 ? 0 : r + 1;  // c_y = -1 group from row r + 1
    const int cx = x0 + kXOff - LEAD;        // box covers logical columns x0-LEAD .. x0+BW-LEAD-1
    const bool in = LB_IN(ra >= 0 && ra < ny && r >= 0 && r < ny && rc >= 0 && rc < ny && cx >= 0, 3);
    mbar_arrive_expect_tx(&S_.full[s], in ? SM::kTxBytes : 0u);  // 0: the phase completes empty
    if (in) {
      copy_row_boxes(S_.stage[s], GE, srcp, cx, ra, r, rc, &S_.full[s], k < 2);
    }
  };
  auto slot = [&](int k) -> int { return (int)((kb + (uint32_t)k) % NST); };
  auto wait_row = [&](int k) -> bool {
    const uint32_t K = kb + (uint32_t)k;
    return mbar_wait_bounded(&S_.full[K % NST], (K / NST) & 1u, kWaitLimitNs);
  };
  // moments of staged row k into ring slot k & 3 (own column and the strip's halo columns)
  T rho_next = T(0);
  auto ring_moments = [&](int k) {
    const S* st = S_.stage[slot(k)];
    T* rg = &S_.ring[k & (kRing - 1)][0][0];
    constexpr int RS = SM::kRingW;
    T r1, jx, jy, bx, by;
    if (active) {
      moments_from<T, S, BW>(st, GE, t + LEAD, r1, jx, jy, bx, by);
      rg[0 * RS + t + 1] = jx;
      rg[1 * RS + t + 1] = jy;
      rg[2 * RS + t + 1] = bx;
      rg[3 * RS + t + 1] = by;
      rho_next = r1;
    }
    if (t == 0) {  // column x0 - 1
      moments_from<T, S, BW>(st, GE, LEAD - 1, r1, jx, jy, bx, by);
      rg[0 * RS] = jx;
      rg[1 * RS] = jy;
      rg[2 * RS] = bx;
      rg[3 * RS] = by;
    }
    if (t == ncol - 1) {  // column x0 + ncol
      moments_from<T, S, BW>(st, GE, ncol + LEAD, r1, jx, jy, bx, by);
      rg[0 * RS + ncol + 1] = jx;
      rg[1 * RS + ncol + 1] = jy;
      rg[2 * RS + ncol + 1] = bx;
      rg[3 * RS + ncol + 1] = by;
    }
  };

  if (t == 0) {
    S_.abort_flag[0] = 0;
    S_.abort_flag[1] = 0;
  }
  __syncthreads();  // barriers initialised / the previous tile's shared memory released
  const int first = NST < L ? NST : L;
  if (t == 0) {
    fence_proxy_async_smem();
    for (int k = 0; k < first; ++k) issue(k);
  }
  int issued = first;  // meaningful in thread 0 only

  // prologue: rows k = 0 and k = 1
  if (wait_row(0)) ring_moments(0); else S_.abort_flag[1] = 1;
  if (wait_row(1)) ring_moments(1); else S_.abort_flag[1] = 1;
  T rho_cur = rho_next;

  const size_t pitch = (size_t)g.pitch;
  for (int m = 1; m <= L - 2; ++m) {
    // A: moments of the next row
    if (wait_row(m + 1)) ring_moments(m + 1); else S_.abort_flag[m & 1] = 1;
    // B
    __syncthreads();
    if (S_.abort_flag[m & 1]) {
      if (t == 0) {
        atomicOr(err, 1u);
        for (int k = m + 1; k < issued; ++k) wait_row(k);  // drain copies still in flight
      }
      return false;
    }
    if (t == 0 && m - 1 + NST < L) {
      fence_proxy_async_smem();
      issue(m - 1 + NST);
      ++issued;
    }
    // C: gradients, collision and store of row m
    if (active) {
      constexpr int RS = SM::kRingW;
      const T* rc = &S_.ring[m & (kRing - 1)][0][0];
      const T* rn = &S_.ring[(dir > 0 ? m + 1 : m - 1) & (kRing - 1)][0][0];  // row y + 1
      const T* rs = &S_.ring[(dir > 0 ? m - 1 : m + 1) & (kRing - 1)][0][0];  // row y - 1
      const int si = t + 1;
      T dJ[4], dB[4];
      if (ISO) {
        // undivided isotropic differences (scale 1/12 in kq):
        // 4 (a_E - a_W) + (a_NE - a_NW) + (a_SE - a_SW),  4 (a_N - a_S) + (a_NE - a_SE) + (a_NW - a_SW)
        T dx[4], dy[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const T e = rc[f * RS + si + 1], w = rc[f * RS + si - 1];
          const T ne = rn[f * RS + si + 1], nw = rn[f * RS + si - 1], nn = rn[f * RS + si];
          const T se = rs[f * RS + si + 1], sw = rs[f * RS + si - 1], ss = rs[f * RS + si];
          dx[f] = T(4) * (e - w) + ((ne - nw) + (se - sw));
          dy[f] = T(4) * (nn - ss) + ((ne - se) + (nw - sw));
        }
        dJ[0] = dx[0]; dJ[1] = dy[0]; dJ[2] = dx[1]; dJ[3] = dy[1];
        dB[0] = dx[2]; dB[1] = dy[2]; dB[2] = dx[3]; dB[3] = dy[3];
      } else {
        // undivided central differences a(+1) - a(-1) (scale 1/2 in kq)
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          const T ddx = rc[f * RS + si + 1] - rc[f * RS + si - 1];
          const T ddy = rn[f * RS + si] - rs[f * RS + si];
          if (f < 2) { dJ[2 * f] = ddx; dJ[2 * f + 1] = ddy; }
          else { dB[2 * (f - 2)] = ddx; dB[2 * (f - 2) + 1] = ddy; }
        }
      }
      const T jx = rc[0 * RS + si], jy = rc[1 * RS + si], bx = rc[2 * RS + si], by = rc[3 * RS + si];
      const S* st = S_.stage[slot(m)];
      T p[kQ];
#pragma unroll
      for (int q = 0; q < kQ; ++q) p[q] = staged<T, S, BW>(st, GE, q, t + LEAD);
      const int y = row_of(m);
      const int x = x0 + t;
      if (CORR) {
        const size_t cell = (size_t)y * nx + x, cplane = (size_t)nx * ny;
        const T cq[4] = {(T)corr[cell], (T)corr[cplane + cell], (T)corr[2 * cplane + cell],
                         (T)corr[3 * cplane + cell]};
        collide<T, true>(p, rho_cur, jx, jy, bx, by, dJ, dB, c, cq);
      } else {
        collide(p, rho_cur, jx, jy, bx, by, dJ, dB, c);
      }
      S* o = dst + (size_t)y * pitch + kXOff + x;
      const S* end = dst + (size_t)g.pitch * ny;  // one past the copy (checking build)
      store_planes<S, T, 0>(o, p, g.plane, dst, end);
      if (x < 2) {  // right ghosts: logical columns nx, nx + 1
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          S* a = o + (size_t)plane_of(q) * g.plane + nx;
          if (LB_IN(a >= dst && a < end, 2)) *a = store_as<S>(p[q]);
        }
      }
      if (x >= nx - 2) {  // left ghosts: logical columns -2, -1
#pragma unroll
        for (int q = 0; q < kQ; ++q) {
          S* a = o + (size_t)plane_of(q) * g.plane - nx;
          if (LB_IN(a >= dst && a < end, 2)) *a = store_as<S>(p[q]);
        }
      }
    }
    rho_cur = rho_next;
  }
  kbase = kb + (uint32_t)L;
  return true;
}

// The pair (staged value of population q at box columns col, col + 1) for two adjacent cells.
template <int BW>
__device__ __forceinline__ F2 staged_pair(const __half* st, int ge, int q, int col) {
  const int i = q % 9;
  const int c = col - vel_x(i);
  if (!LB_IN(c >= 0 && c + 1 < BW && (vel_x(i) != 0 || c % 2 == 0), 0)) return f2(0.f);
  const __half* a = st + group_of(i) * ge + (3 * (q / 9) + index_in_group(i)) * BW + c;
  if (vel_x(i) == 0) {  // even column: one aligned 32-bit load
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(a));
    return f2(v.x, v.y);
  }
  return f2(__half2float(a[0]), __half2float(a[1]));
}

// Relative binary16 storage (LBMHD_FP16_REL): stored f values are s_i = f*_i - w_i (1 + 3 c_i . U)
// with U the velocity reference of the cell that wrote them (planes 27, 28); the deviation f_i - w_i
// of a pulled population is s_i + 3 w_i c_i . U(source cell).  urow[g] is the staged U row
// ([2][BW]: U_x, then U_y) of the source row of plane group g.
template <int BW>
__device__ __forceinline__ F2 u_pair(const __half* ur, int comp, int c) {  // U_comp at columns c, c + 1
  const __half* a = ur + comp * BW + c;
  if ((c & 1) == 0) {  // even column: one aligned 32-bit load
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(a));
    return f2(v.x, v.y);
  }
  return f2(__half2float(a[0]), __half2float(a[1]));
}
__device__ __forceinline__ constexpr float w3_of(int i) { return i < 5 ? 1.f / 3.f : 1.f / 12.f; }  // 3 w_i

template <int BW, bool REL>
__device__ __forceinline__ F2 staged_pair_rel(const __half* st, int ge, int q, int col, const __half* const* urow) {
  F2 v = staged_pair<BW>(st, ge, q, col);
  if constexpr (REL) {
    if (q >= 1 && q < 9) {
      const int c = col - vel_x(q);
      const __half* ur = urow[group_of(q)];
      if (!LB_IN(c >= 0 && c + 1 < BW, 0)) return v;
      if (vel_x(q) != 0) v = fma2(f2((float)vel_x(q) * w3_of(q)), u_pair<BW>(ur, 0, c), v);
      if (vel_y(q) != 0) v = fma2(f2((float)vel_y(q) * w3_of(q)), u_pair<BW>(ur, 1, c), v);
    }
  }
  return v;
}

// Scalar (one cell) pulled value for the relative form, as staged_pair_rel.
template <int BW, bool REL>
__device__ __forceinline__ float staged_rel(const __half* st, int ge, int q, int col, const __half* const* urow) {
  float v = staged<float, __half, BW>(st, ge, q, col);
  if constexpr (REL) {
    if (q >= 1 && q < 9) {
      const int c = col - vel_x(q);
      const __half* ur = urow[group_of(q)];
      if (!LB_IN(c >= 0 && c < BW, 0)) return v;
      if (vel_x(q) != 0) v = fmaf((float)vel_x(q) * w3_of(q), __half2float(ur[c]), v);
      if (vel_y(q) != 0) v = fmaf((float)vel_y(q) * w3_of(q), __half2float(ur[BW + c]), v);
    }
  }
  return v;
}

template <int BW, bool REL>
__device__ __forceinline__ void moments_one_rel(const __half* st, int ge, int col, const __half* const* urow,
                                                float& rho1, float& jx, float& jy, float& bx, float& by) {
  auto v = [&](int q) -> float { return staged_rel<BW, REL>(st, ge, q, col, urow); };
  const float f0 = v(0), f1 = v(1), f2_ = v(2), f3 = v(3), f4 = v(4), f5 = v(5), f6 = v(6), f7 = v(7), f8 = v(8);
  rho1 = ((f0 + f1) + (f2_ + f3)) + ((f4 + f5) + (f6 + f7)) + f8;
  jx = (f1 - f3) + (f5 - f6) + (f8 - f7);
  jy = (f2_ - f4) + (f5 - f8) + (f6 - f7);
  bx = ((v(9) + v(10)) + (v(11) + v(12))) + ((v(13) + v(14)) + (v(15) + v(16))) + v(17);
  by = ((v(18) + v(19)) + (v(20) + v(21))) + ((v(22) + v(23)) + (v(24) + v(25))) + v(26);
}

template <int BW, bool REL = false>
__device__ __forceinline__ void moments_pair(const __half* st, int ge, int col, F2& rho1, F2& jx, F2& jy, F2& bx,
                                             F2& by, const __half* const* urow = nullptr) {
  auto v = [&](int q) -> F2 { return staged_pair_rel<BW, REL>(st, ge, q, col, urow); };
  const F2 f0 = v(0), f1 = v(1), f2_ = v(2), f3 = v(3), f4 = v(4), f5 = v(5), f6 = v(6), f7 = v(7), f8 = v(8);
  rho1 = ((f0 + f1) + (f2_ + f3)) + ((f4 + f5) + (f6 + f7)) + f8;
  jx = (f1 - f3) + (f5 - f6) + (f8 - f7);
  jy = (f2_ - f4) + (f5 - f8) + (f6 - f7);
  bx = ((v(9) + v(10)) + (v(11) + v(12))) + ((v(13) + v(14)) + (v(15) + v(16))) + v(17);
  by = ((v(18) + v(19)) + (v(20) + v(21))) + ((v(22) + v(23)) + (v(24) + v(25))) + v(26);
}

// Store the 27 values of two adjacent cells (binary16 pairs, one 32-bit store per plane), planes
// in address order; `both` false stores the first cell only (odd strip width).
template <int PL>
__device__ __forceinline__ void store_planes_pair(__half* op, const F2* p, size_t plane, bool both,
                                                  const __half* lo_end, const __half* hi_end) {
  if constexpr (PL < kQ) {
    constexpr int q = q_of_plane(PL);
    if (LB_IN(op >= lo_end && op + (both ? 2 : 1) <= hi_end, 2)) {
      if (both)
        *reinterpret_cast<__half2*>(op) = __floats2half2_rn(lo(p[q]), hi(p[q]));
      else
        *op = __float2half_rn(lo(p[q]));
    }
    store_planes_pair<PL + 1>(op + plane, p, plane, both, lo_end, hi_end);
  }
}

// One tile of a binary16 grid with two adjacent cells per thread (kStepThreads / 2 threads per
// strip of kStepThreads columns): the pipeline of run_tile, with the moments, the collision
// and the stores of a cell pair in packed binary32 (F2).  Same arguments and contract as run_tile.
// REL: relative binary16 storage (LBMHD_FP16_REL, single-grid steps only): usrcp maps the U
// planes (27, 28: U_x, U_y of the writing cell, boxes {BW, 2, 1}); each staged row also brings the
// U row of the source row one ahead in march order (the first also the two before it) into the U
// ring, the pulled f values are taken relative to their source cells' U (staged_pair_rel), and
// the post-collision f values are stored relative to this cell's own velocity, which is stored
// in binary16 as its U.
template <int ISO, int NST, bool REL = false>
__device__ __forceinline__ bool run_tile_pair(const CUtensorMap* srcp, __half* __restrict__ dst, const StepGeom& g,
                                              const KCoef<float>& c1, int x0, int y0, int band_parity,
                                              uint32_t& kbase, unsigned* __restrict__ err,
                                              const CUtensorMap* usrcp = nullptr) {
  using SM = StepSmem<__half, NST, REL>;
  constexpr int GE = SM::kGroupElems;
  constexpr int LEAD = SM::kLead;
  constexpr int BW = SM::kBoxW;
  constexpr int RW = SM::kRingW;
  static_assert(SM::kRingOff == 2, "pair layout");
  SM& S_ = step_smem<__half, NST, REL>();

  const int t = threadIdx.x;
  const int c0 = 2 * t;  // first of this thread's two strip columns
  const int nx = g.nx, ny = g.ny;
  const int ncol = min(kStepThreads, nx - x0);
  const bool active = c0 < ncol;
  // ring indices 1 .. ncol + 3 are read or written (uniform over the block)
  if (!LB_IN(ncol >= 1 && ncol + 3 < RW, 1)) return true;
  const int last = (ncol - 1) / 2;  // thread holding the strip's last column
  const int y1 = min(y0 + g.band, ny);
  const int L = (y1 - y0) + 2;
  const int dir = (band_parity & 1) ? -1 : 1;
  const uint32_t kb = kbase;
  const KCoef2 c = pair_coef(c1);
  auto row_of = [&](int k) -> int {
    int r = dir > 0 ? y0 - 1 + k : y1 - k;
    if (r < 0) r += ny;
    if (r >= ny) r -= ny;
    return r;
  };
  auto issue = [&](int k) {
    if (g.skip_copy && k == 2 && blockIdx.x == 0 && blockIdx.y == 0) return;  // test hook
    const uint32_t K = kb + (uint32_t)k;
    const int s = (int)(K % NST);
    const int r = row_of(k);
    const int ra = r == 0 ? ny - 1 : r - 1;
    const int rc = r == ny - 1 ? 0 : r + 1;
    const int cx = x0 + kXOff - LEAD;
    const bool in = LB_IN(ra >= 0 && ra < ny && r >= 0 && r < ny && rc >= 0 && rc < ny && cx >= 0, 3);
    constexpr uint32_t kUBytes = 2u * BW * 2u;  // one U row
    const uint32_t ubytes = REL ? (k == 0 ? 3u : 1u) * kUBytes : 0u;
    mbar_arrive_expect_tx(&S_.full[s], in ? SM::kTxBytes + ubytes : 0u);  // 0: the phase completes empty
    if (in) {
      copy_row_boxes(S_.stage[s], GE, srcp, cx, ra, r, rc, &S_.full[s], k < 2);
      if constexpr (REL) {  // U rows of march indices k + 1 (and k - 1, k for the first row)
        for (int j = (k == 0 ? -1 : k + 1); j <= k + 1; ++j)
          tma_load_3d(&S_.uring[(j + kURing) % kURing][0], usrcp, cx, kQ, row_of(j), &S_.full[s]);
      }
    }
  };
  // staged U rows of the source rows of the three plane groups of march row k (groups 0, 1, 2
  // are pulled from rows y - 1, y, y + 1: march indices k - dir, k, k + dir)
  auto urows = [&](int k, const __half* (&u)[3]) {
    if constexpr (REL) {
      u[0] = &S_.uring[(k - dir + kURing) % kURing][0];
      u[1] = &S_.uring[(k + kURing) % kURing][0];
      u[2] = &S_.uring[(k + dir + kURing) % kURing][0];
    } else {
      u[0] = u[1] = u[2] = nullptr;
    }
  };
  auto slot = [&](int k) -> int { return (int)((kb + (uint32_t)k) % NST); };
  auto wait_row = [&](int k) -> bool {
    const uint32_t K = kb + (uint32_t)k;
    return mbar_wait_bounded(&S_.full[K % NST], (K / NST) & 1u, kWaitLimitNs);
  };
  // moments of staged row k into ring slot k & 3: the thread's cell pair at ring index c0 + 2,
  // the halo columns -1 (index 1) and ncol (index ncol + 2; covered by the last pair when ncol
  // is odd)
  F2 rho_next = f2(0.f);
  auto ring_moments = [&](int k) {
    const __half* st = S_.stage[slot(k)];
    float* rg = &S_.ring[k & (kRing - 1)][0][0];
    const __half* ur[3];
    urows(k, ur);
    if (active) {
      F2 r1, jx, jy, bx, by;
      moments_pair<BW, REL>(st, GE, c0 + LEAD, r1, jx, jy, bx, by, ur);
      *reinterpret_cast<uint64_t*>(rg + 0 * RW + c0 + 2) = jx.v;
      *reinterpret_cast<uint64_t*>(rg + 1 * RW + c0 + 2) = jy.v;
      *reinterpret_cast<uint64_t*>(rg + 2 * RW + c0 + 2) = bx.v;
      *reinterpret_cast<uint64_t*>(rg + 3 * RW + c0 + 2) = by.v;
      rho_next = r1;
    }
    float r1, jx, jy, bx, by;
    if (t == 0) {
      moments_one_rel<BW, REL>(st, GE, LEAD - 1, ur, r1, jx, jy, bx, by);
      rg[0 * RW + 1] = jx;
      rg[1 * RW + 1] = jy;
      rg[2 * RW + 1] = bx;
      rg[3 * RW + 1] = by;
    }
    if (t == last && (ncol & 1) == 0) {
      moments_one_rel<BW, REL>(st, GE, ncol + LEAD, ur, r1, jx, jy, bx, by);
      rg[0 * RW + ncol + 2] = jx;
      rg[1 * RW + ncol + 2] = jy;
      rg[2 * RW + ncol + 2] = bx;
      rg[3 * RW + ncol + 2] = by;
    }
  };

  if (t == 0) {
    S_.abort_flag[0] = 0;
    S_.abort_flag[1] = 0;
  }
  __syncthreads();
  const int first = NST < L ? NST : L;
  if (t == 0) {
    fence_proxy_async_smem();
    for (int k = 0; k < first; ++k) issue(k);
  }
  int issued = first;

  if (wait_row(0)) ring_moments(0); else S_.abort_flag[1] = 1;
  if (wait_row(1)) ring_moments(1); else S_.abort_flag[1] = 1;
  F2 rho_cur = rho_next;

  const size_t pitch = (size_t)g.pitch;
  for (int m = 1; m <= L - 2; ++m) {
    if (wait_row(m + 1)) ring_moments(m + 1); else S_.abort_flag[m & 1] = 1;
    __syncthreads();
    if (S_.abort_flag[m & 1]) {
      if (t == 0) {
        atomicOr(err, 1u);
        for (int k = m + 1; k < issued; ++k) wait_row(k);
      }
      return false;
    }
    if (t == 0 && m - 1 + NST < L) {
      fence_proxy_async_smem();
      issue(m - 1 + NST);
      ++issued;
    }
    if (active) {
      const float* rc = &S_.ring[m & (kRing - 1)][0][0];
      const float* rn = &S_.ring[(dir > 0 ? m + 1 : m - 1) & (kRing - 1)][0][0];
      const float* rs = &S_.ring[(dir > 0 ? m - 1 : m + 1) & (kRing - 1)][0][0];
      const int si = c0 + 2;  // ring index of the first cell
      F2 dJ[4], dB[4], own[4];
      if (ISO) {
        // per cell as in run_tile: 4 (a_E - a_W) + (a_NE - a_NW) + (a_SE - a_SW), etc.
        F2 dx[4], dy[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          float ddx[2], ddy[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int j = si + h;
            const float e = rc[f * RW + j + 1], w = rc[f * RW + j - 1];
            const float ne = rn[f * RW + j + 1], nw = rn[f * RW + j - 1], nn = rn[f * RW + j];
            const float se = rs[f * RW + j + 1], sw = rs[f * RW + j - 1], ss = rs[f * RW + j];
            ddx[h] = 4.f * (e - w) + ((ne - nw) + (se - sw));
            ddy[h] = 4.f * (nn - ss) + ((ne - se) + (nw - sw));
          }
          dx[f] = f2(ddx[0], ddx[1]);
          dy[f] = f2(ddy[0], ddy[1]);
          own[f].v = *reinterpret_cast<const uint64_t*>(rc + f * RW + si);
        }
        dJ[0] = dx[0]; dJ[1] = dy[0]; dJ[2] = dx[1]; dJ[3] = dy[1];
        dB[0] = dx[2]; dB[1] = dy[2]; dB[2] = dx[3]; dB[3] = dy[3];
      } else {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
          own[f].v = *reinterpret_cast<const uint64_t*>(rc + f * RW + si);
          F2 nrow, srow;
          nrow.v = *reinterpret_cast<const uint64_t*>(rn + f * RW + si);
          srow.v = *reinterpret_cast<const uint64_t*>(rs + f * RW + si);
          const F2 ddx = f2(hi(own[f]) - rc[f * RW + si - 1], rc[f * RW + si + 2] - lo(own[f]));
          const F2 ddy = nrow - srow;
          if (f < 2) { dJ[2 * f] = ddx; dJ[2 * f + 1] = ddy; }
          else { dB[2 * (f - 2)] = ddx; dB[2 * (f - 2) + 1] = ddy; }
        }
      }
      const __half* st = S_.stage[slot(m)];
      const __half* ur[3];
      urows(m, ur);
      F2 p[kQ];
#pragma unroll
      for (int q = 0; q < kQ; ++q) p[q] = staged_pair_rel<BW, REL>(st, GE, q, c0 + LEAD, ur);
      F2 ir;
      collide_pair(p, rho_cur, own[0], own[1], own[2], own[3], dJ, dB, c, &ir);
      const int y = row_of(m);
      const int x = x0 + c0;
      __half* o = dst + (size_t)y * pitch + kXOff + x;
      const __half* end = dst + (size_t)g.pitch * ny;  // one past the copy (checking build)
      __half2 uh[2];  // this cell pair's velocity reference U_x, U_y (binary16)
      if constexpr (REL) {
        // u = J / rho of the cells (collision invariants), rounded to binary16; the f values are
        // stored relative to w_i (1 + 3 c_i . U): f_1 -= U_x / 3, f_3 += U_x / 3, f_2 -= U_y / 3,
        // f_4 += U_y / 3, f_5 -= (U_x + U_y) / 12, f_7 += (U_x + U_y) / 12, f_6 -= (U_y - U_x) / 12,
        // f_8 += (U_y - U_x) / 12
        const F2 ux = own[0] * ir, uy = own[1] * ir;
        uh[0] = __floats2half2_rn(lo(ux), hi(ux));
        uh[1] = __floats2half2_rn(lo(uy), hi(uy));
        const float2 fx = __half22float2(uh[0]), fy = __half22float2(uh[1]);
        const F2 Ux = f2(fx.x, fx.y), Uy = f2(fy.x, fy.y);
        const F2 a = f2(1.f / 3.f) * Ux, b = f2(1.f / 3.f) * Uy;
        const F2 d1 = f2(1.f / 12.f) * (Ux + Uy), d2 = f2(1.f / 12.f) * (Uy - Ux);
        p[1] = p[1] - a;
        p[3] = p[3] + a;
        p[2] = p[2] - b;
        p[4] = p[4] + b;
        p[5] = p[5] - d1;
        p[7] = p[7] + d1;
        p[6] = p[6] - d2;
        p[8] = p[8] + d2;
      }
      store_planes_pair<0>(o, p, g.plane, c0 + 1 < ncol, dst, end);
      if constexpr (REL) {
#pragma unroll
        for (int comp = 0; comp < 2; ++comp) {
          __half* a = o + (size_t)(kQ + comp) * g.plane;
          if (LB_IN(a >= dst && a + (c0 + 1 < ncol ? 2 : 1) <= end, 2)) {
            if (c0 + 1 < ncol) *reinterpret_cast<__half2*>(a) = uh[comp];
            else *a = __low2half(uh[comp]);
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int xh = x + h;
        if (h == 1 && c0 + 1 >= ncol) break;
        if (xh < 2 || xh >= nx - 2) {  // ghosts: logical nx, nx + 1 and -2, -1
          __half* gp = o + h + (xh < 2 ? nx : -nx);
#pragma unroll
          for (int q = 0; q < kQ; ++q) {
            __half* a = gp + (size_t)plane_of(q) * g.plane;
            if (LB_IN(a >= dst && a < end, 2)) *a = __float2half_rn(h ? hi(p[q]) : lo(p[q]));
          }
          if constexpr (REL) {
#pragma unroll
            for (int comp = 0; comp < 2; ++comp) {
              __half* a = gp + (size_t)(kQ + comp) * g.plane;
              if (LB_IN(a >= dst && a < end, 2)) *a = h ? __high2half(uh[comp]) : __low2half(uh[comp]);
            }
          }
        }
      }
    }
    rho_cur = rho_next;
  }
  kbase = kb + (uint32_t)L;
  return true;
}

// Threads of a step block: one per strip column, or one per column pair for binary16 storage.
template <typename S>
__host__ __device__ constexpr int step_threads() {
  return sizeof(S) == 2 ? kStepThreads / 2 : kStepThreads;
}

// One tile of the strip starting at x0 (binary16: two cells per thread).
template <typename S, int ISO, int NST, bool CORR = false>
__device__ __forceinline__ bool run_any_tile(const CUtensorMap* srcp, S* __restrict__ dst, const StepGeom& g,
                                             const KCoef<typename ArithOf<S>::type>& c, int x0, int y0,
                                             int band_parity, uint32_t& kbase, unsigned* __restrict__ err,
                                             const float* __restrict__ corr = nullptr) {
  if constexpr (sizeof(S) == 2)
    return run_tile_pair<ISO, NST>(srcp, dst, g, c, x0, y0, band_parity, kbase, err);
  else
    return run_tile<S, ISO, NST, CORR>(srcp, dst, g, c, x0, y0, band_parity, kbase, err, corr);
}

// Tile (strip, band) of the block with linear index L = blockIdx.y * strips + blockIdx.x.  Blocks
// are dispatched in linear order, and of the blocks that share an SM the later-dispatched run
// slower (2048^2 binary32: 134.6 / 135.4 / 136.0 / 137.5 us for the four of an SM, from per-block
// timestamps).  The two edge strips, which also write the periodic ghost columns, are 1.6% slower
// again, so their tiles take the first linear indices: the slowest pairing (edge strip, last
// dispatched) disappears.  Measured: 0.27% less time per step at 2048^2 and 4096^2 binary32,
// bitwise the same state.
__device__ __forceinline__ void tile_of_block(int& strip, int& band) {
  const int ns = (int)gridDim.x, nb = (int)gridDim.y;
  strip = (int)blockIdx.x;
  band = (int)blockIdx.y;
  if (ns < 3) return;
  const int L = band * ns + strip;
  if (L < 2 * nb) {
    strip = (L & 1) ? ns - 1 : 0;
    band = L >> 1;
  } else {
    const int li = L - 2 * nb;
    strip = 1 + li % (ns - 2);
    band = li / (ns - 2);
  }
}

// One grid: one block per tile (strip, band), see tile_of_block.  CORR: add the correction planes
// corr[4][ny][nx].  flip (0 / 1, the source copy's index, so it alternates from step to step)
// reverses every band's marching direction: a band then starts each step at the rows it (and its
// neighbour) wrote last in the previous step, which are still in L2 (about the last 5 rows per
// band at 2048^2 binary32), instead of at the far end, long evicted.
template <typename S, int ISO, int NST, int MINB, bool CORR = false>
__global__ void __launch_bounds__(step_threads<S>(), MINB)
    fused_step_kernel(const __grid_constant__ CUtensorMap src, S* __restrict__ dst, StepGeom g,
                      KCoef<typename ArithOf<S>::type> c, unsigned* __restrict__ err,
                      const float* __restrict__ corr, int flip) {
  int strip, band;
  tile_of_block(strip, band);
  if (band * g.band >= g.ny) return;  // uniform per block
  init_stage_barriers(step_smem<S, NST>(), &src);
  grid_dependency_wait();  // the previous step has written src (and read dst)
  uint32_t kbase = 0;
  run_any_tile<S, ISO, NST, CORR>(&src, dst, g, c, strip * kStepThreads, band * g.band, band + flip, kbase,
                                  err, corr);
}

// Relative binary16 storage (LBMHD_FP16_REL; single grids): fused_step_kernel's binary16 step
// with the U planes' tensor map (fixed marching direction, as for binary16).
template <int ISO, int NST, int MINB>
__global__ void __launch_bounds__(kStepThreads / 2, MINB)
    fused_step_rel_kernel(const __grid_constant__ CUtensorMap src, const __grid_constant__ CUtensorMap usrc,
                          __half* __restrict__ dst, StepGeom g, KCoef<float> c, unsigned* __restrict__ err) {
  int strip, band;
  tile_of_block(strip, band);
  if (band * g.band >= g.ny) return;  // uniform per block
  init_stage_barriers(step_smem<__half, NST, true>(), &src, &usrc);
  grid_dependency_wait();
  uint32_t kbase = 0;
  run_tile_pair<ISO, NST, true>(&src, dst, g, c, strip * kStepThreads, band * g.band, band, kbase, err, &usrc);
}

// Ensemble: every member grid advances one step in this launch.  work[i] = {member, x0, y0,
// band index}; blocks take tiles either by a static stride over the list (queue == nullptr) or
// from an atomic counter (persistent blocks; the counter is zeroed before each launch).
template <typename S>
struct EnsembleMember {
  CUtensorMap map[2];  // tensor maps of the member's two population copies (64-byte aligned)
  S* pops[2];
  StepGeom g;
  KCoef<typename ArithOf<S>::type> c;
};

template <typename S, int ISO, int NST, int MINB>
__global__ void __launch_bounds__(step_threads<S>(), MINB)
    ensemble_step_kernel(const EnsembleMember<S>* __restrict__ members, const int4* __restrict__ work,
                         int nwork, int parity, unsigned long long* queue, unsigned* __restrict__ err) {
  __shared__ int next_item;
  init_stage_barriers(step_smem<S, NST>(), nullptr);
  grid_dependency_wait();
  uint32_t kbase = 0;
  int w = blockIdx.x;
  if (queue) {
    if (threadIdx.x == 0) next_item = (int)atomicAdd(queue, 1ull);
    __syncthreads();
    w = next_item;
  }
  while (w < nwork) {
    const int4 it = work[w];
    const EnsembleMember<S>& mb = members[it.x];
    // the march direction alternates with the step (parity) as for single grids: not for
    // binary16 storage
    const int flip = sizeof(S) == 2 ? 0 : parity;
    if (!run_any_tile<S, ISO, NST>(&mb.map[parity], mb.pops[parity ^ 1], mb.g, mb.c, it.y, it.z, it.w + flip,
                                   kbase, err))
      return;
    if (queue) {
      __syncthreads();  // everyone has read next_item before it is overwritten
      if (threadIdx.x == 0) next_item = (int)atomicAdd(queue, 1ull);
      __syncthreads();
      w = next_item;
    } else {
      w += gridDim.x;
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

// Pipeline depth and residency per storage type (at least 3 stages: iteration m waits for row
// m + 1, which must already have been issued).  binary32 rows are 15 KB per stage: 3 stages and
// 4 blocks per SM (16 warps) measured fastest at 2048^2 and 4096^2 -- more resident warps beat
// deeper pipelines (4 stages x 3 blocks: 0.81 of the copy bandwidth, 3 x 4: 0.92).  binary16
// rows are 8 KB; that form runs two cells per thread (64-thread blocks, packed binary32
// arithmetic) and is bound by latency at the 12 warps per SM that shared memory allows: 3
// stages x 6 blocks measured best at 2048^2 (46.4 GLUPS; 5 x 4: 43.4, 4 x 5: 40.0, 3 x 5: 39.8).
// binary64 rows are 30 KB: 3 stages, 2 blocks per SM; that form is bound by the binary64
// arithmetic rate.  Overridable at build time for sweeps.
#ifndef LBMHD_F32_STAGES
#define LBMHD_F32_STAGES 3
#endif
#ifndef LBMHD_F32_BLOCKS
#define LBMHD_F32_BLOCKS 4
#endif
#ifndef LBMHD_F64_STAGES
#define LBMHD_F64_STAGES 3
#endif
#ifndef LBMHD_F64_BLOCKS
#define LBMHD_F64_BLOCKS 2
#endif
#ifndef LBMHD_WAVES
#define LBMHD_WAVES 1
#endif
// Fewest rows per band.  Grids too small to fill one wave with long bands (below about
// 512^2) are bound by the pipeline's fill latency, not by memory, so thin bands pay: with one
// row at least, 128^2 binary32 runs at 5.4 GLUPS (4 rows: 2.9), 256^2 at 13.5 (11.8), 256^2
// binary16 at 14.2 (9.0) and the 64^2 binary64 run at 0.28 (0.10); 512^2 and up are unchanged.
#ifndef LBMHD_MIN_BAND
#define LBMHD_MIN_BAND 1
#endif
#ifndef LBMHD_F16_STAGES
#define LBMHD_F16_STAGES 3
#endif
#ifndef LBMHD_F16_BLOCKS
#define LBMHD_F16_BLOCKS 6
#endif
template <typename S> struct StepConfig;
template <> struct StepConfig<float> {
  static constexpr int kStages = LBMHD_F32_STAGES, kMinBlocks = LBMHD_F32_BLOCKS;
};
template <> struct StepConfig<double> {
  static constexpr int kStages = LBMHD_F64_STAGES, kMinBlocks = LBMHD_F64_BLOCKS;
};
template <> struct StepConfig<__half> {
  static constexpr int kStages = LBMHD_F16_STAGES, kMinBlocks = LBMHD_F16_BLOCKS;
};

template <typename S, int ISO, bool CORR = false>
constexpr auto kernel_ptr() {
  return &fused_step_kernel<S, ISO, StepConfig<S>::kStages, StepConfig<S>::kMinBlocks, CORR>;
}

template <typename S>
constexpr size_t smem_bytes() {
  return sizeof(StepSmem<S, StepConfig<S>::kStages>) + 128;  // + alignment slack
}

template <int ISO>
constexpr auto rel_kernel_ptr() {
  return &fused_step_rel_kernel<ISO, StepConfig<__half>::kStages, StepConfig<__half>::kMinBlocks>;
}
constexpr size_t rel_smem_bytes() { return sizeof(StepSmem<__half, StepConfig<__half>::kStages, true>) + 128; }
// six relative-form blocks per SM: 6 x (rel_smem_bytes + 1 KB reserved) within 228 KB
static_assert(6 * (rel_smem_bytes() + 1024) <= 228 * 1024, "relative binary16 blocks fit six per SM");

// Steps are launched with programmatic stream serialisation (launch_programmatic): a step's
// blocks may be scheduled while the previous kernel in the stream drains and wait
// (grid_dependency_wait) before touching global memory.  Measured: 6.5% less time per step at
// 256^2 binary32, 10% at 128^2, 3% at 512^2, large grids unchanged (bitwise the same
// results); letting dependants launch early (griddepcontrol.launch_dependents at block start)
// instead of at block exit made small grids slower (128^2 binary32 23% slower).
template <typename S>
cudaError_t launch_step(const CUtensorMap& src, S* dst, const StepGeom& g, const StepCoef& c,
                        int stencil, unsigned* err, const float* corr, int flip, cudaStream_t s) {
  dim3 grid((g.nx + kStepThreads - 1) / kStepThreads, (g.ny + g.band - 1) / g.band);
  auto k = cast_coef<typename ArithOf<S>::type>(c);
  const int nt = step_threads<S>();
  const size_t sm = smem_bytes<S>();
  if (corr) {
    if constexpr (sizeof(S) == 2)
      return cudaErrorNotSupported;  // the correction is offered for binary64 / binary32 storage
    else
      return stencil == 1 ? launch_programmatic(kernel_ptr<S, 1, true>(), grid, nt, sm, s, src, dst, g, k, err, corr, flip)
                          : launch_programmatic(kernel_ptr<S, 0, true>(), grid, nt, sm, s, src, dst, g, k, err, corr, flip);
  }
  const float* none = nullptr;
  return stencil == 1 ? launch_programmatic(kernel_ptr<S, 1>(), grid, nt, sm, s, src, dst, g, k, err, none, flip)
                      : launch_programmatic(kernel_ptr<S, 0>(), grid, nt, sm, s, src, dst, g, k, err, none, flip);
}

cudaError_t launch_step_rel(const CUtensorMap& src, const CUtensorMap& usrc, __half* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, cudaStream_t s) {
  dim3 grid((g.nx + kStepThreads - 1) / kStepThreads, (g.ny + g.band - 1) / g.band);
  const KCoef<float> k = cast_coef<float>(c);
  const int nt = kStepThreads / 2;
  const size_t sm = rel_smem_bytes();
  return stencil == 1 ? launch_programmatic(rel_kernel_ptr<1>(), grid, nt, sm, s, src, usrc, dst, g, k, err)
                      : launch_programmatic(rel_kernel_ptr<0>(), grid, nt, sm, s, src, usrc, dst, g, k, err);
}

template <typename S, int ISO>
constexpr auto ensemble_kernel_ptr() {
  return &ensemble_step_kernel<S, ISO, StepConfig<S>::kStages, StepConfig<S>::kMinBlocks>;
}

template <typename S>
cudaError_t set_smem_attr() {
  const int b = (int)smem_bytes<S>();
  cudaError_t e = cudaFuncSetAttribute(kernel_ptr<S, 0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel_ptr<S, 1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if constexpr (sizeof(S) != 2) {
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel_ptr<S, 0, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kernel_ptr<S, 1, true>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  }
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ensemble_kernel_ptr<S, 0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(ensemble_kernel_ptr<S, 1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

template <typename S>
void pack_members(int n, const CUtensorMap* maps, void* const* pops, const StepGeom* geoms,
                  const StepCoef* coefs, void* out) {
  EnsembleMember<S>* m = static_cast<EnsembleMember<S>*>(out);
  for (int i = 0; i < n; ++i) {
    m[i].map[0] = maps[2 * i];
    m[i].map[1] = maps[2 * i + 1];
    m[i].pops[0] = static_cast<S*>(pops[2 * i]);
    m[i].pops[1] = static_cast<S*>(pops[2 * i + 1]);
    m[i].g = geoms[i];
    m[i].c = cast_coef<typename ArithOf<S>::type>(coefs[i]);
  }
}

template <typename S>
cudaError_t launch_ens(int stencil, const void* members, const int4* work, int nwork, int parity,
                       unsigned long long* queue, int grid, unsigned* err, cudaStream_t s) {
  const EnsembleMember<S>* mb = static_cast<const EnsembleMember<S>*>(members);
  if (!queue)  // static schedule: the previous launch is the previous step kernel
    return stencil == 1
               ? launch_programmatic(ensemble_kernel_ptr<S, 1>(), dim3(grid), step_threads<S>(), smem_bytes<S>(), s,
                                     mb, work, nwork, parity, queue, err)
               : launch_programmatic(ensemble_kernel_ptr<S, 0>(), dim3(grid), step_threads<S>(), smem_bytes<S>(), s,
                                     mb, work, nwork, parity, queue, err);
  // persistent schedule: a memset of the tile counter precedes each launch; ordinary ordering
  if (stencil == 1)
    ensemble_kernel_ptr<S, 1>()<<<grid, step_threads<S>(), smem_bytes<S>(), s>>>(mb, work, nwork, parity, queue, err);
  else
    ensemble_kernel_ptr<S, 0>()<<<grid, step_threads<S>(), smem_bytes<S>(), s>>>(mb, work, nwork, parity, queue, err);
  return cudaGetLastError();
}

}  // namespace

#ifdef LBMHD_BOUNDS_CHECK
unsigned bounds_check_flags() {
  unsigned v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_bounds_flags, sizeof v) != cudaSuccess) return ~0u;
  cudaMemcpyToSymbol(g_bounds_flags, &z, sizeof z);
  return v;
}
#endif

cudaError_t prepare_step_kernels() {
  cudaError_t e = set_smem_attr<float>();
  if (e == cudaSuccess) e = set_smem_attr<double>();
  if (e == cudaSuccess) e = set_smem_attr<__half>();
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rel_kernel_ptr<0>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rel_smem_bytes());
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(rel_kernel_ptr<1>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rel_smem_bytes());
#ifdef LBMHD_BOUNDS_CHECK
  const char* env = getenv("LBMHD_BOUNDS_FORCE");
  const unsigned force = env ? (unsigned)strtoul(env, nullptr, 0) : 0u;
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_bounds_force, &force, sizeof force);
#endif
  return e;
}

cudaError_t launch_step_f64(const CUtensorMap& src, double* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, const float* corr,
                            int flip, cudaStream_t s) {
  return launch_step<double>(src, dst, g, c, stencil, err, corr, flip, s);
}

cudaError_t launch_step_f32(const CUtensorMap& src, float* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, const float* corr,
                            int flip, cudaStream_t s) {
  return launch_step<float>(src, dst, g, c, stencil, err, corr, flip, s);
}

cudaError_t launch_step_f16(const CUtensorMap& src, __half* dst, const StepGeom& g,
                            const StepCoef& c, int stencil, unsigned* err, const float* corr,
                            int flip, cudaStream_t s) {
  return launch_step<__half>(src, dst, g, c, stencil, err, corr, flip, s);
}

cudaError_t launch_step_f16rel(const CUtensorMap& src, const CUtensorMap& usrc, __half* dst, const StepGeom& g,
                               const StepCoef& c, int stencil, unsigned* err, cudaStream_t s) {
  return launch_step_rel(src, usrc, dst, g, c, stencil, err, s);
}

size_t ensemble_member_bytes(int precision) {
  return precision == 0 ? sizeof(EnsembleMember<double>)
                        : (precision == 1 ? sizeof(EnsembleMember<float>) : sizeof(EnsembleMember<__half>));
}

void pack_ensemble_members(int precision, int n, const CUtensorMap* maps, void* const* pops,
                           const StepGeom* geoms, const StepCoef* coefs, void* host_out) {
  if (precision == 0) pack_members<double>(n, maps, pops, geoms, coefs, host_out);
  else if (precision == 1) pack_members<float>(n, maps, pops, geoms, coefs, host_out);
  else pack_members<__half>(n, maps, pops, geoms, coefs, host_out);
}

cudaError_t launch_ensemble_step(int precision, int stencil, const void* members, const int4* work,
                                 int nwork, int parity, unsigned long long* queue, int grid,
                                 unsigned* err, cudaStream_t s) {
  if (precision == 0) return launch_ens<double>(stencil, members, work, nwork, parity, queue, grid, err, s);
  if (precision == 1) return launch_ens<float>(stencil, members, work, nwork, parity, queue, grid, err, s);
  return launch_ens<__half>(stencil, members, work, nwork, parity, queue, grid, err, s);
}

int resident_step_blocks(int precision, int num_sms) {
  const int per_sm = precision == 0   ? StepConfig<double>::kMinBlocks
                     : precision == 1 ? StepConfig<float>::kMinBlocks
                                      : StepConfig<__half>::kMinBlocks;  // binary16, both forms
  return num_sms * per_sm;
}

// Rows per block: with the blocks that fit on the GPU at once (`resident`), give every strip
// floor(resident / strips) bands so the whole grid runs in one wave; never fewer than
// LBMHD_MIN_BAND rows.
int step_band_rows(int nx, int ny, int precision, int num_sms) {
  const int strips = (nx + kStepThreads - 1) / kStepThreads;
  const int per_sm = precision == 0   ? StepConfig<double>::kMinBlocks
                     : precision == 1 ? StepConfig<float>::kMinBlocks
                                      : StepConfig<__half>::kMinBlocks;  // binary16, both forms
  const long resident = (long)num_sms * per_sm * LBMHD_WAVES;
  long bands = resident / strips;
  if (bands < 1) bands = 1;
  long band = (ny + bands - 1) / bands;
  if (band < LBMHD_MIN_BAND) band = LBMHD_MIN_BAND;
  if (band > ny) band = ny;
  return (int)band;
}

}  // namespace lbmhd_gpu
