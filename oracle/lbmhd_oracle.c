/*
 * Plain FP64 CPU oracle for one time step of the filtered (LES) lattice Boltzmann MHD
 * model of Flint & Vahala, "A large eddy lattice Boltzmann simulation of
 * magnetohydrodynamic turbulence" (arXiv:1705.09807).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library.  It shares no code, header, table or constant with
 * the CUDA path: every matrix below is typed in from the paper, every equilibrium is the
 * paper's table written out, and the step runs in the order the paper states it.  It is
 * deliberately slow: dense 9x9 transforms, full-grid temporaries, no fusion.
 *
 * Citations use the paper's section and its equation labels:
 *   Sec. 2   Eq. LBKinEqn / LBMagEqn   kinetic equations for f_i and g_i (MRT / SRT)
 *            Eq. feq / geq            equilibrium distributions
 *            Eq. Transformation       moments M = T f, N = T_m g
 *            Eq. FluidTMatrix / MagTMatrix   the matrices T and T_m
 *            Eq. KinMomentEq / MagMomentEq   equilibrium moments M^eq, N^eq
 *            nu / xi / eta relations (after Eq. FinalLESeq)
 *   Sec. 2.1 Eq. FilterExampleSmall / FilterExampleLarge  filtered products to O(Delta^2)
 *            filtered M_3^eq example
 *   Sec. 3   SRT restriction, density gradients neglected, simplified filtered M_3^eq
 *
 * Readings of places where the paper is silent (each also listed in the design notes):
 *   R1  weights w_i = w'_i = {4/9, 1/9 x4, 1/36 x4} (the paper says "appropriate").
 *   R2  N^eq uses u = J/rho in the products (Eq. geq and the induction equation use u).
 *   R5  gradients d_beta by finite differences on the periodic grid: central 2-point
 *       (stencil 0) or the isotropic 9-point d_beta a = sum_i 3 w_i c_i,beta a(x+c_i) (stencil 1).
 *   R6  gradients are taken of J = rho u (Sec. 3 writes d_beta(rho u)).
 *   R7  gradients use the current (post-stream, pre-collision) moments of the same step.
 *   R9  one step = collide then stream; the stored state is the post-stream populations.
 *   Filtered products drop every d(rho) term (Sec. 3).
 *
 * Rounding: IEEE binary64, round to nearest; build with -O2 -ffp-contract=off, never
 * -ffast-math.  The threaded step splits rows only; per-cell arithmetic is identical for
 * any thread count, so results are bitwise independent of nthreads.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* ---- lattice: Sec. 2, the velocity lists after Eq. MagTMatrix ---------------------- */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
/* R1: standard D2Q9 weights for both w_i (Eq. feq) and w'_i (Eq. geq) */
static const double WGT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* ---- Eq. FluidTMatrix, as printed -------------------------------------------------- */
static const double TF[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},         {0, 1, 0, -1, 0, 1, -1, -1, 1},
    {0, 0, 1, 0, -1, 1, 1, -1, -1},      {0, 0, 0, 0, 0, 1, -1, 1, -1},
    {0, 1, -1, 1, -1, 0, 0, 0, 0},       {0, -2, 0, 2, 0, 1, -1, -1, 1},
    {0, 0, -2, 0, 2, 1, 1, -1, -1},      {4, -5, -5, -5, -5, 4, 4, 4, 4},
    {4, 0, 0, 0, 0, -1, -1, -1, -1}};
/* ---- Eq. MagTMatrix, as printed ---------------------------------------------------- */
static const double TMAG[9][9] = {
    {1, 1, 1, 1, 1, 1, 1, 1, 1},   {0, 1, 0, -1, 0, 1, -1, -1, 1}, {0, 0, 1, 0, -1, 1, 1, -1, -1},
    {0, 0, 0, 0, 0, 1, -1, 1, -1}, {0, 1, 0, 1, 0, 1, 1, 1, 1},    {0, 0, 1, 0, 1, 1, 1, 1, 1},
    {0, 0, 0, 0, 0, 1, 1, -1, -1}, {0, 0, 0, 0, 0, 1, -1, -1, 1},  {0, 0, 0, 0, 0, 1, 1, 1, 1}};

static double TF_INV[9][9];
static double TMAG_INV[9][9];
static int g_inverses_ready = 0;
static pthread_once_t g_once = PTHREAD_ONCE_INIT;

/* Gauss-Jordan elimination with partial pivoting in long double.  Both matrices are
 * "1-1" (invertible, Sec. 2 after Eq. Transformation); returns 0 if a pivot vanishes. */
static int invert9(const double A[9][9], double Ainv[9][9]) {
  long double a[9][18];
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c) a[r][c] = (c < 9) ? (long double)A[r][c] : (c - 9 == r ? 1.0L : 0.0L);
  for (int col = 0; col < 9; ++col) {
    int piv = col;
    for (int r = col + 1; r < 9; ++r)
      if (fabsl(a[r][col]) > fabsl(a[piv][col])) piv = r;
    if (fabsl(a[piv][col]) < 1e-30L) return 0;
    if (piv != col)
      for (int c = 0; c < 18; ++c) {
        long double t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
      }
    long double p = a[col][col];
    for (int c = 0; c < 18; ++c) a[col][c] /= p;
    for (int r = 0; r < 9; ++r) {
      if (r == col) continue;
      long double m = a[r][col];
      if (m == 0.0L) continue;
      for (int c = 0; c < 18; ++c) a[r][c] -= m * a[col][c];
    }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) Ainv[r][c] = (double)a[r][c + 9];
  return 1;
}

static void make_inverses(void) {
  int ok = invert9(TF, TF_INV) && invert9(TMAG, TMAG_INV);
  g_inverses_ready = ok ? 1 : -1;
}

static int ensure_inverses(void) {
  pthread_once(&g_once, make_inverses);
  return g_inverses_ready == 1;
}

/* Export of every table the oracle uses, so the tests can hold them against the paper. */
int oracle_tables(int* cx, int* cy, double* w, double* T, double* Tm, double* Tinv, double* Tminv) {
  if (!ensure_inverses()) return -1;
  for (int i = 0; i < 9; ++i) {
    cx[i] = CX[i];
    cy[i] = CY[i];
    w[i] = WGT[i];
    for (int j = 0; j < 9; ++j) {
      T[9 * i + j] = TF[i][j];
      Tm[9 * i + j] = TMAG[i][j];
      Tinv[9 * i + j] = TF_INV[i][j];
      Tminv[9 * i + j] = TMAG_INV[i][j];
    }
  }
  return 0;
}

/* ---- Eq. feq: fluid equilibrium distribution ---------------------------------------- */
void oracle_feq(double rho, double ux, double uy, double bx, double by, double* feq) {
  double usq = ux * ux + uy * uy;
  double bsq = bx * bx + by * by;
  for (int i = 0; i < 9; ++i) {
    double cu = CX[i] * ux + CY[i] * uy;
    double cb = CX[i] * bx + CY[i] * by;
    double csq = (double)(CX[i] * CX[i] + CY[i] * CY[i]);
    feq[i] = WGT[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq) +
             4.5 * WGT[i] * (0.5 * bsq * csq - cb * cb);
  }
}

/* ---- Eq. geq: magnetic equilibrium distribution, geq[alpha*9 + i] ------------------- */
void oracle_geq(double ux, double uy, double bx, double by, double* geq) {
  double B[2] = {bx, by}, U[2] = {ux, uy};
  for (int a = 0; a < 2; ++a)
    for (int i = 0; i < 9; ++i) {
      double cu = CX[i] * ux + CY[i] * uy;
      double cb = CX[i] * bx + CY[i] * by;
      geq[a * 9 + i] = WGT[i] * (B[a] + 3.0 * (cu * B[a] - cb * U[a]));
    }
}

/* ---- filtered products, Sec. 2.1 with Sec. 3's simplification ----------------------
 * Eq. FilterExampleSmall:  bar(XY)   = Xb Yb + (Delta^2/12) d_b Xb d_b Yb
 * Eq. FilterExampleLarge:  bar(XY/Z) = Xb Yb / Zb + (Delta^2/(12 Zb)) d_b Xb d_b Yb
 *                                       - (terms in d_b Zb), dropped: Sec. 3 neglects
 *                                         filtered density gradients.
 * gX[beta], gY[beta] are d_beta of X and Y at the cell; kd = Delta^2/12. */
static double filt_prod(double X, double Y, const double* gX, const double* gY, double kd) {
  return X * Y + kd * (gX[0] * gY[0] + gX[1] * gY[1]);
}
static double filt_ratio(double X, double Y, double Z, const double* gX, const double* gY,
                         double kd) {
  return X * Y / Z + kd / Z * (gX[0] * gY[0] + gX[1] * gY[1]);
}

/* ---- Eq. KinMomentEq with the Delta^2 terms of Sec. 2.1 / Sec. 3 -----------------------
 * M^eq as the printed table, with every nonlinear product replaced by its filtered form:
 *   (rho u_a)(rho u_b)/rho  -> filt_ratio(J_a, J_b, rho)
 *   B_a B_b                 -> filt_prod(B_a, B_b)
 * J[a], B[a]: filtered J = rho u and B at the cell;  gJ[a][beta] = d_beta J_a,
 * gB[a][beta] = d_beta B_a;  kd = Delta^2/12.  Delta = 0 gives the table exactly. */
static void meq_corrected(double rho, const double* J, const double* B, const double* gJ,
                          const double* gB, double kd, const double* cq, double* M);

void oracle_meq(double rho, const double* J, const double* B, const double* gJ,
                const double* gB, double kd, double* M) {
  meq_corrected(rho, J, B, gJ, gB, kd, NULL, M);
}

/* As oracle_meq, plus an optional additive correction cq[0..3] of the four subgrid terms:
 * cq[0] is added to the xy stress (M_3), cq[1] to the normal-stress difference (M_4), cq[2] to
 * the trace (J_x^2 + J_y^2)/rho that M_7 and M_8 carry with factor -3. */
static void meq_corrected(double rho, const double* J, const double* B, const double* gJ,
                          const double* gB, double kd, const double* cq, double* M) {
  const double* gJx = gJ;
  const double* gJy = gJ + 2;
  const double* gBx = gB;
  const double* gBy = gB + 2;
  double JxJy = filt_ratio(J[0], J[1], rho, gJx, gJy, kd);
  double JxJx = filt_ratio(J[0], J[0], rho, gJx, gJx, kd);
  double JyJy = filt_ratio(J[1], J[1], rho, gJy, gJy, kd);
  double BxBy = filt_prod(B[0], B[1], gBx, gBy, kd);
  double BxBx = filt_prod(B[0], B[0], gBx, gBx, kd);
  double ByBy = filt_prod(B[1], B[1], gBy, gBy, kd);
  M[0] = rho;                                  /* M_0^eq = M_0 = rho      */
  M[1] = J[0];                                 /* M_1^eq = M_1 = rho u_x  */
  M[2] = J[1];                                 /* M_2^eq = M_2 = rho u_y  */
  M[3] = JxJy - BxBy;                          /* (rho u_x rho u_y)/rho - B_x B_y */
  M[4] = JxJx - JyJy - BxBx + ByBy;            /* ((rho u_x)^2-(rho u_y)^2)/rho - B_x^2 + B_y^2 */
  M[5] = -J[0];                                /* -rho u_x */
  M[6] = -J[1];                                /* -rho u_y */
  M[7] = -3.0 * (JxJx + JyJy);                 /* -3((rho u_x)^2+(rho u_y)^2)/rho */
  M[8] = 5.0 / 3.0 * rho - 3.0 * (JxJx + JyJy); /* 5/3 rho - 3(...)/rho */
  if (cq) {
    M[3] += cq[0];
    M[4] += cq[1];
    M[7] -= 3.0 * cq[2];
    M[8] -= 3.0 * cq[2];
  }
}

/* ---- Eq. MagMomentEq with the Delta^2 terms ------------------------------------------
 * N^eq_{alpha q} as the printed table, with u = J/rho (R2), so each product
 * u_beta B_alpha = (rho u_beta) B_alpha / rho is filtered by Eq. FilterExampleLarge.
 * N[alpha*9 + q]. */
static void neq_corrected(double rho, const double* J, const double* B, const double* gJ,
                          const double* gB, double kd, const double* cq, double* N);

void oracle_neq(double rho, const double* J, const double* B, const double* gJ,
                const double* gB, double kd, double* N) {
  neq_corrected(rho, J, B, gJ, gB, kd, NULL, N);
}

/* As oracle_neq, plus an optional correction cq[3] of the electric field
 * E = P[x][y] - P[y][x] (added to P[x][y], so every N entry carrying E receives it). */
static void neq_corrected(double rho, const double* J, const double* B, const double* gJ,
                          const double* gB, double kd, const double* cq, double* N) {
  /* P[b][a] = filtered (rho u_b) B_a / rho */
  double P[2][2];
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) P[b][a] = filt_ratio(J[b], B[a], rho, gJ + 2 * b, gB + 2 * a, kd);
  if (cq) P[0][1] += cq[3];
  for (int a = 0; a < 2; ++a) {
    double* Na = N + 9 * a;
    Na[0] = B[a];                          /* N_a0 = B_a */
    Na[1] = P[0][a] - P[a][0];             /* rho u_x B_a - rho u_a B_x (over rho) */
    Na[2] = P[1][a] - P[a][1];             /* rho u_y B_a - rho u_a B_y (over rho) */
    Na[3] = 0.0;                           /* N_a3 = 0 */
    Na[4] = B[a] / 3.0;                    /* N_a4 = B_a/3 */
    Na[5] = B[a] / 3.0;                    /* N_a5 = B_a/3 */
    Na[6] = (P[1][a] - P[a][1]) / 3.0;     /* (rho u_y B_a - rho u_a B_y)/3 */
    Na[7] = (P[0][a] - P[a][0]) / 3.0;     /* (rho u_x B_a - rho u_a B_x)/3 */
    Na[8] = B[a] / 9.0;                    /* N_a8 = B_a/9 */
  }
}

/* ---- moments of the populations at one cell (Sec. 2, after Eq. LBMagEqn) ----------- */
static void cell_moments(const double* f, const double* g, size_t ncell, size_t c, double* rho,
                         double* J, double* B) {
  double r = 0.0, jx = 0.0, jy = 0.0, bx = 0.0, by = 0.0;
  for (int i = 0; i < 9; ++i) {
    double fi = f[(size_t)i * ncell + c];
    r += fi;
    jx += fi * CX[i];
    jy += fi * CY[i];
    bx += g[(size_t)i * ncell + c];
    by += g[(size_t)(9 + i) * ncell + c];
  }
  *rho = r;
  J[0] = jx;
  J[1] = jy;
  B[0] = bx;
  B[1] = by;
}

static inline int wrap(int i, int n) {
  int r = i % n;
  return r < 0 ? r + n : r;
}

/* d_beta of a scalar field at (x, y) by the chosen stencil (R5). */
static void field_gradient(const double* a, int nx, int ny, int x, int y, int stencil,
                           double* d) {
  if (stencil == 0) {
    d[0] = 0.5 * (a[(size_t)y * nx + wrap(x + 1, nx)] - a[(size_t)y * nx + wrap(x - 1, nx)]);
    d[1] = 0.5 * (a[(size_t)wrap(y + 1, ny) * nx + x] - a[(size_t)wrap(y - 1, ny) * nx + x]);
  } else {
    double sx = 0.0, sy = 0.0;
    for (int i = 1; i < 9; ++i) {
      double v = a[(size_t)wrap(y + CY[i], ny) * nx + wrap(x + CX[i], nx)];
      sx += 3.0 * WGT[i] * CX[i] * v;
      sy += 3.0 * WGT[i] * CY[i] * v;
    }
    d[0] = sx;
    d[1] = sy;
  }
}

/* Collision of one cell in moment space (Sec. 2 after Eq. geq; Eq. Transformation):
 *   M = T f,  N_a = T_m g_a
 *   M*_j = M_j - s_j (M_j - Mbar^eq_j)        (MRT, Eq. LBKinEqn)
 *   N*_aj = N_aj - s_m (N_aj - Nbar^eq_aj)    (SRT, Eq. LBMagEqn)
 *   f* = T^{-1} M*,  g*_a = T_m^{-1} N*_a.                                                */
static void collide_cell(const double* fc, const double* gc, double rho, const double* J,
                         const double* B, const double* gJ, const double* gB, const double* s,
                         double s_m, double kd, const double* cq, double* fstar, double* gstar) {
  double M[9], Meq[9], Ms[9], N[18], Neq[18], Ns[18];
  for (int j = 0; j < 9; ++j) {
    double acc = 0.0;
    for (int i = 0; i < 9; ++i) acc += TF[j][i] * fc[i];
    M[j] = acc;
  }
  for (int a = 0; a < 2; ++a)
    for (int j = 0; j < 9; ++j) {
      double acc = 0.0;
      for (int i = 0; i < 9; ++i) acc += TMAG[j][i] * gc[9 * a + i];
      N[9 * a + j] = acc;
    }
  meq_corrected(rho, J, B, gJ, gB, kd, cq, Meq);
  neq_corrected(rho, J, B, gJ, gB, kd, cq, Neq);
  for (int j = 0; j < 9; ++j) Ms[j] = M[j] - s[j] * (M[j] - Meq[j]);
  for (int q = 0; q < 18; ++q) Ns[q] = N[q] - s_m * (N[q] - Neq[q]);
  for (int i = 0; i < 9; ++i) {
    double acc = 0.0;
    for (int j = 0; j < 9; ++j) acc += TF_INV[i][j] * Ms[j];
    fstar[i] = acc;
  }
  for (int a = 0; a < 2; ++a)
    for (int i = 0; i < 9; ++i) {
      double acc = 0.0;
      for (int j = 0; j < 9; ++j) acc += TMAG_INV[i][j] * Ns[9 * a + j];
      gstar[9 * a + i] = acc;
    }
}

/* ---- full-grid step ------------------------------------------------------------------ */
typedef struct {
  int nx, ny, y0, y1, stencil;
  const double *f, *g, *rho, *jx, *jy, *bx, *by, *s;
  double s_m, kd;
  double *fs, *gs;
  const double* corr; /* optional correction planes [4][ny][nx] */
} row_job;

static void gather_cell(const double* f, const double* g, size_t ncell, size_t c, double* fc,
                        double* gc) {
  for (int i = 0; i < 9; ++i) {
    fc[i] = f[(size_t)i * ncell + c];
    gc[i] = g[(size_t)i * ncell + c];
    gc[9 + i] = g[(size_t)(9 + i) * ncell + c];
  }
}

static void* collide_rows(void* arg) {
  row_job* jb = (row_job*)arg;
  size_t ncell = (size_t)jb->nx * jb->ny;
  for (int y = jb->y0; y < jb->y1; ++y)
    for (int x = 0; x < jb->nx; ++x) {
      size_t c = (size_t)y * jb->nx + x;
      double fc[9], gc[18], fst[9], gst[18], J[2], B[2], gJ[4], gB[4];
      gather_cell(jb->f, jb->g, ncell, c, fc, gc);
      J[0] = jb->jx[c];
      J[1] = jb->jy[c];
      B[0] = jb->bx[c];
      B[1] = jb->by[c];
      field_gradient(jb->jx, jb->nx, jb->ny, x, y, jb->stencil, gJ);
      field_gradient(jb->jy, jb->nx, jb->ny, x, y, jb->stencil, gJ + 2);
      field_gradient(jb->bx, jb->nx, jb->ny, x, y, jb->stencil, gB);
      field_gradient(jb->by, jb->nx, jb->ny, x, y, jb->stencil, gB + 2);
      double cq[4];
      if (jb->corr)
        for (int q = 0; q < 4; ++q) cq[q] = jb->corr[(size_t)q * ncell + c];
      collide_cell(fc, gc, jb->rho[c], J, B, gJ, gB, jb->s, jb->s_m, jb->kd, jb->corr ? cq : NULL,
                   fst, gst);
      for (int i = 0; i < 9; ++i) {
        jb->fs[(size_t)i * ncell + c] = fst[i];
        jb->gs[(size_t)i * ncell + c] = gst[i];
        jb->gs[(size_t)(9 + i) * ncell + c] = gst[9 + i];
      }
    }
  return NULL;
}

static int check_args(int nx, int ny, const double* s, double s_m, double delta, int stencil) {
  if (nx < 3 || ny < 3) return -1;
  if (!s || !(delta >= 0.0)) return -1;
  if (stencil != 0 && stencil != 1) return -1;
  for (int j = 3; j < 9; ++j)
    if (!(s[j] > 0.0 && s[j] < 2.0)) return -1;
  if (!(s_m > 0.0 && s_m < 2.0)) return -1;
  return 0;
}

/* Advance f[9][ny][nx], g[2][9][ny][nx] (post-stream populations) by nsteps steps.
 * Each step (Sec. 3: collide in moment space, stream in distribution space):
 *   1 moments rho, J, B of every cell          (Sec. 2, after Eq. LBMagEqn)
 *   2 gradients d_beta J_a, d_beta B_a         (R5, R6, R7)
 *   3 collide every cell in moment space        (collide_cell)
 *   4 stream: f_i(x + c_i) <- f*_i(x), periodic (left side of Eq. LBKinEqn / LBMagEqn)
 * s[9]: fluid rates in the order of the rows of T (s[0..2] act on conserved moments and do
 * not change the result); s_m: magnetic rate; delta: filter width (kd = delta^2/12).
 * Returns 0, or -1 on invalid arguments, -3 if memory runs out. */
static int step_impl(int nx, int ny, const double* s, double s_m, double delta, int stencil,
                     double* f, double* g, int nsteps, int nthreads, const double* corr);

int oracle_step(int nx, int ny, const double* s, double s_m, double delta, int stencil,
                double* f, double* g, int nsteps, int nthreads) {
  return step_impl(nx, ny, s, s_m, delta, stencil, f, g, nsteps, nthreads, NULL);
}

/* oracle_step with a fixed additive correction of the four subgrid terms at every cell and
 * step: corr[4][ny][nx] = (xy stress, normal-stress difference, trace, electric field). */
int oracle_step_corrected(int nx, int ny, const double* s, double s_m, double delta, int stencil,
                          double* f, double* g, int nsteps, int nthreads, const double* corr) {
  if (!corr) return -1;
  return step_impl(nx, ny, s, s_m, delta, stencil, f, g, nsteps, nthreads, corr);
}

static int step_impl(int nx, int ny, const double* s, double s_m, double delta, int stencil,
                     double* f, double* g, int nsteps, int nthreads, const double* corr) {
  if (check_args(nx, ny, s, s_m, delta, stencil) || !f || !g || nsteps < 0) return -1;
  if (!ensure_inverses()) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > ny) nthreads = ny;
  size_t ncell = (size_t)nx * ny;
  double* rho = malloc(ncell * sizeof(double));
  double* jx = malloc(ncell * sizeof(double));
  double* jy = malloc(ncell * sizeof(double));
  double* bx = malloc(ncell * sizeof(double));
  double* by = malloc(ncell * sizeof(double));
  double* fs = malloc(9 * ncell * sizeof(double));
  double* gs = malloc(18 * ncell * sizeof(double));
  row_job* jobs = malloc((size_t)nthreads * sizeof(row_job));
  pthread_t* th = malloc((size_t)nthreads * sizeof(pthread_t));
  int rc = 0;
  if (!rho || !jx || !jy || !bx || !by || !fs || !gs || !jobs || !th) {
    rc = -3;
    goto done;
  }
  double kd = delta * delta / 12.0;
  for (int n = 0; n < nsteps; ++n) {
    /* 1. moments */
    for (size_t c = 0; c < ncell; ++c) {
      double J[2], B[2];
      cell_moments(f, g, ncell, c, &rho[c], J, B);
      jx[c] = J[0];
      jy[c] = J[1];
      bx[c] = B[0];
      by[c] = B[1];
    }
    /* 2 + 3. gradients and collision, rows split over threads */
    for (int t = 0; t < nthreads; ++t) {
      row_job jb = {nx, ny, (int)((long)ny * t / nthreads), (int)((long)ny * (t + 1) / nthreads),
                    stencil, f, g, rho, jx, jy, bx, by, s, s_m, kd, fs, gs, corr};
      jobs[t] = jb;
    }
    if (nthreads == 1) {
      collide_rows(&jobs[0]);
    } else {
      int started = 0;
      for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, collide_rows, &jobs[t]) != 0) break;
        ++started;
      }
      for (int t = started; t < nthreads; ++t) collide_rows(&jobs[t]);
      for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    }
    /* 4. stream */
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t c = (size_t)y * nx + x;
        for (int i = 0; i < 9; ++i) {
          size_t d = (size_t)wrap(y + CY[i], ny) * nx + wrap(x + CX[i], nx);
          f[(size_t)i * ncell + d] = fs[(size_t)i * ncell + c];
          g[(size_t)i * ncell + d] = gs[(size_t)i * ncell + c];
          g[(size_t)(9 + i) * ncell + d] = gs[(size_t)(9 + i) * ncell + c];
        }
      }
  }
done:
  free(rho);
  free(jx);
  free(jy);
  free(bx);
  free(by);
  free(fs);
  free(gs);
  free(jobs);
  free(th);
  return rc;
}

/* Post-collision populations f*, g* of the single cell (x, y) for the current state, the
 * same arithmetic as one cell of oracle_step's step 3.  It needs only the 3x3 (central
 * stencil: plus-shaped) neighbourhood, so large grids can be checked at sampled cells. */
int oracle_collide_cell(int nx, int ny, const double* s, double s_m, double delta, int stencil,
                        const double* f, const double* g, int x, int y, double* fstar,
                        double* gstar) {
  if (check_args(nx, ny, s, s_m, delta, stencil) || !f || !g || x < 0 || y < 0 || x >= nx ||
      y >= ny)
    return -1;
  if (!ensure_inverses()) return -1;
  size_t ncell = (size_t)nx * ny;
  /* moments on the 3x3 neighbourhood, then gradients from it */
  double nb[5][3][3];
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      size_t c = (size_t)wrap(y + dy, ny) * nx + wrap(x + dx, nx);
      double r, J[2], B[2];
      cell_moments(f, g, ncell, c, &r, J, B);
      nb[0][dy + 1][dx + 1] = r;
      nb[1][dy + 1][dx + 1] = J[0];
      nb[2][dy + 1][dx + 1] = J[1];
      nb[3][dy + 1][dx + 1] = B[0];
      nb[4][dy + 1][dx + 1] = B[1];
    }
  double grad[4][2];
  for (int q = 0; q < 4; ++q) {
    /* the 3x3 patch as a periodic 3x3 "grid" centred at (1, 1) gives the same stencil */
    double patch[9];
    for (int yy = 0; yy < 3; ++yy)
      for (int xx = 0; xx < 3; ++xx) patch[yy * 3 + xx] = nb[q + 1][yy][xx];
    field_gradient(patch, 3, 3, 1, 1, stencil, grad[q]);
  }
  size_t c = (size_t)y * nx + x;
  double fc[9], gc[18];
  gather_cell(f, g, ncell, c, fc, gc);
  double J[2] = {nb[1][1][1], nb[2][1][1]}, B[2] = {nb[3][1][1], nb[4][1][1]};
  double gJ[4] = {grad[0][0], grad[0][1], grad[1][0], grad[1][1]};
  double gB[4] = {grad[2][0], grad[2][1], grad[3][0], grad[3][1]};
  collide_cell(fc, gc, nb[0][1][1], J, B, gJ, gB, s, s_m, delta * delta / 12.0, NULL, fstar, gstar);
  return 0;
}

/* Initial state (reading R8): f_i = f_i^eq(rho, u, B) (Eq. feq), g_i = g_i^eq(u, B) (Eq. geq),
 * no Delta terms.  Fields are [ny][nx], x fastest. */
int oracle_init(int nx, int ny, const double* rho, const double* ux, const double* uy,
                const double* bx, const double* by, double* f, double* g) {
  if (nx < 1 || ny < 1 || !rho || !ux || !uy || !bx || !by || !f || !g) return -1;
  size_t ncell = (size_t)nx * ny;
  for (size_t c = 0; c < ncell; ++c) {
    double fe[9], ge[18];
    oracle_feq(rho[c], ux[c], uy[c], bx[c], by[c], fe);
    oracle_geq(ux[c], uy[c], bx[c], by[c], ge);
    for (int i = 0; i < 9; ++i) {
      f[(size_t)i * ncell + c] = fe[i];
      g[(size_t)i * ncell + c] = ge[i];
      g[(size_t)(9 + i) * ncell + c] = ge[9 + i];
    }
  }
  return 0;
}

/* Macroscopic fields of the current populations: rho, u = J/rho, B. */
int oracle_moments(int nx, int ny, const double* f, const double* g, double* rho, double* ux,
                   double* uy, double* bx, double* by) {
  if (nx < 1 || ny < 1 || !f || !g || !rho || !ux || !uy || !bx || !by) return -1;
  size_t ncell = (size_t)nx * ny;
  for (size_t c = 0; c < ncell; ++c) {
    double r, J[2], B[2];
    cell_moments(f, g, ncell, c, &r, J, B);
    rho[c] = r;
    ux[c] = J[0] / r;
    uy[c] = J[1] / r;
    bx[c] = B[0];
    by[c] = B[1];
  }
  return 0;
}
