/*
 * cg_oracle.c -- FP64 CPU oracle for the two-component colour-gradient LBM
 * on D3Q27 with central-moment MRT collision (arXiv 2309.07801).
 *
 * TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library; the product path never does.
 *
 * Everything here is written from the definitions, in the paper's order and
 * notation, with no factorisation, fusion or reordering:
 *   - equilibria in phase space from the Hermite expansion (Sec. III, App. B);
 *   - raw/central moments as the sums of Sec. II.B (Eqs. for m and k);
 *   - the collision of Eq. (general form) in Sec. II.B, each group of
 *     combined moments solved for the individual moments;
 *   - back to populations by the binomial shift of the central moments and a
 *     brute-force Gauss-Jordan inverse of the 27x27 raw-moment matrix;
 *   - recoloring of Sec. II.A (Eqs. recoloring and R), pull streaming, and
 *     fullway bounce-back at solid cells (Sec. IV).
 *
 * Readings of points the paper leaves open:
 *   - (c_s^k)^2 = xi (1 - alpha_k) (the stray rho_k in Sec. II.A dropped);
 *   - the lattice c_s^2 = 1/3 everywhere except the equation of state;
 *   - Q_a = -3 d_a[(p - rho c_s^2) u_a] component by component (Sec. III.E);
 *   - kappa = -(d_a n_a - n_a n_b d_a n_b), every derivative with the
 *     isotropic difference of Sec. II.A applied to the stored field;
 *   - n = 0 where |grad phi|^2 <= 1e-24;
 *   - at a solid neighbour the stencils take the centre cell's phi and n
 *     and zero for (p - rho c_s^2) u;
 *   - the initial state is the post-collision state
 *     f^k_i = (rho_k/rho) f^eq_i(rho, p, u); the first step starts by streaming;
 *   - solid cells keep what streams in, reverse it, and do not collide.
 */
#include "cg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- lattice (Sec. II.A) ------------------------------------------------ */

/* D3Q27 velocities in the printed order */
static const int CI[27][3] = {
    {0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
    {-1, 1, 0},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1},
    {1, 0, 1},   {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},  {1, 1, 1},
    {-1, -1, -1},{1, 1, -1},  {-1, -1, 1}, {1, -1, 1},  {-1, 1, -1},
    {-1, 1, 1},  {1, -1, -1}};

static const double CS2 = 1.0 / 3.0;  /* lattice speed of sound squared */
static const double XI = 9.0 / 19.0;  /* D3Q27 rest-weight parameter */
static const double NORMAL_EPS = 1e-24;

static double weight_of(int i) {
  int c2 = CI[i][0] * CI[i][0] + CI[i][1] * CI[i][1] + CI[i][2] * CI[i][2];
  switch (c2) {
    case 0: return 8.0 / 27.0;
    case 1: return 2.0 / 27.0;
    case 2: return 1.0 / 54.0;
    default: return 1.0 / 216.0;
  }
}

/* tables filled once: weights, opposites, Hermite polynomials H[i][a+3b+9c] */
static double WT[27];
static int OPP[27];
static double HT[27][27];
static int TABLES_READY = 0;
static void ensure_tables(void);

static double weight(int i) { return WT[i]; }

static int opposite(int i) { return OPP[i]; }

static int opposite_of(int i) {
  for (int j = 0; j < 27; ++j)
    if (CI[j][0] == -CI[i][0] && CI[j][1] == -CI[i][1] && CI[j][2] == -CI[i][2])
      return j;
  return -1;
}

void ocg_lattice(int32_t *c, double *w) {
  ensure_tables();
  for (int i = 0; i < 27; ++i) {
    for (int a = 0; a < 3; ++a) c[3 * i + a] = CI[i][a];
    w[i] = weight(i);
  }
}

static int K(int a, int b, int c) { return a + 3 * b + 9 * c; }

static double ipow(double x, int e) {
  double r = 1.0;
  for (int k = 0; k < e; ++k) r *= x;
  return r;
}

/* ---- Hermite polynomials (App. B) ---------------------------------------- */

static double h1d(int order, int c) {
  if (order == 0) return 1.0;
  if (order == 1) return (double)c;
  return (double)(c * c) - CS2;
}

double ocg_hermite(int i, int a, int b, int c) {
  return h1d(a, CI[i][0]) * h1d(b, CI[i][1]) * h1d(c, CI[i][2]);
}

static void ensure_tables(void) {
  if (TABLES_READY) return;
#ifdef _OPENMP
#pragma omp critical(ocg_tables)
#endif
  {
    if (!TABLES_READY) {
      for (int i = 0; i < 27; ++i) {
        WT[i] = weight_of(i);
        OPP[i] = opposite_of(i);
        for (int c = 0; c < 3; ++c)
          for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) HT[i][K(a, b, c)] = ocg_hermite(i, a, b, c);
      }
      TABLES_READY = 1;
    }
  }
}

#define H(a, b, c) HT[i][K(a, b, c)]

/* g^{eq,2}, Eq. (equilibria for standard LBM, 2nd order) */
static double g2(int i, double rho, const double u[3]) {
  double cu = CI[i][0] * u[0] + CI[i][1] * u[1] + CI[i][2] * u[2];
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  return rho * weight(i) *
         (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
}

/* g^{eq,6}, Eq. (equilibria for standard LBM, 6th order), term by term */
static double g6(int i, double rho, const double u[3]) {
  const double ux = u[0], uy = u[1], uz = u[2];
  const double cs4 = CS2 * CS2, cs6 = cs4 * CS2, cs8 = cs6 * CS2,
               cs10 = cs8 * CS2, cs12 = cs10 * CS2;
  double t1 = (ux * H(1, 0, 0) + uy * H(0, 1, 0) + uz * H(0, 0, 1)) / CS2;
  double t2 = (ux * ux * H(2, 0, 0) + uy * uy * H(0, 2, 0) + uz * uz * H(0, 0, 2) +
               2.0 * (ux * uy * H(1, 1, 0) + uy * uz * H(0, 1, 1) +
                      ux * uz * H(1, 0, 1))) /
              (2.0 * cs4);
  double t3 = (ux * ux * uy * H(2, 1, 0) + ux * ux * uz * H(2, 0, 1) +
               ux * uy * uy * H(1, 2, 0) + ux * uz * uz * H(1, 0, 2) +
               uy * uz * uz * H(0, 1, 2) + uy * uy * uz * H(0, 2, 1) +
               2.0 * ux * uy * uz * H(1, 1, 1)) /
              (2.0 * cs6);
  double t4 = (ux * ux * uy * uy * H(2, 2, 0) + ux * ux * uz * uz * H(2, 0, 2) +
               uy * uy * uz * uz * H(0, 2, 2) +
               2.0 * (ux * uy * uz * uz * H(1, 1, 2) + ux * uy * uy * uz * H(1, 2, 1) +
                      ux * ux * uy * uz * H(2, 1, 1))) /
              (4.0 * cs8);
  double t5 = (ux * ux * uy * uz * uz * H(2, 1, 2) + ux * ux * uy * uy * uz * H(2, 2, 1) +
               ux * uy * uy * uz * uz * H(1, 2, 2)) /
              (4.0 * cs10);
  double t6 = ux * ux * uy * uy * uz * uz * H(2, 2, 2) / (8.0 * cs12);
  return rho * weight(i) * (1.0 + t1 + t2 + t3 + t4 + t5 + t6);
}

/* isotropic operator E_i, Eq. (isotropic operator) */
static double E_op(int i) {
  const double cs4 = CS2 * CS2, cs6 = cs4 * CS2, cs8 = cs6 * CS2;
  return weight(i) * ((H(2, 0, 0) + H(0, 2, 0) + H(0, 0, 2)) / (2.0 * cs4) -
                      (H(2, 2, 0) + H(0, 2, 2) + H(2, 0, 2)) / (4.0 * cs6) +
                      H(2, 2, 2) / (8.0 * cs8));
}

/* third-order part of the correction operator Phi_i (Li et al., Sec. III.C) */
static double phi3(int i, const double u[3]) {
  const double cs6 = CS2 * CS2 * CS2;
  return weight(i) *
         (u[0] * (H(1, 2, 0) + H(1, 0, 2)) + u[1] * (H(2, 1, 0) + H(0, 1, 2)) +
          u[2] * (H(2, 0, 1) + H(0, 2, 1))) /
         (2.0 * cs6);
}

/* full Phi_i of the generalized equilibria, Eq. of Sec. III.D */
static double phi6(int i, const double u[3]) {
  const double ux = u[0], uy = u[1], uz = u[2];
  const double cs4 = CS2 * CS2, cs8 = cs4 * cs4, cs10 = cs8 * CS2,
               cs12 = cs10 * CS2;
  double o4 = ((ux * ux + uy * uy) * H(2, 2, 0) + (uy * uy + uz * uz) * H(0, 2, 2) +
               (ux * ux + uz * uz) * H(2, 0, 2) +
               2.0 * (uy * uz * H(2, 1, 1) + ux * uz * H(1, 2, 1) +
                      ux * uy * H(1, 1, 2))) /
              (4.0 * cs8);
  double o5 = (ux * (uy * uy + uz * uz - CS2) * H(1, 2, 2) +
               uy * (ux * ux + uz * uz - CS2) * H(2, 1, 2) +
               uz * (ux * ux + uy * uy - CS2) * H(2, 2, 1)) /
              (4.0 * cs10);
  double o6 = (ux * ux * uy * uy + uy * uy * uz * uz + ux * ux * uz * uz -
               CS2 * (ux * ux + uy * uy + uz * uz)) *
              H(2, 2, 2) / (8.0 * cs12);
  return phi3(i, u) + weight(i) * (o4 + o5 + o6);
}

/* lattice-specific parameter varphi_i of Sec. II.A */
static double varphi(int i, double rho, double p) {
  if (i == 0) return 1.0 - p / (XI * rho);
  return weight(i) * p / (rho * CS2);
}

#undef H

void ocg_feq(int model, double rho, double p, const double u[3], double *feq) {
  ensure_tables();
  const double dev = p - rho * CS2; /* deviation from the ideal gas */
  const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 27; ++i) {
    double cu = CI[i][0] * u[0] + CI[i][1] * u[1] + CI[i][2] * u[2];
    double c2 = CI[i][0] * CI[i][0] + CI[i][1] * CI[i][1] + CI[i][2] * CI[i][2];
    switch (model) {
      case OCG_MODEL_A: feq[i] = g2(i, rho, u) + dev * E_op(i); break;
      case OCG_MODEL_B: feq[i] = g6(i, rho, u) + dev * E_op(i); break;
      case OCG_MODEL_C: feq[i] = g6(i, rho, u) + dev * (E_op(i) + phi3(i, u)); break;
      case OCG_MODEL_D: feq[i] = g6(i, rho, u) + dev * (E_op(i) + phi6(i, u)); break;
      case 4: feq[i] = g2(i, rho, u) + dev * (E_op(i) + phi3(i, u)); break;
      case 5:
        feq[i] = rho * (varphi(i, rho, p) +
                        weight(i) * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) -
                                     uu / (2.0 * CS2)));
        break;
      case 6:
        feq[i] = rho * (varphi(i, rho, p) +
                        weight(i) * (cu / CS2 + cu * cu / (2.0 * CS2 * CS2) -
                                     uu / (2.0 * CS2) +
                                     cu / (2.0 * CS2) * (p / (rho * CS2) - 1.0) *
                                         (c2 / CS2 - 3.0 - 2.0)));
        break;
      default: feq[i] = NAN;
    }
  }
}

/* ---- moments (Sec. II.B) -------------------------------------------------- */

void ocg_raw_moments(const double *f, double *m) {
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int i = 0; i < 27; ++i)
          s += f[i] * ipow(CI[i][0], a) * ipow(CI[i][1], b) * ipow(CI[i][2], c);
        m[K(a, b, c)] = s;
      }
}

void ocg_central_moments(const double *f, const double u[3], double *k) {
  /* pw[axis][c+1][e] = (c - u_axis)^e */
  double pw[3][3][3];
  for (int ax = 0; ax < 3; ++ax)
    for (int cv = -1; cv <= 1; ++cv)
      for (int e = 0; e < 3; ++e) pw[ax][cv + 1][e] = ipow(cv - u[ax], e);
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int i = 0; i < 27; ++i)
          s += f[i] * pw[0][CI[i][0] + 1][a] * pw[1][CI[i][1] + 1][b] *
               pw[2][CI[i][2] + 1][c];
        k[K(a, b, c)] = s;
      }
}

void ocg_moment_matrix(double *M) {
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 27; ++i)
          M[K(a, b, c) * 27 + i] =
              ipow(CI[i][0], a) * ipow(CI[i][1], b) * ipow(CI[i][2], c);
}

void ocg_moment_matrix_inverse(double *Minv) {
  double A[27][54];
  double M[27 * 27];
  ocg_moment_matrix(M);
  for (int r = 0; r < 27; ++r)
    for (int s = 0; s < 54; ++s)
      A[r][s] = (s < 27) ? M[r * 27 + s] : (s - 27 == r ? 1.0 : 0.0);
  for (int col = 0; col < 27; ++col) {
    int piv = col;
    for (int r = col + 1; r < 27; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    if (piv != col)
      for (int s = 0; s < 54; ++s) {
        double t = A[col][s];
        A[col][s] = A[piv][s];
        A[piv][s] = t;
      }
    double d = A[col][col];
    for (int s = 0; s < 54; ++s) A[col][s] /= d;
    for (int r = 0; r < 27; ++r) {
      if (r == col) continue;
      double fct = A[r][col];
      if (fct == 0.0) continue;
      for (int s = 0; s < 54; ++s) A[r][s] -= fct * A[col][s];
    }
  }
  for (int r = 0; r < 27; ++r)
    for (int s = 0; s < 27; ++s) Minv[r * 27 + s] = A[r][27 + s];
}

/* ---- collision, Eq. (general form) of Sec. II.B ---------------------------- */

void ocg_collide_cm(const double *k, const double *keq, const double *om,
                    const double F[3], const double Q[3], double *ks) {
  const double cs2 = CS2, cs4 = CS2 * CS2;
#define KK(a, b, c) k[K(a, b, c)]
#define KE(a, b, c) keq[K(a, b, c)]
#define KS(a, b, c) ks[K(a, b, c)]
  /* zeroth order: conserved */
  KS(0, 0, 0) = KK(0, 0, 0);
  /* first order */
  KS(1, 0, 0) = (1 - om[0]) * KK(1, 0, 0) + (1 - om[0] / 2) * F[0];
  KS(0, 1, 0) = (1 - om[0]) * KK(0, 1, 0) + (1 - om[0] / 2) * F[1];
  KS(0, 0, 1) = (1 - om[0]) * KK(0, 0, 1) + (1 - om[0] / 2) * F[2];
  /* second order, off-diagonal */
  KS(1, 1, 0) = (1 - om[1]) * KK(1, 1, 0) + om[1] * KE(1, 1, 0);
  KS(0, 1, 1) = (1 - om[1]) * KK(0, 1, 1) + om[1] * KE(0, 1, 1);
  KS(1, 0, 1) = (1 - om[1]) * KK(1, 0, 1) + om[1] * KE(1, 0, 1);
  /* second order, diagonal: two differences (omega_1) and the trace (omega_2) */
  {
    double d1 = (1 - om[1]) * (KK(2, 0, 0) - KK(0, 2, 0)) +
                om[1] * (KE(2, 0, 0) - KE(0, 2, 0)) + (1 - om[1] / 2) * (Q[0] - Q[1]);
    double d2 = (1 - om[1]) * (KK(2, 0, 0) - KK(0, 0, 2)) +
                om[1] * (KE(2, 0, 0) - KE(0, 0, 2)) + (1 - om[1] / 2) * (Q[0] - Q[2]);
    double tr = (1 - om[2]) * (KK(2, 0, 0) + KK(0, 2, 0) + KK(0, 0, 2)) +
                om[2] * (KE(2, 0, 0) + KE(0, 2, 0) + KE(0, 0, 2)) +
                (1 - om[2] / 2) * (Q[0] + Q[1] + Q[2]);
    /* solve k200-k020=d1, k200-k002=d2, k200+k020+k002=tr */
    double M3[3][4] = {{1, -1, 0, d1}, {1, 0, -1, d2}, {1, 1, 1, tr}};
    for (int col = 0; col < 3; ++col) {
      int piv = col;
      for (int r = col + 1; r < 3; ++r)
        if (fabs(M3[r][col]) > fabs(M3[piv][col])) piv = r;
      for (int s = 0; s < 4; ++s) {
        double t = M3[col][s];
        M3[col][s] = M3[piv][s];
        M3[piv][s] = t;
      }
      for (int r = 0; r < 3; ++r) {
        if (r == col) continue;
        double fct = M3[r][col] / M3[col][col];
        for (int s = 0; s < 4; ++s) M3[r][s] -= fct * M3[col][s];
      }
    }
    KS(2, 0, 0) = M3[0][3] / M3[0][0];
    KS(0, 2, 0) = M3[1][3] / M3[1][1];
    KS(0, 0, 2) = M3[2][3] / M3[2][2];
  }
  /* third order: sums (omega_3, with forcing) and differences (omega_4) */
  {
    const int pairs[3][2][3] = {{{1, 2, 0}, {1, 0, 2}},
                                {{2, 1, 0}, {0, 1, 2}},
                                {{2, 0, 1}, {0, 2, 1}}};
    for (int a = 0; a < 3; ++a) {
      const int *p1 = pairs[a][0], *p2 = pairs[a][1];
      double k1 = k[K(p1[0], p1[1], p1[2])], k2 = k[K(p2[0], p2[1], p2[2])];
      double e1 = keq[K(p1[0], p1[1], p1[2])], e2 = keq[K(p2[0], p2[1], p2[2])];
      double sum = (1 - om[3]) * (k1 + k2) + om[3] * (e1 + e2) +
                   2.0 * (1 - om[3] / 2) * F[a] * cs2;
      double dif = (1 - om[4]) * (k1 - k2) + om[4] * (e1 - e2);
      ks[K(p1[0], p1[1], p1[2])] = (sum + dif) / 2.0;
      ks[K(p2[0], p2[1], p2[2])] = (sum - dif) / 2.0;
    }
    KS(1, 1, 1) = (1 - om[5]) * KK(1, 1, 1) + om[5] * KE(1, 1, 1);
  }
  /* fourth order: two combinations with omega_6, the sum with omega_7 */
  {
    double A = (1 - om[6]) * (KK(2, 2, 0) - 2 * KK(2, 0, 2) + KK(0, 2, 2)) +
               om[6] * (KE(2, 2, 0) - 2 * KE(2, 0, 2) + KE(0, 2, 2));
    double B = (1 - om[6]) * (KK(2, 2, 0) + KK(2, 0, 2) - 2 * KK(0, 2, 2)) +
               om[6] * (KE(2, 2, 0) + KE(2, 0, 2) - 2 * KE(0, 2, 2));
    double C = (1 - om[7]) * (KK(2, 2, 0) + KK(2, 0, 2) + KK(0, 2, 2)) +
               om[7] * (KE(2, 2, 0) + KE(2, 0, 2) + KE(0, 2, 2));
    /* solve k220-2k202+k022=A, k220+k202-2k022=B, k220+k202+k022=C */
    double M3[3][4] = {{1, -2, 1, A}, {1, 1, -2, B}, {1, 1, 1, C}};
    for (int col = 0; col < 3; ++col) {
      int piv = col;
      for (int r = col + 1; r < 3; ++r)
        if (fabs(M3[r][col]) > fabs(M3[piv][col])) piv = r;
      for (int s = 0; s < 4; ++s) {
        double t = M3[col][s];
        M3[col][s] = M3[piv][s];
        M3[piv][s] = t;
      }
      for (int r = 0; r < 3; ++r) {
        if (r == col) continue;
        double fct = M3[r][col] / M3[col][col];
        for (int s = 0; s < 4; ++s) M3[r][s] -= fct * M3[col][s];
      }
    }
    KS(2, 2, 0) = M3[0][3] / M3[0][0];
    KS(2, 0, 2) = M3[1][3] / M3[1][1];
    KS(0, 2, 2) = M3[2][3] / M3[2][2];
  }
  KS(2, 1, 1) = (1 - om[8]) * KK(2, 1, 1) + om[8] * KE(2, 1, 1);
  KS(1, 2, 1) = (1 - om[8]) * KK(1, 2, 1) + om[8] * KE(1, 2, 1);
  KS(1, 1, 2) = (1 - om[8]) * KK(1, 1, 2) + om[8] * KE(1, 1, 2);
  /* fifth order, with forcing */
  KS(1, 2, 2) = (1 - om[9]) * KK(1, 2, 2) + om[9] * KE(1, 2, 2) + (1 - om[9] / 2) * F[0] * cs4;
  KS(2, 1, 2) = (1 - om[9]) * KK(2, 1, 2) + om[9] * KE(2, 1, 2) + (1 - om[9] / 2) * F[1] * cs4;
  KS(2, 2, 1) = (1 - om[9]) * KK(2, 2, 1) + om[9] * KE(2, 2, 1) + (1 - om[9] / 2) * F[2] * cs4;
  /* sixth order */
  KS(2, 2, 2) = (1 - om[10]) * KK(2, 2, 2) + om[10] * KE(2, 2, 2);
#undef KK
#undef KE
#undef KS
}

static double binom2(int n, int k) {
  /* binomial coefficient for n <= 2 */
  if (k < 0 || k > n) return 0.0;
  return (n == 2 && k == 1) ? 2.0 : 1.0;
}

static double MINV[27 * 27];
static int MINV_READY = 0;

static void ensure_minv(void) {
#ifdef _OPENMP
#pragma omp critical(ocg_minv)
#endif
  {
    if (!MINV_READY) {
      ocg_moment_matrix_inverse(MINV);
      MINV_READY = 1;
    }
  }
}

void ocg_cm_to_f(const double *k, const double u[3], double *f) {
  double m[27];
  double up[3][3]; /* up[axis][e] = u_axis^e */
  for (int ax = 0; ax < 3; ++ax)
    for (int e = 0; e < 3; ++e) up[ax][e] = ipow(u[ax], e);
  /* raw moment m_abc = sum_i f_i c^a c^b c^c with c = (c - u) + u, expanded */
  for (int c = 0; c < 3; ++c)
    for (int b = 0; b < 3; ++b)
      for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int cc = 0; cc <= c; ++cc)
          for (int bb = 0; bb <= b; ++bb)
            for (int aa = 0; aa <= a; ++aa)
              s += binom2(a, aa) * binom2(b, bb) * binom2(c, cc) *
                   up[0][a - aa] * up[1][b - bb] * up[2][c - cc] *
                   k[K(aa, bb, cc)];
        m[K(a, b, c)] = s;
      }
  ensure_minv();
  for (int i = 0; i < 27; ++i) {
    double s = 0.0;
    for (int r = 0; r < 27; ++r) s += MINV[i * 27 + r] * m[r];
    f[i] = s;
  }
}

/* ---- whole domain ----------------------------------------------------------- */

struct ocg_domain {
  ocg_params p;
  int64_t N;
  double cr2, cb2;
  uint8_t *solid;
  double *fr, *fb; /* post-collision, [27][N] */
  double *gr, *gb; /* post-streaming work arrays */
  double *rho_r, *rho_b, *press, *phi, *kappa, *om1;
  double *j, *u, *grad, *n, *F, *w, *Q, *R; /* [3][N] */
};

int64_t ocg_cells(const ocg_domain *d) { return d->N; }

int ocg_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

static double *dalloc(int64_t n) { return (double *)calloc((size_t)n, sizeof(double)); }

ocg_domain *ocg_create(const ocg_params *prm) {
  if (prm->nx <= 0 || prm->ny <= 0 || prm->nz <= 0) return NULL;
  ocg_domain *d = (ocg_domain *)calloc(1, sizeof(ocg_domain));
  d->p = *prm;
  d->N = (int64_t)prm->nx * prm->ny * prm->nz;
  d->cr2 = XI * (1.0 - prm->alpha_r);
  d->cb2 = XI * (1.0 - prm->alpha_b);
  int64_t N = d->N;
  d->solid = (uint8_t *)calloc((size_t)N, 1);
  d->fr = dalloc(27 * N); d->fb = dalloc(27 * N);
  d->gr = dalloc(27 * N); d->gb = dalloc(27 * N);
  d->rho_r = dalloc(N); d->rho_b = dalloc(N); d->press = dalloc(N);
  d->phi = dalloc(N); d->kappa = dalloc(N); d->om1 = dalloc(N);
  d->j = dalloc(3 * N); d->u = dalloc(3 * N); d->grad = dalloc(3 * N);
  d->n = dalloc(3 * N); d->F = dalloc(3 * N); d->w = dalloc(3 * N);
  d->Q = dalloc(3 * N); d->R = dalloc(3 * N);
  ensure_minv();
  ensure_tables();
  return d;
}

void ocg_destroy(ocg_domain *d) {
  if (!d) return;
  free(d->solid); free(d->fr); free(d->fb); free(d->gr); free(d->gb);
  free(d->rho_r); free(d->rho_b); free(d->press); free(d->phi); free(d->kappa);
  free(d->om1); free(d->j); free(d->u); free(d->grad); free(d->n); free(d->F);
  free(d->w); free(d->Q); free(d->R);
  free(d);
}

static int64_t wrap(int64_t v, int64_t n) { return ((v % n) + n) % n; }

/* index of the cell at (x,y,z) + s*c_i, with periodic wrap on every axis
 * (non-periodic axes have solid end layers, so the wrap is never seen by a
 * fluid cell) */
static int64_t neighbour(const ocg_domain *d, int64_t cell, int i, int s) {
  int64_t nx = d->p.nx, ny = d->p.ny, nz = d->p.nz;
  int64_t x = cell % nx, y = (cell / nx) % ny, z = cell / (nx * ny);
  x = wrap(x + s * CI[i][0], nx);
  y = wrap(y + s * CI[i][1], ny);
  z = wrap(z + s * CI[i][2], nz);
  return x + nx * (y + ny * z);
}

/* Which walls a solid cell belongs to.  Returns 1 when every wall face of the
 * cell is a slip wall (then *flip has bit a set for each wall-normal axis a),
 * 0 otherwise (no-slip: obstacles, no-slip or moving faces; *uw = the summed
 * velocity of the moving faces). */
static int wall_kind(const ocg_domain *d, int64_t cell, int *flip, double uw[3]) {
  const int64_t n[3] = {d->p.nx, d->p.ny, d->p.nz};
  const int64_t xyz[3] = {cell % n[0], (cell / n[0]) % n[1], cell / (n[0] * n[1])};
  int faces = 0, slip = 0, other = 0;
  *flip = 0;
  uw[0] = uw[1] = uw[2] = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (d->p.bc[a] == OCG_BC_PERIODIC) continue;
    int face = -1;
    if (xyz[a] == 0) face = 2 * a;
    else if (xyz[a] == n[a] - 1) face = 2 * a + 1;
    if (face < 0) continue;
    ++faces;
    if (d->p.bc[a] == OCG_BC_SLIP) {
      ++slip;
      *flip |= 1 << a;
    } else {
      ++other;
      if (d->p.bc[a] == OCG_BC_MOVING)
        for (int b = 0; b < 3; ++b) uw[b] += d->p.wall_u[face][b];
    }
  }
  return faces > 0 && other == 0 && slip > 0;
}

/* index of the velocity c_i with the components of the axes in `flip` negated */
static int reflected(int i, int flip) {
  int c[3];
  for (int a = 0; a < 3; ++a) c[a] = (flip >> a) & 1 ? -CI[i][a] : CI[i][a];
  for (int j = 0; j < 27; ++j)
    if (CI[j][0] == c[0] && CI[j][1] == c[1] && CI[j][2] == c[2]) return j;
  return i;
}

static double order_parameter(const ocg_domain *d, double rr, double rb) {
  double a = rr / d->p.rho_r0, b = rb / d->p.rho_b0;
  return (a + b > 0.0) ? (a - b) / (a + b) : 0.0;
}

int ocg_init(ocg_domain *d, const double *rho_r, const double *rho_b,
             const double *u, const uint8_t *solid) {
  const int64_t N = d->N;
  for (int64_t c = 0; c < N; ++c) {
    int64_t x = c % d->p.nx, y = (c / d->p.nx) % d->p.ny, z = c / (d->p.nx * d->p.ny);
    uint8_t s = solid ? (solid[c] != 0) : 0;
    if (d->p.bc[0] != OCG_BC_PERIODIC && (x == 0 || x == d->p.nx - 1)) s = 1;
    if (d->p.bc[1] != OCG_BC_PERIODIC && (y == 0 || y == d->p.ny - 1)) s = 1;
    if (d->p.bc[2] != OCG_BC_PERIODIC && (z == 0 || z == d->p.nz - 1)) s = 1;
    d->solid[c] = s;
  }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    double feq[27];
    if (d->solid[c]) {
      for (int i = 0; i < 27; ++i) d->fr[i * N + c] = d->fb[i * N + c] = 0.0;
      d->rho_r[c] = d->rho_b[c] = d->press[c] = d->phi[c] = 0.0;
      for (int a = 0; a < 3; ++a) d->u[a * N + c] = 0.0;
      continue;
    }
    double rr = rho_r[c], rb = rho_b[c], rho = rr + rb;
    double p = rr * d->cr2 + rb * d->cb2;
    double uc[3] = {u[c], u[N + c], u[2 * N + c]};
    ocg_feq(d->p.model, rho, p, uc, feq);
    for (int i = 0; i < 27; ++i) {
      d->fr[i * N + c] = rr / rho * feq[i];
      d->fb[i * N + c] = rb / rho * feq[i];
    }
    d->rho_r[c] = rr;
    d->rho_b[c] = rb;
    d->press[c] = p;
    d->phi[c] = order_parameter(d, rr, rb);
    for (int a = 0; a < 3; ++a) d->u[a * N + c] = uc[a];
  }
  /* walls start as if they had received the initial populations of their
   * fluid neighbours one step earlier (the fullway rule of one_step applied
   * to the initial state), so the first step sees no empty wall */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    if (!d->solid[c]) continue;
    int flip;
    double uw[3];
    const int slip = wall_kind(d, c, &flip, uw);
    for (int i = 0; i < 27; ++i) {
      const int j = slip ? reflected(i, flip) : opposite(i);
      const int64_t src = neighbour(d, c, j, -1);
      double r = 0.0, b = 0.0;
      if (!d->solid[src]) {
        r = d->fr[j * N + src];
        b = d->fb[j * N + src];
        if (!slip) {
          const double cu = CI[i][0] * uw[0] + CI[i][1] * uw[1] + CI[i][2] * uw[2];
          r += 2.0 * weight(i) * rho_r[src] * cu / CS2;
          b += 2.0 * weight(i) * rho_b[src] * cu / CS2;
        }
      }
      d->fr[i * N + c] = r;
      d->fb[i * N + c] = b;
    }
  }
  return 0;
}

int ocg_set_populations(ocg_domain *d, const double *fr, const double *fb) {
  memcpy(d->fr, fr, sizeof(double) * 27 * d->N);
  memcpy(d->fb, fb, sizeof(double) * 27 * d->N);
  return 0;
}

/* one time step: stream, macroscopic fields, gradients, collide, recolor */
static void one_step(ocg_domain *d) {
  const int64_t N = d->N;
  const ocg_params *P = &d->p;

  /* streaming (Eq. streaming step), in pull form */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c)
    for (int i = 0; i < 27; ++i) {
      int64_t src = neighbour(d, c, i, -1);
      d->gr[i * N + c] = d->fr[i * N + src];
      d->gb[i * N + c] = d->fb[i * N + src];
    }

  /* densities, momentum, pressure (EOS), order parameter (Sec. II.A) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    double rr = 0, rb = 0, jx = 0, jy = 0, jz = 0;
    for (int i = 0; i < 27; ++i) {
      double fi = d->gr[i * N + c] + d->gb[i * N + c];
      rr += d->gr[i * N + c];
      rb += d->gb[i * N + c];
      jx += fi * CI[i][0];
      jy += fi * CI[i][1];
      jz += fi * CI[i][2];
    }
    d->rho_r[c] = rr;
    d->rho_b[c] = rb;
    d->j[c] = jx; d->j[N + c] = jy; d->j[2 * N + c] = jz;
    d->press[c] = rr * d->cr2 + rb * d->cb2;
    d->phi[c] = order_parameter(d, rr, rb);
  }

  /* colour gradient and unit normal (isotropic difference, Sec. II.A) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    double g[3] = {0, 0, 0};
    if (!d->solid[c]) {
      for (int i = 0; i < 27; ++i) {
        int64_t nb = neighbour(d, c, i, +1);
        double v = d->solid[nb] ? d->phi[c] : d->phi[nb];
        for (int a = 0; a < 3; ++a) g[a] += weight(i) * v * CI[i][a];
      }
      for (int a = 0; a < 3; ++a) g[a] /= CS2;
    }
    double g2n = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    for (int a = 0; a < 3; ++a) {
      d->grad[a * N + c] = g[a];
      d->n[a * N + c] = (g2n > NORMAL_EPS) ? g[a] / sqrt(g2n) : 0.0;
    }
  }

  /* curvature, CSF force, body force, velocity, (p - rho cs2) u */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    if (d->solid[c]) {
      d->kappa[c] = 0.0;
      for (int a = 0; a < 3; ++a) d->F[a * N + c] = d->u[a * N + c] = d->w[a * N + c] = 0.0;
      continue;
    }
    double dn[3][3] = {{0}}; /* dn[a][b] = d_a n_b */
    for (int i = 0; i < 27; ++i) {
      int64_t nb = neighbour(d, c, i, +1);
      int64_t src = d->solid[nb] ? c : nb;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) dn[a][b] += weight(i) * d->n[b * N + src] * CI[i][a];
    }
    double div = 0.0, nnd = 0.0;
    for (int a = 0; a < 3; ++a) {
      div += dn[a][a] / CS2;
      for (int b = 0; b < 3; ++b)
        nnd += d->n[a * N + c] * d->n[b * N + c] * dn[a][b] / CS2;
    }
    double kappa = -(div - nnd);
    d->kappa[c] = kappa;
    double rho = d->rho_r[c] + d->rho_b[c];
    double fb_[3] = {0, 0, 0};
    switch (P->force_mode) {
      case OCG_FORCE_CONST: for (int a = 0; a < 3; ++a) fb_[a] = P->g[a]; break;
      case OCG_FORCE_GRAVITY: for (int a = 0; a < 3; ++a) fb_[a] = rho * P->g[a]; break;
      case OCG_FORCE_BUOYANCY:
        for (int a = 0; a < 3; ++a) fb_[a] = (rho - P->rho_ref) * P->g[a];
        break;
      default: break;
    }
    for (int a = 0; a < 3; ++a) {
      double Fa = 0.5 * P->sigma * kappa * d->grad[a * N + c] + fb_[a];
      d->F[a * N + c] = Fa;
      double ua = (d->j[a * N + c] + Fa / 2.0) / rho;
      d->u[a * N + c] = ua;
      d->w[a * N + c] = (d->press[c] - rho * CS2) * ua;
    }
  }

  /* correction term Q (Sec. III.E) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    double q[3] = {0, 0, 0};
    if (!d->solid[c] && P->use_Q) {
      for (int i = 0; i < 27; ++i) {
        int64_t nb = neighbour(d, c, i, +1);
        for (int a = 0; a < 3; ++a) q[a] += weight(i) * d->w[a * N + nb] * CI[i][a];
      }
      for (int a = 0; a < 3; ++a) q[a] = -3.0 * q[a] / CS2;
    }
    for (int a = 0; a < 3; ++a) d->Q[a * N + c] = q[a];
  }

  /* collision in central-moment space and recoloring; bounce-back at solids */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    if (d->solid[c]) {
      /* fullway bounce-back: what arrived along c_j leaves along c_i next step.
       * No-slip and moving walls: j = opposite(i), and a moving wall adds
       * 2 w_i rho_k (c_i . u_w) / c_s^2 to colour k of a population that came
       * from a fluid cell, rho_k of that cell.  Slip walls: c_j is c_i with
       * the wall-normal components negated (specular reflection). */
      int flip;
      double uw[3];
      const int slip = wall_kind(d, c, &flip, uw);
      for (int i = 0; i < 27; ++i) {
        const int j = slip ? reflected(i, flip) : opposite(i);
        double r = d->gr[j * N + c], b = d->gb[j * N + c];
        const int64_t src = neighbour(d, c, j, -1);
        if (!slip && !d->solid[src]) {  /* momentum exchange with the fluid only */
          const double cu = CI[i][0] * uw[0] + CI[i][1] * uw[1] + CI[i][2] * uw[2];
          r += 2.0 * weight(i) * d->rho_r[src] * cu / CS2;
          b += 2.0 * weight(i) * d->rho_b[src] * cu / CS2;
        }
        d->fr[i * N + c] = r;
        d->fb[i * N + c] = b;
      }
      for (int a = 0; a < 3; ++a) d->R[a * N + c] = 0.0;
      d->om1[c] = 0.0;
      continue;
    }
    double f[27], feq[27], k[27], keq[27], ks[27], fs[27];
    double rr = d->rho_r[c], rb = d->rho_b[c], rho = rr + rb, p = d->press[c];
    double uc[3] = {d->u[c], d->u[N + c], d->u[2 * N + c]};
    double Fc[3] = {d->F[c], d->F[N + c], d->F[2 * N + c]};
    double Qc[3] = {d->Q[c], d->Q[N + c], d->Q[2 * N + c]};
    /* viscosity interpolation and relaxation time, mu = (tau - 1/2) p */
    double phi = d->phi[c];
    double nu = 0.5 * (1.0 + phi) * P->nu_r + 0.5 * (1.0 - phi) * P->nu_b;
    double tau = 0.5 + rho * nu / p;
    double om[11];
    for (int q = 0; q < 11; ++q) om[q] = P->omega[q];
    om[1] = 1.0 / tau;
    d->om1[c] = om[1];
    for (int i = 0; i < 27; ++i) f[i] = d->gr[i * N + c] + d->gb[i * N + c];
    ocg_central_moments(f, uc, k);
    ocg_feq(P->model, rho, p, uc, feq);
    ocg_central_moments(feq, uc, keq);
    ocg_collide_cm(k, keq, om, Fc, Qc, ks);
    ocg_cm_to_f(ks, uc, fs);
    double Rc[3];
    for (int a = 0; a < 3; ++a) {
      Rc[a] = P->beta * rr * rb / (rho * rho) * p * d->n[a * N + c];
      d->R[a * N + c] = Rc[a];
    }
    for (int i = 0; i < 27; ++i) {
      double cR = CI[i][0] * Rc[0] + CI[i][1] * Rc[1] + CI[i][2] * Rc[2];
      d->fr[i * N + c] = rr / rho * fs[i] + weight(i) / CS2 * cR;
      d->fb[i * N + c] = rb / rho * fs[i] - weight(i) / CS2 * cR;
    }
  }
}

int ocg_step(ocg_domain *d, int64_t nsteps) {
  for (int64_t s = 0; s < nsteps; ++s) one_step(d);
  return 0;
}

void ocg_read_macros(const ocg_domain *d, double *rho_r, double *rho_b, double *u,
                     double *p, double *phi) {
  const int64_t N = d->N;
  for (int64_t c = 0; c < N; ++c) {
    if (rho_r) rho_r[c] = d->rho_r[c];
    if (rho_b) rho_b[c] = d->rho_b[c];
    if (p) p[c] = d->solid[c] ? 0.0 : d->press[c];
    if (phi) phi[c] = d->solid[c] ? 0.0 : d->phi[c];
    if (u)
      for (int a = 0; a < 3; ++a) u[a * N + c] = d->solid[c] ? 0.0 : d->u[a * N + c];
  }
}

void ocg_read_populations(const ocg_domain *d, double *fr, double *fb) {
  if (fr) memcpy(fr, d->fr, sizeof(double) * 27 * d->N);
  if (fb) memcpy(fb, d->fb, sizeof(double) * 27 * d->N);
}

int ocg_read_field(const ocg_domain *d, int which, double *out) {
  const int64_t N = d->N;
  const double *src = NULL;
  int64_t len = 3 * N;
  switch (which) {
    case 0: src = d->grad; break;
    case 1: src = d->n; break;
    case 2: src = d->kappa; len = N; break;
    case 3: src = d->F; break;
    case 4: src = d->Q; break;
    case 5: src = d->om1; len = N; break;
    case 6: src = d->w; break;
    case 7: src = d->R; break;
    default: return -1;
  }
  memcpy(out, src, sizeof(double) * len);
  return 0;
}

/* compensated (Neumaier) summation, so the reduction itself stays well below
 * the round-off of the step it is used to check */
static void neumaier_add(double *sum, double *comp, double v) {
  double t = *sum + v;
  if (fabs(*sum) >= fabs(v))
    *comp += (*sum - t) + v;
  else
    *comp += (v - t) + *sum;
  *sum = t;
}

void ocg_mass(const ocg_domain *d, double out[2]) {
  const int64_t N = d->N;
  double sr = 0.0, cr = 0.0, sb = 0.0, cb = 0.0;
  for (int i = 0; i < 27; ++i)
    for (int64_t c = 0; c < N; ++c) {
      neumaier_add(&sr, &cr, d->fr[i * N + c]);
      neumaier_add(&sb, &cb, d->fb[i * N + c]);
    }
  out[0] = sr + cr;
  out[1] = sb + cb;
}
