/* cg_oracle2d.c -- CPU reference (FP64) of the colour-gradient CM-MRT step on
 * the D2Q9 lattice (App. A of arXiv 2309.07801), for the paper's
 * two-dimensional tests.  Test infrastructure only: it shares no code with the
 * CUDA library.  Written from:
 *   - the D2Q9 velocities and weights printed in App. A;
 *   - g^{eq,4} with the Hermite polynomials of App. A, the isotropic operator
 *     E_i and the generalized equilibria (Eq. general form in 2D, App. A);
 *   - raw and central moments by their defining sums (Sec. II.B in 2D);
 *   - the collision of Sec. II.B restricted to the nine 2D moments (reading:
 *     first order with omega_0 and F, k_11 and k_20 - k_02 with omega_1,
 *     k_20 + k_02 with omega_2, k_21 and k_12 with omega_3 and c_s^2 F,
 *     k_22 with omega_4; Q on the diagonal second-order moments);
 *   - densities, momentum, the EOS p = sum rho_k (c_s^k)^2 with
 *     (c_s^k)^2 = xi (1 - alpha_k) and xi = 3/5 (reading: alpha = w_0 = 4/9
 *     gives the lattice c_s^2 = 1/3, as xi = 9/19 does for D3Q27), the order
 *     parameter, the CSF force, Q, recoloring (Sec. II.A, Sec. III.E);
 *   - pull streaming and fullway bounce-back at solid cells (Sec. IV).
 * Cells: index x + nx y; populations [9][N] in the order of App. A. */
#include "cg_oracle2d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const int C2[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
static const double CS2D = 1.0 / 3.0;
static const double XI2D = 3.0 / 5.0;

static double w2(int i) {
  int c2 = C2[i][0] * C2[i][0] + C2[i][1] * C2[i][1];
  return c2 == 0 ? 4.0 / 9.0 : (c2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
}

static int opp2(int i) {
  for (int j = 0; j < 9; ++j)
    if (C2[j][0] == -C2[i][0] && C2[j][1] == -C2[i][1]) return j;
  return i;
}

void o2_lattice(int32_t *c, double *w) {
  for (int i = 0; i < 9; ++i) {
    c[2 * i] = C2[i][0];
    c[2 * i + 1] = C2[i][1];
    w[i] = w2(i);
  }
}

/* Hermite polynomials of App. A, index a + 3 b (a, b = 0..2) */
double o2_hermite(int i, int a, int b) {
  const double cx = C2[i][0], cy = C2[i][1];
  const double h1x = cx, h1y = cy, h2x = cx * cx - CS2D, h2y = cy * cy - CS2D;
  const double hx = a == 0 ? 1.0 : (a == 1 ? h1x : h2x);
  const double hy = b == 0 ? 1.0 : (b == 1 ? h1y : h2y);
  return hx * hy;
}

/* generalized equilibria (Model D) for D2Q9, App. A */
void o2_feq(double rho, double p, const double u[2], double *f) {
  const double cs4 = CS2D * CS2D, cs6 = cs4 * CS2D, cs8 = cs4 * cs4;
  const double ux = u[0], uy = u[1];
  for (int i = 0; i < 9; ++i) {
    const double w = w2(i);
    const double H10 = o2_hermite(i, 1, 0), H01 = o2_hermite(i, 0, 1);
    const double H20 = o2_hermite(i, 2, 0), H02 = o2_hermite(i, 0, 2), H11 = o2_hermite(i, 1, 1);
    const double H21 = o2_hermite(i, 2, 1), H12 = o2_hermite(i, 1, 2), H22 = o2_hermite(i, 2, 2);
    const double g4 = rho * w *
                      (1.0 + (ux * H10 + uy * H01) / CS2D +
                       (ux * ux * H20 + uy * uy * H02 + 2.0 * ux * uy * H11) / (2.0 * cs4) +
                       (ux * ux * uy * H21 + ux * uy * uy * H12) / (2.0 * cs6) +
                       ux * ux * uy * uy * H22 / (4.0 * cs8));
    const double E = w * ((H20 + H02) / (2.0 * cs4) - H22 / (4.0 * cs6));
    const double corr = w * ((ux * H12 + uy * H21) / (2.0 * cs6) + (ux * ux + uy * uy) * H22 / (4.0 * cs8));
    f[i] = g4 + (p - rho * CS2D) * (E + corr);
  }
}

static double ipow2(double v, int e) { return e == 0 ? 1.0 : (e == 1 ? v : v * v); }

/* k_ab = sum_i f_i (c_ix - u_x)^a (c_iy - u_y)^b, index a + 3 b */
void o2_central_moments(const double *f, const double u[2], double *k) {
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int i = 0; i < 9; ++i) s += f[i] * ipow2(C2[i][0] - u[0], a) * ipow2(C2[i][1] - u[1], b);
      k[a + 3 * b] = s;
    }
}

/* raw-moment matrix M[r][i] = c_ix^a c_iy^b, r = a + 3 b, and its inverse (Gauss-Jordan) */
void o2_moment_matrix(double *M) {
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a)
      for (int i = 0; i < 9; ++i) M[(a + 3 * b) * 9 + i] = ipow2(C2[i][0], a) * ipow2(C2[i][1], b);
}

static double MINV2[81];
static int MINV2_READY = 0;

void o2_moment_matrix_inverse(double *out) {
  double A[9][18];
  double M[81];
  o2_moment_matrix(M);
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 18; ++c) A[r][c] = c < 9 ? M[r * 9 + c] : (c - 9 == r ? 1.0 : 0.0);
  for (int col = 0; col < 9; ++col) {
    int piv = col;
    for (int r = col + 1; r < 9; ++r)
      if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
    for (int c = 0; c < 18; ++c) {
      double t = A[col][c];
      A[col][c] = A[piv][c];
      A[piv][c] = t;
    }
    double d = A[col][col];
    for (int c = 0; c < 18; ++c) A[col][c] /= d;
    for (int r = 0; r < 9; ++r)
      if (r != col) {
        double m = A[r][col];
        for (int c = 0; c < 18; ++c) A[r][c] -= m * A[col][c];
      }
  }
  for (int r = 0; r < 9; ++r)
    for (int c = 0; c < 9; ++c) out[r * 9 + c] = A[r][c + 9];
}

static void ensure_minv2(void) {
  if (!MINV2_READY) {
    o2_moment_matrix_inverse(MINV2);
    MINV2_READY = 1;
  }
}

/* central moments about u -> populations: binomial shift to raw moments, then M^-1 */
void o2_cm_to_f(const double *k, const double u[2], double *f) {
  double m[9];
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      double s = 0.0;
      for (int bb = 0; bb <= b; ++bb)
        for (int aa = 0; aa <= a; ++aa) {
          const double ca = (a == 2 && aa == 1) ? 2.0 : 1.0, cb = (b == 2 && bb == 1) ? 2.0 : 1.0;
          s += ca * cb * ipow2(u[0], a - aa) * ipow2(u[1], b - bb) * k[aa + 3 * bb];
        }
      m[a + 3 * b] = s;
    }
  ensure_minv2();
  for (int i = 0; i < 9; ++i) {
    double s = 0.0;
    for (int r = 0; r < 9; ++r) s += MINV2[i * 9 + r] * m[r];
    f[i] = s;
  }
}

/* collision in central-moment space (2D reading of Sec. II.B, see the header) */
void o2_collide_cm(const double *k, const double *keq, const double *om, const double F[2], const double Q[2],
                   double *ks) {
  const double o0 = om[0], o1 = om[1], o2 = om[2], o3 = om[3], o4 = om[4];
  for (int r = 0; r < 9; ++r) ks[r] = k[r];
  ks[0] = k[0];
  ks[1] = (1.0 - o0) * k[1] + (1.0 - o0 / 2.0) * F[0];   /* k_10 */
  ks[3] = (1.0 - o0) * k[3] + (1.0 - o0 / 2.0) * F[1];   /* k_01 */
  ks[4] = (1.0 - o1) * k[4] + o1 * keq[4];               /* k_11 */
  {
    const double d = k[2] - k[6], de = keq[2] - keq[6];  /* k_20 - k_02 */
    const double t = k[2] + k[6], te = keq[2] + keq[6];
    const double ds = (1.0 - o1) * d + o1 * de + (1.0 - o1 / 2.0) * (Q[0] - Q[1]);
    const double ts = (1.0 - o2) * t + o2 * te + (1.0 - o2 / 2.0) * (Q[0] + Q[1]);
    ks[2] = 0.5 * (ts + ds);
    ks[6] = 0.5 * (ts - ds);
  }
  ks[5] = (1.0 - o3) * k[5] + o3 * keq[5] + (1.0 - o3 / 2.0) * F[1] * CS2D;  /* k_21 */
  ks[7] = (1.0 - o3) * k[7] + o3 * keq[7] + (1.0 - o3 / 2.0) * F[0] * CS2D;  /* k_12 */
  ks[8] = (1.0 - o4) * k[8] + o4 * keq[8];                                    /* k_22 */
}

/* ---- whole domain ---------------------------------------------------------- */

struct o2_domain {
  o2_params p;
  int64_t N;
  double cr2, cb2;
  uint8_t *solid;
  double *fr, *fb, *gr, *gb;                         /* [9][N] */
  double *rho_r, *rho_b, *press, *phi, *u, *F, *w, *Q, *n, *grad;  /* scalars / [2][N] */
};

static int64_t wrap2(int64_t v, int64_t n) { return ((v % n) + n) % n; }

static int64_t nbr2(const o2_domain *d, int64_t c, int i, int s) {
  int64_t x = c % d->p.nx, y = c / d->p.nx;
  x = wrap2(x + s * C2[i][0], d->p.nx);
  y = wrap2(y + s * C2[i][1], d->p.ny);
  return x + d->p.nx * y;
}

static double order_param2(const o2_domain *d, double rr, double rb) {
  const double a = rr / d->p.rho_r0, b = rb / d->p.rho_b0;
  return a + b > 0.0 ? (a - b) / (a + b) : 0.0;
}

o2_domain *o2_create(const o2_params *p) {
  if (p->nx < 1 || p->ny < 1) return NULL;
  o2_domain *d = (o2_domain *)calloc(1, sizeof(o2_domain));
  d->p = *p;
  d->N = (int64_t)p->nx * p->ny;
  d->cr2 = XI2D * (1.0 - p->alpha_r);
  d->cb2 = XI2D * (1.0 - p->alpha_b);
  const int64_t N = d->N;
  d->solid = (uint8_t *)calloc((size_t)N, 1);
  d->fr = (double *)calloc(9 * N, sizeof(double));
  d->fb = (double *)calloc(9 * N, sizeof(double));
  d->gr = (double *)calloc(9 * N, sizeof(double));
  d->gb = (double *)calloc(9 * N, sizeof(double));
  d->rho_r = (double *)calloc(N, sizeof(double));
  d->rho_b = (double *)calloc(N, sizeof(double));
  d->press = (double *)calloc(N, sizeof(double));
  d->phi = (double *)calloc(N, sizeof(double));
  d->u = (double *)calloc(2 * N, sizeof(double));
  d->F = (double *)calloc(2 * N, sizeof(double));
  d->w = (double *)calloc(2 * N, sizeof(double));
  d->Q = (double *)calloc(2 * N, sizeof(double));
  d->n = (double *)calloc(2 * N, sizeof(double));
  d->grad = (double *)calloc(2 * N, sizeof(double));
  return d;
}

void o2_destroy(o2_domain *d) {
  if (!d) return;
  free(d->solid); free(d->fr); free(d->fb); free(d->gr); free(d->gb);
  free(d->rho_r); free(d->rho_b); free(d->press); free(d->phi); free(d->u);
  free(d->F); free(d->w); free(d->Q); free(d->n); free(d->grad);
  free(d);
}

int o2_init(o2_domain *d, const double *rho_r, const double *rho_b, const double *u) {
  const int64_t N = d->N;
  for (int64_t c = 0; c < N; ++c) {
    const int64_t x = c % d->p.nx, y = c / d->p.nx;
    uint8_t s = 0;
    if (d->p.bc[0] && (x == 0 || x == d->p.nx - 1)) s = 1;
    if (d->p.bc[1] && (y == 0 || y == d->p.ny - 1)) s = 1;
    d->solid[c] = s;
  }
  for (int64_t c = 0; c < N; ++c) {
    if (d->solid[c]) continue;
    const double rr = rho_r[c], rb = rho_b[c], rho = rr + rb, p = rr * d->cr2 + rb * d->cb2;
    const double uc[2] = {u[c], u[N + c]};
    double feq[9];
    o2_feq(rho, p, uc, feq);
    for (int i = 0; i < 9; ++i) {
      d->fr[i * N + c] = rr / rho * feq[i];
      d->fb[i * N + c] = rb / rho * feq[i];
    }
    d->rho_r[c] = rr;
    d->rho_b[c] = rb;
    d->press[c] = p;
    d->phi[c] = order_param2(d, rr, rb);
    d->u[c] = uc[0];
    d->u[N + c] = uc[1];
  }
  /* walls start with the reversed initial populations of their fluid neighbours */
  for (int64_t c = 0; c < N; ++c) {
    if (!d->solid[c]) continue;
    for (int i = 0; i < 9; ++i) {
      const int j = opp2(i);
      const int64_t src = nbr2(d, c, j, -1);
      d->fr[i * N + c] = d->solid[src] ? 0.0 : d->fr[j * N + src];
      d->fb[i * N + c] = d->solid[src] ? 0.0 : d->fb[j * N + src];
    }
  }
  return 0;
}

/* isotropic difference (1/c_s^2) sum_i w_i c_i chi(x + c_i); a solid neighbour
 * contributes the centre value */
static void grad2(const o2_domain *d, const double *chi, int64_t c, double g[2]) {
  g[0] = g[1] = 0.0;
  for (int i = 1; i < 9; ++i) {
    const int64_t nb = nbr2(d, c, i, 1);
    const double v = d->solid[nb] ? chi[c] : chi[nb];
    g[0] += w2(i) * C2[i][0] * v;
    g[1] += w2(i) * C2[i][1] * v;
  }
  g[0] /= CS2D;
  g[1] /= CS2D;
}

static void one_step2(o2_domain *d) {
  const int64_t N = d->N;
  const o2_params *P = &d->p;
  /* streaming */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c)
    for (int i = 0; i < 9; ++i) {
      const int64_t src = nbr2(d, c, i, -1);
      d->gr[i * N + c] = d->fr[i * N + src];
      d->gb[i * N + c] = d->fb[i * N + src];
    }
  /* densities, pressure, order parameter */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    double rr = 0.0, rb = 0.0;
    for (int i = 0; i < 9; ++i) {
      rr += d->gr[i * N + c];
      rb += d->gb[i * N + c];
    }
    d->rho_r[c] = rr;
    d->rho_b[c] = rb;
    d->press[c] = d->solid[c] ? 0.0 : rr * d->cr2 + rb * d->cb2;
    d->phi[c] = d->solid[c] ? 0.0 : order_param2(d, rr, rb);
  }
  /* colour gradient and unit normal */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    double g[2] = {0.0, 0.0};
    if (!d->solid[c]) grad2(d, d->phi, c, g);
    const double g2 = g[0] * g[0] + g[1] * g[1];
    const double inv = g2 > 1e-24 ? 1.0 / sqrt(g2) : 0.0;
    for (int a = 0; a < 2; ++a) {
      d->grad[a * N + c] = g[a];
      d->n[a * N + c] = g[a] * inv;
    }
  }
  /* curvature, forces, velocity, (p - rho c_s^2) u */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    if (d->solid[c]) {
      for (int a = 0; a < 2; ++a) d->F[a * N + c] = d->u[a * N + c] = d->w[a * N + c] = 0.0;
      continue;
    }
    double dn[2][2];
    for (int b = 0; b < 2; ++b) {
      double gb[2];
      grad2(d, d->n + b * N, c, gb);
      dn[0][b] = gb[0];
      dn[1][b] = gb[1];
    }
    const double nc[2] = {d->n[c], d->n[N + c]};
    double div = dn[0][0] + dn[1][1], nnd = 0.0;
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) nnd += nc[a] * nc[b] * dn[a][b];
    const double kappa = -(div - nnd);
    const double rr = d->rho_r[c], rb = d->rho_b[c], rho = rr + rb, p = d->press[c];
    double j[2] = {0.0, 0.0};
    for (int i = 0; i < 9; ++i) {
      const double f = d->gr[i * N + c] + d->gb[i * N + c];
      j[0] += f * C2[i][0];
      j[1] += f * C2[i][1];
    }
    for (int a = 0; a < 2; ++a) {
      double fb = 0.0;
      if (P->force_mode == 1) fb = P->g[a];
      else if (P->force_mode == 2) fb = rho * P->g[a];
      else if (P->force_mode == 3) fb = (rho - P->rho_ref) * P->g[a];
      const double Fa = 0.5 * P->sigma * kappa * d->grad[a * N + c] + fb;
      d->F[a * N + c] = Fa;
      d->u[a * N + c] = (j[a] + 0.5 * Fa) / rho;
      d->w[a * N + c] = (p - rho * CS2D) * d->u[a * N + c];
    }
  }
  /* correction term Q_a = -3 d_a[(p - rho c_s^2) u_a] */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    /* plain sum: (p - rho c_s^2) u is 0 at solid cells, no substitution */
    double q[2] = {0.0, 0.0};
    if (!d->solid[c] && P->use_Q)
      for (int i = 1; i < 9; ++i) {
        const int64_t nb = nbr2(d, c, i, 1);
        for (int a = 0; a < 2; ++a) q[a] += w2(i) * C2[i][a] * d->w[a * N + nb];
      }
    for (int a = 0; a < 2; ++a) d->Q[a * N + c] = -3.0 * q[a] / CS2D;
  }
  /* collision, recoloring; fullway bounce-back at solid cells */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int64_t c = 0; c < N; ++c) {
    if (d->solid[c]) {
      for (int i = 0; i < 9; ++i) {
        const int o = opp2(i);
        d->fr[i * N + c] = d->gr[o * N + c];
        d->fb[i * N + c] = d->gb[o * N + c];
      }
      continue;
    }
    const double rr = d->rho_r[c], rb = d->rho_b[c], rho = rr + rb, p = d->press[c];
    const double uc[2] = {d->u[c], d->u[N + c]}, Fc[2] = {d->F[c], d->F[N + c]}, Qc[2] = {d->Q[c], d->Q[N + c]};
    const double phi = d->phi[c];
    const double nu = 0.5 * (1.0 + phi) * P->nu_r + 0.5 * (1.0 - phi) * P->nu_b;
    double om[5];
    for (int q = 0; q < 5; ++q) om[q] = P->omega[q];
    om[1] = 1.0 / (0.5 + rho * nu / p);
    double f[9], feq[9], k[9], keq[9], ks[9], fs[9];
    for (int i = 0; i < 9; ++i) f[i] = d->gr[i * N + c] + d->gb[i * N + c];
    o2_central_moments(f, uc, k);
    o2_feq(rho, p, uc, feq);
    o2_central_moments(feq, uc, keq);
    o2_collide_cm(k, keq, om, Fc, Qc, ks);
    o2_cm_to_f(ks, uc, fs);
    const double rf = P->beta * rr * rb * p / (rho * rho);
    const double R[2] = {rf * d->n[c], rf * d->n[N + c]};
    for (int i = 0; i < 9; ++i) {
      const double t = w2(i) / CS2D * (C2[i][0] * R[0] + C2[i][1] * R[1]);
      d->fr[i * N + c] = rr / rho * fs[i] + t;
      d->fb[i * N + c] = rb / rho * fs[i] - t;
    }
  }
}

int o2_step(o2_domain *d, int64_t n) {
  for (int64_t s = 0; s < n; ++s) one_step2(d);
  return 0;
}

int o2_read_macros(const o2_domain *d, double *rho_r, double *rho_b, double *u, double *p, double *phi) {
  const int64_t N = d->N;
  for (int64_t c = 0; c < N; ++c) {
    if (rho_r) rho_r[c] = d->rho_r[c];
    if (rho_b) rho_b[c] = d->rho_b[c];
    if (p) p[c] = d->press[c];
    if (phi) phi[c] = d->phi[c];
    if (u) {
      u[c] = d->solid[c] ? 0.0 : d->u[c];
      u[N + c] = d->solid[c] ? 0.0 : d->u[N + c];
    }
  }
  return 0;
}

int o2_read_populations(const o2_domain *d, double *fr, double *fb) {
  memcpy(fr, d->fr, sizeof(double) * 9 * d->N);
  memcpy(fb, d->fb, sizeof(double) * 9 * d->N);
  return 0;
}

void o2_mass(const o2_domain *d, double out[2]) {
  double s[2] = {0.0, 0.0}, e[2] = {0.0, 0.0};
  for (int64_t i = 0; i < 9 * d->N; ++i) {
    const double v[2] = {d->fr[i], d->fb[i]};
    for (int k = 0; k < 2; ++k) {
      const double t = s[k] + v[k];
      e[k] += fabs(s[k]) >= fabs(v[k]) ? (s[k] - t) + v[k] : (v[k] - t) + s[k];
      s[k] = t;
    }
  }
  out[0] = s[0] + e[0];
  out[1] = s[1] + e[1];
}
