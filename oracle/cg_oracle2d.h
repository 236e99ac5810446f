/* cg_oracle2d.h -- CPU reference (FP64) of the colour-gradient CM-MRT step on
 * the D2Q9 lattice (App. A of arXiv 2309.07801).  Test infrastructure: used
 * only by the tests; it shares no code with the CUDA library. */
#ifndef CG_ORACLE2D_H
#define CG_ORACLE2D_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct o2_params {
  int32_t nx, ny;
  int32_t bc[2];          /* per axis: 0 periodic, 1 fullway bounce-back (end layers solid) */
  double rho_r0, rho_b0;
  double alpha_r, alpha_b;/* (c_s^k)^2 = (3/5)(1 - alpha_k) */
  double nu_r, nu_b;
  double sigma, beta;
  double omega[5];        /* omega_0..omega_4 (first order, shear [replaced by 1/tau],
                             bulk, third order, fourth order) */
  double g[2];
  double rho_ref;
  int32_t force_mode;     /* 0 none, 1 F = g, 2 F = rho g, 3 F = (rho - rho_ref) g */
  int32_t use_Q;
} o2_params;

void o2_lattice(int32_t *c, double *w);
double o2_hermite(int i, int a, int b);
void o2_feq(double rho, double p, const double u[2], double *f);
void o2_central_moments(const double *f, const double u[2], double *k);
void o2_moment_matrix(double *M);
void o2_moment_matrix_inverse(double *Minv);
void o2_cm_to_f(const double *k, const double u[2], double *f);
void o2_collide_cm(const double *k, const double *keq, const double *om, const double F[2],
                   const double Q[2], double *ks);

typedef struct o2_domain o2_domain;
o2_domain *o2_create(const o2_params *p);
void o2_destroy(o2_domain *d);
int o2_init(o2_domain *d, const double *rho_r, const double *rho_b, const double *u);
int o2_step(o2_domain *d, int64_t n);
int o2_read_macros(const o2_domain *d, double *rho_r, double *rho_b, double *u, double *p, double *phi);
int o2_read_populations(const o2_domain *d, double *fr, double *fb);
void o2_mass(const o2_domain *d, double out[2]);

#ifdef __cplusplus
}
#endif
#endif
