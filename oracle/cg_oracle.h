/*
 * cg_oracle.h -- FP64 CPU oracle for the D3Q27 two-component colour-gradient
 * lattice Boltzmann step with central-moment MRT collision and the
 * generalized (velocity-independent) equilibrium central moments
 * (Saito et al., "Generalized equilibria for color-gradient lattice Boltzmann
 * model based on higher-order Hermite polynomials", arXiv 2309.07801).
 *
 * TEST INFRASTRUCTURE ONLY.  This header and cg_oracle.c are the slow,
 * plain reference that the CUDA path is checked against.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it.  It shares
 * no header, table or helper with the CUDA library.
 *
 * Conventions
 *   - Velocity order: the 27 lattice vectors exactly as printed in Sec. II.A
 *     (Eq. for c_i); the opposite of odd i is i+1.
 *   - Moment index r = a + 3*b + 9*c for the moment of orders (a,b,c) in
 *     (x,y,z), each in {0,1,2}.
 *   - Cell index n = x + nx*(y + ny*z); population arrays are [27][N].
 *   - The stored state is post-collision, post-recoloring (pre-streaming):
 *     one step = stream, macroscopic fields, gradients, collide, recolor.
 */
#ifndef CG_ORACLE_H
#define CG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OCG_MODEL_A = 0, OCG_MODEL_B = 1, OCG_MODEL_C = 2, OCG_MODEL_D = 3 };
/* walls (Sec. IV, introduction: no-slip, slip and moving walls, all by the
 * fullway bounce-back scheme): the end layers of a non-periodic axis are solid */
enum { OCG_BC_PERIODIC = 0, OCG_BC_BOUNCEBACK = 1, OCG_BC_SLIP = 2, OCG_BC_MOVING = 3 };
enum { OCG_FORCE_NONE = 0, OCG_FORCE_CONST = 1, OCG_FORCE_GRAVITY = 2,
       OCG_FORCE_BUOYANCY = 3 };

typedef struct ocg_params {
  int32_t nx, ny, nz;
  int32_t bc[3];          /* per axis: periodic, or a wall kind (OCG_BC_*) with
                             solid layers at index 0 and n-1 */
  double rho_r0, rho_b0;  /* reference densities (Sec. II.A, Eq. order parameter) */
  double alpha_r, alpha_b;/* rest fractions; (c_s^k)^2 = xi (1 - alpha_k) */
  double nu_r, nu_b;      /* kinematic viscosities */
  double sigma, beta;     /* interfacial tension, recoloring parameter */
  double omega[11];       /* relaxation rates; omega[1] is replaced by 1/tau */
  double g[3];            /* acceleration vector for the body force */
  double rho_ref;         /* reference density for the buoyancy form */
  int32_t force_mode;     /* OCG_FORCE_* */
  int32_t model;          /* OCG_MODEL_* */
  int32_t use_Q;          /* 1: correction term Q of Sec. III.E applied */
  int32_t pad_;
  double wall_u[6][3];    /* velocity of the walls x-, x+, y-, y+, z-, z+ (moving walls) */
} ocg_params;

/* lattice tables: c[27*3] (row i = c_ix,c_iy,c_iz), w[27] */
void ocg_lattice(int32_t *c, double *w);

/* Hermite polynomial H_{i,abc} of App. B */
double ocg_hermite(int i, int a, int b, int c);

/* phase-space equilibria of Sec. III: model A (g2 + (p-rho cs2)E),
 * B (g6 + (p-rho cs2)E), C (g6 + (p-rho cs2)(E+Phi_3)), D (Eq. of Sec. III.D).
 * variant 4 = Li et al. original with g2 (Eq. of Sec. III.C, general form),
 * variant 5 = Eq. "standard CG 2nd" written with varphi_i (Sec. II.A),
 * variant 6 = Li et al. original written with varphi_i and D (Sec. III.C). */
void ocg_feq(int model, double rho, double p, const double u[3], double *feq);

/* raw and central moments by definition (Sec. II.B) */
void ocg_raw_moments(const double *f, double *m);
void ocg_central_moments(const double *f, const double u[3], double *k);
void ocg_moment_matrix(double *M);          /* M[r*27+i] */
void ocg_moment_matrix_inverse(double *Minv);/* Gauss-Jordan, partial pivoting */

/* collision in central-moment space, Eq. (general form) of Sec. II.B.
 * omega[11] must already hold omega_1 = 1/tau. */
void ocg_collide_cm(const double *k, const double *keq, const double *omega,
                    const double F[3], const double Q[3], double *kstar);
/* central moments about u -> raw moments (binomial shift) -> f = M^{-1} m */
void ocg_cm_to_f(const double *k, const double u[3], double *f);

/* whole-domain reference */
typedef struct ocg_domain ocg_domain;
ocg_domain *ocg_create(const ocg_params *prm);
void ocg_destroy(ocg_domain *d);
/* rho_r, rho_b: [N]; u: [3][N]; solid: [N] or NULL.  Populations at solid
 * cells start at zero. */
int ocg_init(ocg_domain *d, const double *rho_r, const double *rho_b,
             const double *u, const uint8_t *solid);
/* post-collision two-colour populations [27][N] each (paper order) */
int ocg_set_populations(ocg_domain *d, const double *fr, const double *fb);
int ocg_step(ocg_domain *d, int64_t nsteps);
/* macroscopic fields of the latest post-streaming state (or the initial
 * fields before the first step): rho_r, rho_b, p, phi: [N]; u: [3][N] */
void ocg_read_macros(const ocg_domain *d, double *rho_r, double *rho_b,
                     double *u, double *p, double *phi);
void ocg_read_populations(const ocg_domain *d, double *fr, double *fb);
/* intermediate fields of the latest step: which = 0 grad phi [3][N],
 * 1 n [3][N], 2 kappa [N], 3 F [3][N], 4 Q [3][N], 5 omega_1 [N],
 * 6 (p - rho cs2) u [3][N], 7 recoloring R [3][N] */
int ocg_read_field(const ocg_domain *d, int which, double *out);
/* per-colour mass over all cells (solid cells hold in-transit populations) */
void ocg_mass(const ocg_domain *d, double out[2]);
int64_t ocg_cells(const ocg_domain *d);
int ocg_threads(void);

#ifdef __cplusplus
}
#endif
#endif
