/*
 * cg27.h -- C ABI of the GB300 (sm_103a) implementation of the time step of
 * the three-dimensional two-component colour-gradient lattice Boltzmann model
 * with central-moment MRT collision and generalized equilibria
 * (S. Saito et al., arXiv 2309.07801).
 *
 * One time step, in the paper's terms:
 *   streaming  f_i(x + c_i, t+1) = f_i^*(x, t)                      (Sec. II.A)
 *   fields     rho_k, rho, rho u = sum f_i c_i + F/2, p, phi       (Sec. II.A)
 *   interface  grad phi, n, kappa = -div_s n, F_s = sigma kappa grad phi / 2
 *   correction Q = -3 d_a[(p - rho c_s^2) u_a]                      (Sec. III.E)
 *   collision  central-moment MRT toward the velocity-independent
 *              equilibrium central moments                      (Secs. II.B, III.D)
 *   recoloring f^{r,*}, f^{b,*} with R = beta rho_r rho_b p n / rho^2 (Sec. II.A)
 *   walls      fullway bounce-back at solid cells                    (Sec. IV)
 *
 * Conventions shared by every entry point
 *   - All values are in lattice units.  Cell (x, y, z) has linear index
 *     x + nx * (y + ny * z): x is fastest.  Vector fields are passed as three
 *     consecutive scalar fields (all x components, then y, then z).
 *   - Host arrays are owned by the caller; the library copies them in or out
 *     during the call and keeps no host pointer afterwards.
 *   - Device memory is owned by the caller: cg_workspace_bytes() tells how
 *     much, the caller allocates it (e.g. a uint8 CUDA tensor) and passes it to
 *     cg_create().  The library never calls cudaMalloc/cudaFree.
 *   - Work is enqueued on the CUDA stream given to cg_create() (NULL = the
 *     legacy default stream).  cg_step() returns without waiting; the read
 *     calls synchronise that stream before returning.
 *   - Every function returns CG_OK (0) or a negative CG_ERR_* code; the text of
 *     the last error of the calling thread is returned by cg_last_error().
 *     No exception crosses the ABI.
 *   - Population order at the ABI (cg_read_populations) is the 27-velocity
 *     order printed in Sec. II.A (the opposite of odd i is i + 1), or for a
 *     D2Q9 domain the 9-velocity order printed in App. A ([9][N] arrays).
 */
#ifndef CG27_H
#define CG27_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CG27_ABI_VERSION 5

/* return codes */
#define CG_OK 0
#define CG_ERR_INVALID_ARG (-1) /* bad pointer, size or parameter value */
#define CG_ERR_UNSUPPORTED (-2) /* valid request this build does not implement */
#define CG_ERR_CUDA (-3)        /* a CUDA runtime call failed (text has details) */
#define CG_ERR_NONFINITE (-4)   /* a non-finite density was produced */
#define CG_ERR_WORKSPACE (-5)   /* workspace missing, too small or misaligned */

/* boundary kind per axis.  Every wall kind makes cells 0 and n-1 of the axis
 * solid and uses the fullway bounce-back scheme (Sec. IV, introduction: no-slip,
 * slip and moving walls): what reaches a solid cell along c_j leaves it one step
 * later along c_i, colour by colour.
 *   BOUNCEBACK  c_i = -c_j (no-slip, wall at rest)
 *   SLIP        c_i = c_j with the wall-normal component negated (specular)
 *   MOVING      c_i = -c_j, plus 2 w_i rho_k (c_i . u_w) / c_s^2 for colour k,
 *               rho_k of the fluid cell the population came from and u_w the
 *               face's velocity in wall_u
 * A solid cell on several wall faces (an edge or corner of the box) is a slip
 * cell only if all those faces are slip walls (then every such normal component
 * is negated); otherwise it bounces back, with the sum of the velocities of its
 * moving faces.  Cells of the user's solid mask are no-slip walls at rest. */
#define CG_BC_PERIODIC 0
#define CG_BC_BOUNCEBACK 1
#define CG_BC_SLIP 2
#define CG_BC_MOVING 3

/* body force added to the interfacial force (Sec. IV test problems) */
#define CG_FORCE_NONE 0
#define CG_FORCE_CONST 1    /* F = g                    (layered flow, Sec. IV.C) */
#define CG_FORCE_GRAVITY 2  /* F = rho g                (rising bubble, Sec. IV.D) */
#define CG_FORCE_BUOYANCY 3 /* F = (rho - rho_ref) g    (Rayleigh-Taylor, Sec. IV.E) */

/* equilibrium central moments (Table "Summary of equilibria models") */
#define CG_MODEL_A 0 /* g^{eq,2} + (p - rho cs^2) E_i          (Sec. III.A) */
#define CG_MODEL_B 1 /* g^{eq,6} + (p - rho cs^2) E_i          (Sec. III.B) */
#define CG_MODEL_C 2 /* g^{eq,6}, Phi_i up to O(u^3) (Li et al.) (Sec. III.C) */
#define CG_MODEL_D 3 /* generalized equilibria, Phi_i up to O(u^6) (Sec. III.D) */

/* lattice */
#define CG_D3Q27 0
#define CG_D2Q9 1 /* the two-dimensional variant of App. A */

/* storage and arithmetic precision */
#define CG_F64 0   /* FP64 storage and arithmetic */
#define CG_F32 1   /* FP32 storage and arithmetic */
#define CG_F16S 2  /* populations stored in FP16 as deviations from the cell's
                      rest-state populations (the equilibrium at u = 0 of
                      Sec. II.A); everything else FP32; periodic domains of
                      at most 159 million cells (27 * cells < 2^32) only */
#define CG_BF16S 3 /* as CG_F16S with BF16 storage */

/* where the populations live between the collision and the next step's pull
 * (the paper streams between two copies, Sec. II):
 *   TWO_BUFFERS  two copies; a step pulls from one and writes the other
 *   IN_PLACE     one copy, updated in place in two alternating phases (the AA
 *                pattern): even steps read and write each cell's own slots
 *                with the directions reversed, odd steps read and write the
 *                neighbours' slots.  Half the population memory; results are
 *                bitwise those of TWO_BUFFERS.  D3Q27 only, not in batches. */
#define CG_STREAM_TWO_BUFFERS 0
#define CG_STREAM_IN_PLACE 1

typedef struct cg_params {
  int32_t nx, ny, nz;     /* cells per axis, each >= 1 (>= 3 on a wall axis) */
  int32_t bc[3];          /* CG_BC_* per axis (x, y, z) */
  double rho_r0, rho_b0;  /* reference densities of the red and blue fluids (> 0) */
  double alpha_r, alpha_b;/* rest fractions in [0, 1); (c_s^k)^2 = (9/19)(1 - alpha_k) */
  double nu_r, nu_b;      /* kinematic viscosities (>= 0) */
  double sigma;           /* interfacial tension coefficient */
  double beta;            /* recoloring parameter */
  double omega[11];       /* relaxation rates omega_0..omega_10 of the collision;
                             omega[1] is ignored (1/tau from the local viscosity) */
  double g[3];            /* acceleration vector used by the body-force modes */
  double rho_ref;         /* reference density of CG_FORCE_BUOYANCY */
  int32_t force_mode;     /* CG_FORCE_* */
  int32_t model;          /* CG_MODEL_* */
  int32_t use_Q;          /* 1: apply the correction term Q (Sec. III.E); 0: omit it */
  int32_t precision;      /* CG_F64, CG_F32, CG_F16S or CG_BF16S */
  int32_t solid_mask;     /* 1: cg_init_fields() may be given a solid mask (reserves
                             workspace for walls; implied by a wall axis) */
  int32_t lattice;        /* CG_D3Q27 (default) or CG_D2Q9 (App. A: nz = 1,
                             bc[2] periodic, periodic or bounce-back x/y, no
                             solid mask, Model D, FP64 or FP32) */
  double wall_u[6][3];    /* velocity of the faces x-, x+, y-, y+, z-, z+ of a
                             CG_BC_MOVING axis (finite; the component normal to
                             the face must be 0); ignored for other kinds */
  int32_t streaming;      /* CG_STREAM_TWO_BUFFERS (default) or CG_STREAM_IN_PLACE */
  int32_t reserved0;      /* must be 0 */
} cg_params;

typedef struct cg_ctx cg_ctx; /* opaque */

/* Fill *p with the defaults of Sec. III.E: Model D, Q on, all omega = 1,
 * rho_r0 = rho_b0 = 1, alpha = 8/27, nu = 0.1, sigma = 0, beta = 0.7,
 * periodic, no body force, FP32, and the given size. */
int cg_params_default(cg_params *p, int32_t nx, int32_t ny, int32_t nz);

/* Bytes of device workspace a domain with these parameters needs
 * (populations double-buffered, side fields, reduction scratch). */
int cg_workspace_bytes(const cg_params *p, size_t *bytes);

/* Create a domain.  d_workspace: device pointer of at least
 * cg_workspace_bytes() bytes, 256-byte aligned, owned by the caller and kept
 * alive until cg_destroy().  cuda_stream: a cudaStream_t (may be NULL).
 * The domain is not usable until cg_init_fields() succeeds. */
int cg_create(const cg_params *p, void *d_workspace, size_t bytes,
              void *cuda_stream, cg_ctx **out);

/* Initialise from host fields: rho_r[N], rho_b[N] (> 0 where fluid), u[3N]
 * (the velocity of the equilibrium), solid[N] (nonzero = solid cell; may be
 * NULL; non-NULL needs params.solid_mask or a wall axis).  Cells 0 and n-1
 * of a wall axis are solid whatever the mask.  Every fluid cell gets the
 * post-collision populations f_i^k = (rho_k / rho) f_i^eq(rho, p, u) of the
 * selected model; a solid cell starts with what the wall rule above makes of
 * the populations its fluid neighbours send it in that state (so the first
 * step sees no empty wall).  The first cg_step() begins with streaming. */
int cg_init_fields(cg_ctx *ctx, const double *rho_r, const double *rho_b,
                   const double *u, const uint8_t *solid);

/* Advance nsteps (>= 0) time steps, enqueued on the domain's stream
 * (asynchronous; returns after enqueueing).  A D3Q27 domain with nz >= 32 runs
 * as CUDA graphs of per-slab kernels (16-plane z slabs, the passes of
 * neighbouring slabs and of up to eight consecutive steps overlapping under
 * their data dependencies; see cg_set_schedule below); the first call with a
 * schedule builds all of its graphs (one step and an eight-step chain, for
 * either parity of the first step), so later calls spend no host time on
 * graph construction; while per-pass timing is on (cg_profile_enable) or the stream is
 * being captured by the caller, each pass is one plain launch instead.  The
 * results are the same either way, bit for bit.  CG_ERR_INVALID_ARG for a
 * negative count, a domain not initialised, or a member of a batch. */
int cg_step(cg_ctx *ctx, int64_t nsteps);

/* Schedule of the step graphs (D3Q27 domains with nz >= 32).  The z range is
 * cut into slabs of `planes` planes; each pass of each slab is one kernel
 * whose tiles march `tz` planes, and the passes of neighbouring slabs and of
 * up to eight steps overlap under their data dependencies (planes = nz: one
 * kernel per pass over the whole domain).  Thin slabs overlap more but repeat
 * the z halo of the stencil passes at every tile start.  Unless the caller
 * fixes it, the schedule is chosen by the library's tuner: the first chained
 * steps of the domain time the candidates -- 16/8, 32/16 and 64/32 planes per
 * slab / per tile where the domain holds two such slabs, and the whole domain
 * at the default depth -- one untimed and two timed eight-step chains each,
 * waiting for the GPU after each candidate, and keep the fastest.  These are
 * ordinary steps: results do not depend on the schedule, bit for bit.
 * cg_set_schedule(ctx, planes, tz) fixes it (1 <= planes <= nz,
 * 1 <= tz <= planes), cg_set_schedule(ctx, 0, 0) starts tuning again; both
 * wait for the domain's stream.  cg_schedule() reports the schedule in use
 * (0, 0 before the first graph step) and whether tuning is under way.
 *
 * Step form.  FP32 domains with two population buffers and no walls (and
 * 8 * stride + nx * ny < 2^31, stride = N rounded up to 64) can also run the
 * step as three passes: the collision of step t forms, in the same kernel,
 * the pulled colour and momentum sums of step t+1 (Sec. II.A streaming and
 * Eq. (recoloring) applied to the post-collision populations), so the
 * macroscopic pass and its second read of the populations leave the step.
 * Its tiles recompute a one-cell ring and one plane above and below (tiles of
 * fused_tz planes); the sums are added in the order of the macroscopic pass,
 * and the results are the same as with the four passes, bit for bit.  Per
 * cell it moves 392 bytes instead of 500 but repeats the collision on the
 * recomputed cells, which is issue-bound: on a GB300 the step is slower
 * (the fused pass takes 9.4 ms per 512^3 step against 8.0 ms for the
 * collision and the macroscopic pass), so the tuner keeps the four passes
 * and the form is chosen explicitly.  cg_set_schedule_form(ctx, planes, tz, fused_tz) fixes the
 * schedule and the form (fused_tz = 0: four passes; 1 <= fused_tz <= planes:
 * the fused pass; it also applies to the plain launches of domains below 32
 * planes or under per-pass timing), all 0 starts tuning again;
 * CG_ERR_UNSUPPORTED for fused_tz > 0 on a domain that cannot take it.
 * cg_set_schedule(ctx, p, tz) is cg_set_schedule_form(ctx, p, tz, 0).
 * cg_schedule_form() reports the form too.  Such a domain holds a second copy
 * of rho_r, rho_b, j (20 more bytes per cell). */
int cg_set_schedule(cg_ctx *ctx, int32_t planes, int32_t tz);
int cg_schedule(cg_ctx *ctx, int32_t *planes, int32_t *tz, int32_t *tuning);
int cg_set_schedule_form(cg_ctx *ctx, int32_t planes, int32_t tz, int32_t fused_tz);
int cg_schedule_form(cg_ctx *ctx, int32_t *planes, int32_t *tz, int32_t *fused_tz, int32_t *tuning);

/* Copy the fields of the latest post-streaming state to host arrays (each may
 * be NULL): rho_r[N], rho_b[N], u[3N] (Eq. for rho u, including F/2), p[N]
 * (Eq. pressure), phi[N] (Eq. order parameter).  Before the first step these
 * are the initial fields.  Solid cells report the densities of the populations
 * they hold and zero for u, p and phi. */
int cg_read_macros(cg_ctx *ctx, double *rho_r, double *rho_b, double *u,
                   double *p, double *phi);

/* Copy the post-collision, post-recoloring populations of both colours to host
 * arrays fr[27N], fb[27N] (population-major: fr[i*N + cell]); either may be
 * NULL. */
int cg_read_populations(cg_ctx *ctx, double *fr, double *fb);

/* Per-colour mass (sum over all cells, solid cells included) of the latest
 * state, accumulated in FP64 in a fixed order; *nonfinite is set to 1 if any
 * step since cg_init_fields() produced a non-finite density, else 0.  Either
 * pointer may be NULL. */
int cg_reduce(cg_ctx *ctx, double out_mass[2], int32_t *nonfinite);

/* Diagnostics of the latest state (the fields cg_read_macros() reports),
 * reduced on the device in FP64 in a fixed order (bitwise reproducible; no
 * field is read back to the host).  Cell (x, y, z) sits at coordinates
 * (x, y, z).  They are the quantities of the paper's tests:
 *   mass[k]            sum of rho_k over all cells (k = 0 red, 1 blue);
 *   red_volume         sum of (1 + phi)/2 over fluid cells (Eq. order
 *                      parameter; the droplet volume of the Laplace test);
 *   momentum[k][a]     sum of rho_k u_a over fluid cells (u includes F/2);
 *                      momentum[1][2] / mass[1] is the bubble velocity V_c of
 *                      Sec. IV.D when no solid cell holds blue mass;
 *   centroid[k][a]     rho_k-weighted centroid: the circular mean
 *                      (n/2pi) atan2(sum rho_k sin(2pi x/n), sum rho_k cos(2pi x/n))
 *                      in [0, n) along a periodic axis, sum rho_k x / sum rho_k
 *                      along a wall axis (the bubble height z_c of Sec. IV.D);
 *   second_moment[6]   sum rho_r d_a d_b / sum rho_r about the red centroid
 *                      (xx, yy, zz, xy, xz, yz), d the minimum-image offset
 *                      along periodic axes (droplet shape, Sec. IV.B);
 *   p_in, p_out        mean pressure (Eq. pressure) over fluid cells with
 *                      |x - center| < r_in and > r_out (minimum image along
 *                      periodic axes; NaN where no cell qualifies), n_in,
 *                      n_out the cell counts: p_in - p_out is the pressure
 *                      jump of the Laplace test (Sec. IV.A);
 *   u_max              largest |u| over fluid cells;
 *   nonfinite          as in cg_reduce().
 * center may be NULL (the origin); r_out may be +infinity (no outer cells).
 * Synchronises the domain's stream.  The scratch lives in the workspace. */
typedef struct cg_diagnostics {
  double mass[2];
  double red_volume;
  double momentum[2][3];
  double centroid[2][3];
  double second_moment[6];
  double p_in, p_out;
  int64_t n_in, n_out;
  double u_max;
  int32_t nonfinite;
  int32_t reserved;
} cg_diagnostics;
int cg_reduce_diagnostics(cg_ctx *ctx, const double center[3], double r_in,
                          double r_out, cg_diagnostics *out);

/* Checkpoint: cg_state_bytes() gives the size of an opaque host blob that
 * cg_save_state() fills and cg_load_state() restores into a domain created
 * with the same parameters.  A restored domain continues bit for bit. */
int cg_state_bytes(cg_ctx *ctx, size_t *bytes);
int cg_save_state(cg_ctx *ctx, void *host, size_t bytes);
int cg_load_state(cg_ctx *ctx, const void *host, size_t bytes);

/* Steps taken since cg_init_fields() (or as restored by cg_load_state()). */
int cg_steps_taken(cg_ctx *ctx, int64_t *steps);

/* Per-pass device timing.  cg_profile_enable(ctx, max_steps) makes the next
 * max_steps calls of the step loop record CUDA events around each of its
 * passes (max_steps = 0 turns timing off).  cg_profile_read() synchronises the
 * stream and returns, for passes 0..CG_NUM_PASSES-1 (streaming of both colours
 * and sums; gradient, normal, curvature, forces and recoloring state;
 * correction term and the divergence of R; streaming of the totals and
 * collision), the summed device
 * time in milliseconds and the number of timed steps. */
#define CG_NUM_PASSES 4
int cg_profile_enable(cg_ctx *ctx, int64_t max_steps);
int cg_profile_read(cg_ctx *ctx, double ms[CG_NUM_PASSES], int64_t *steps);

/* Per-colour mass of two device density fields, without any allocation.
 * The paper has no counterpart: this is a service of the library.  It is for
 * callers that cannot allocate device memory where they need the sums -- code
 * that only holds device pointers to density fields and owns no domain
 * workspace, or code running where cudaMalloc is not allowed (it may
 * synchronise the whole device, or another allocator already reserves all
 * device memory).  d_rho_r, d_rho_b: n values each on the current device, FP32
 * or FP64 as `precision` says; out_mass (host): sum of rho_r and of rho_b,
 * accumulated in FP64 in a fixed order (same values as cg_reduce() up to
 * summation order).  The block partial sums live in a 64 KiB file-scope
 * __device__ array that every GPU loading the library holds until the process
 * exits.  The first call on a device looks up that array's device address
 * (make it before any stream capture) and keeps it for the process: after a
 * cudaDeviceReset() of that device the kept address belongs to the destroyed
 * context, so the process must not call this function again.  Every call overwrites the slots it
 * reads, so nothing has to start at zero, but all calls share the one array:
 * calls that overlap on the GPU (other streams, other host threads) race.
 * n above CG_NOALLOC_MAX_CELLS is rejected with CG_ERR_INVALID_ARG before any
 * launch.  Enqueued on cuda_stream, which it synchronises before returning. */
#define CG_NOALLOC_MAX_CELLS 67108864
int cg_mass_noalloc(const void *d_rho_r, const void *d_rho_b, int64_t n,
                    int32_t precision, void *cuda_stream, double out_mass[2]);

/* Release the domain (the workspace stays the caller's).  A member of a batch
 * must be removed from it first (CG_ERR_INVALID_ARG otherwise). */
int cg_destroy(cg_ctx *ctx);

/* ---- batches: many domains advanced in shared launches -------------------
 * The paper has no counterpart: this is the library's way of running many
 * independent simulations (different sizes and parameters) at once.  The
 * members form up to four contiguous groups of about equal cell counts; a
 * batch step is four launches per group, each pass running over a work list
 * that concatenates the tiles of the group's members, with the arithmetic of
 * cg_step() for every cell.  A member's results are bitwise those of stepping
 * it alone in FP64, and within the storage precision's rounding in FP32 and
 * the 16-bit modes (the batched kernels are compiled separately and may fuse
 * other products into FMAs); they never depend on the other members.  The
 * launches are built into CUDA graphs (per step parity; eight steps per graph
 * when enough are requested) in which the groups' passes run concurrently;
 * the z depth of the tiles, the grid form and the tile shape (block size)
 * are tuned online by timing the candidates on the first steps after the
 * member set has changed by more than a factor two in cells (those steps are
 * ordinary steps: results do not depend on the schedule).
 *
 * Members must share the batch's precision and kernel variant (walls or none;
 * unit-rate Model D or not) and hold at most about 238 million cells (the
 * batch kernels use 32-bit population offsets), else CG_ERR_UNSUPPORTED.  While a domain is a
 * member, cg_step(), cg_init_fields(), cg_load_state() and cg_destroy() on it
 * fail with CG_ERR_INVALID_ARG; the read calls (cg_read_macros,
 * cg_read_populations, cg_reduce, cg_save_state) first wait for the batch's
 * stream.  cg_steps_taken() counts batch steps too. */
typedef struct cg_batch cg_batch;

/* Device bytes of the descriptor table and work lists of a batch of up to
 * max_domains members (1 <= max_domains <= 2^20) of the given precision. */
int cg_batch_workspace_bytes(int32_t max_domains, int32_t precision, size_t *bytes);

/* Create an empty batch.  d_workspace: device pointer of at least
 * cg_batch_workspace_bytes() bytes, 256-byte aligned, owned by the caller and
 * kept alive until cg_batch_destroy().  cuda_stream: the stream all batch
 * launches go to (NULL = the legacy default stream; the batch then uses plain
 * launches instead of graphs). */
int cg_batch_create(int32_t max_domains, int32_t precision, void *d_workspace, size_t bytes,
                    void *cuda_stream, cg_batch **out);

/* Add an initialised domain (synchronises the domain's own stream first).
 * Fails with CG_ERR_INVALID_ARG when the batch is full or the domain is
 * already a member of a batch. */
int cg_batch_add(cg_batch *batch, cg_ctx *ctx);

/* Remove a member (synchronises the batch stream first). */
int cg_batch_remove(cg_batch *batch, cg_ctx *ctx);

/* Number of members. */
int cg_batch_size(cg_batch *batch, int32_t *n);

/* Enqueue nsteps batch steps on the batch stream.  Returns without waiting,
 * except while the depth is being tuned (the tuned steps are timed with
 * events and synchronised). */
int cg_batch_step(cg_batch *batch, int64_t nsteps);

/* Wait for all enqueued batch steps. */
int cg_batch_sync(cg_batch *batch);

/* Fix the z depth of the tiles (planes per tile, > 0), or 0 to tune it
 * online again (together with the grid form unless that is fixed). */
int cg_batch_set_depth(cg_batch *batch, int32_t tz);

/* Current depth (0 before the first step) and whether tuning is under way. */
int cg_batch_depth(cg_batch *batch, int32_t *tz, int32_t *tuning);

/* Grid form of the batch kernels: 0 one block per work item (tile or 128
 * cells), 1 persistent (each group's kernels launch its share of the blocks the
 * GPU holds at once, which walk the work list), or -1 to let the online tuner
 * choose (the default; it times both forms at each candidate depth).  Results
 * do not depend on the form.  CG_ERR_INVALID_ARG for other values. */
int cg_batch_set_persistent(cg_batch *batch, int32_t mode);

/* The grid form in use (0 or 1). */
int cg_batch_persistent(cg_batch *batch, int32_t *mode);

/* Step budget of a member: it takes part in the batch's steps until its step
 * count (cg_steps_taken) reaches total_steps, and sits out the remaining
 * steps of every later cg_batch_step() call (its work items return at once),
 * so that members with different step counts share one call and no member
 * has to stop the others at its own count.  total_steps < 0 removes the
 * budget (the default, and what joining or leaving a batch sets).  Waits for
 * the batch's stream.  CG_ERR_INVALID_ARG if the domain is not a member. */
int cg_batch_set_stop(cg_batch *batch, cg_ctx *ctx, int64_t total_steps);

/* Tile shape of the z-marching batch passes (the block size and the layout
 * of their shared-memory rings): 0 = 32 x 8 threads, 1 = 32 x 4 threads, or
 * -1 to let the online tuner choose (the default; it times every candidate
 * depth and grid form with both shapes).  Results do not depend on the shape.
 * CG_ERR_INVALID_ARG for other values.  cg_batch_tile() reports the shape in
 * use as tile_nx x tile_ny threads. */
int cg_batch_set_tile(cg_batch *batch, int32_t shape);
int cg_batch_tile(cg_batch *batch, int32_t *tile_nx, int32_t *tile_ny);

/* Release the batch (waits for its stream; members become free domains). */
int cg_batch_destroy(cg_batch *batch);

/* Text of the last error on the calling thread ("" if none). */
const char *cg_last_error(void);

/* ABI version of the loaded library (CG27_ABI_VERSION). */
int cg_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif /* CG27_H */
