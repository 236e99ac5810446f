// cg27_device.cuh -- device code of the D3Q27 colour-gradient CM-MRT step
// (arXiv 2309.07801) for sm_103a.
//
// Data layout in device memory (structure of arrays, x fastest, each scalar
// field `stride` elements long):
//   F[27]   post-collision total populations f_i^* (two ping-pong copies);
//           at solid cells the same slots hold the red part of the stored
//           (bounced) populations;
//   S[6]    recoloring state of each cell: rho_r/rho, rho_b/rho, R_x, R_y, R_z
//           and DIVR (two ping-pong copies).  The two-colour post-collision
//           populations of Eq. (recoloring) are f^{r,*}_i = (rho_r/rho) f_i^*
//           + (w_i/c_s^2) c_i.R and f^{b,*}_i = (rho_b/rho) f_i^* - (w_i/c_s^2)
//           c_i.R, so (F, S) holds the full two-colour state in 27 + 5 values.
//           DIVR(x) = sum_i (w_i/c_s^2) c_i.R(x - c_i) is what the R terms add
//           to rho_r (and take from rho_b) after the next pull; it is computed
//           once per cell by the divergence pass so that the pull needs only
//           the two fractions of each source cell.  The 16-bit modes add a
//           seventh field, the rest-direction reference;
//   AUX[27] blue part at solid cells (only with walls, two copies);
//   MASK    per cell: bit q set when the neighbour x + c_q is solid, bit 27
//           when the cell itself is solid (only with walls);
//   MAC[5]  rho_r, rho_b, j_x, j_y, j_z of the post-streaming state;
//   PHI     order parameter; FORCE[3] total force; WV[3] (p - rho c_s^2) u;
//   QC[3]   correction term Q.
// Lattice directions are stored in the lexicographic order
// q = (c_x+1) + 3 (c_y+1) + 9 (c_z+1); moments use r = a + 3 b + 9 c.
//
// One step is four kernels (cg27_step.cuh): k_macro (pull both colours and
// sum), k_fields (colour gradient, normal, curvature, forces, velocity,
// (p - rho c_s^2) u, recoloring state), k_div_sep (correction term Q and DIVR)
// and k_collide (pull the totals, CM-MRT collision, store f^*; recoloring is
// applied by the next pull).
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace cg27 {

// ---- lattice ---------------------------------------------------------------

__host__ __device__ constexpr int CX(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int CY(int q) { return (q / 3) % 3 - 1; }
__host__ __device__ constexpr int CZ(int q) { return q / 9 - 1; }
__host__ __device__ constexpr int OPP(int q) { return 26 - q; }
__host__ __device__ constexpr int CC(int q) { return CX(q) * CX(q) + CY(q) * CY(q) + CZ(q) * CZ(q); }
__host__ __device__ constexpr int CA(int q, int a) { return a == 0 ? CX(q) : (a == 1 ? CY(q) : CZ(q)); }
__host__ __device__ constexpr int KI(int a, int b, int c) { return a + 3 * b + 9 * c; }
constexpr int REST = 13;
constexpr int SELF_SOLID_BIT = 27;

// D3Q27 weights by |c|^2 (Sec. II.A)
template <typename T>
__host__ __device__ constexpr T WQ(int q) {
  return CC(q) == 0 ? T(8) / T(27)
                    : (CC(q) == 1 ? T(2) / T(27) : (CC(q) == 2 ? T(1) / T(54) : T(1) / T(216)));
}

template <typename T>
struct Lat {
  static constexpr T CS2 = T(1) / T(3);  // lattice speed of sound squared
  static constexpr T CS4 = CS2 * CS2;
};

// ---- kernel arguments --------------------------------------------------------

struct Geom {
  int nx, ny, nz, nxy;
  long long stride;  // elements between consecutive scalar fields
};

template <typename T>
struct Ptrs {
  const void* f_in;  // populations, stored as the storage type of the mode
  void* f_out;
  const T* s_in;
  T* s_out;
  const T* aux_in;
  T* aux_out;
  const uint32_t* mask;
  T* mac;      // rho_r, rho_b, j of the step (written by its macroscopic pass)
  T* mac_out;  // of the next step (written by the fused collision pass)
  T* phi;
  T* qc;  // correction term Q
  T* force;
  T* wv;
  unsigned int* flag;
};

template <typename T>
struct Phys {
  T rho_r0, rho_b0;
  T inv_rho_r0, inv_rho_b0;
  T cr2, cb2;  // (c_s^k)^2 = xi (1 - alpha_k)
  T nu_r, nu_b;
  T sigma, beta;
  T om[11];
  T g[3];
  T rho_ref;
  int force_mode, model, use_Q;
  int shift;  // populations stored as deviations from the rest state (16-bit modes)
  T rest1;    // p_ref / c_s^2: the moving rest-state populations are w_q rest1
  int bc[3];         // wall kind per axis (the CG_BC_* values of cg27.h)
  T wall_u[6][3];    // velocity of the faces x-, x+, y-, y+, z-, z+ (moving walls; else 0)
};

// wall kinds per axis, as in cg27.h
constexpr int BC_PERIODIC = 0, BC_SLIP = 2, BC_MOVING = 3;

// ---- population storage ---------------------------------------------------------------
// FP64/FP32 store f_q itself.  The 16-bit modes store the deviation of f_q from
// a rest-state population (the equilibrium at u = 0 of Sec. II.A), divided by
// the lattice weight w_q (pop_encode / pop_decode below):
//   moving directions:  w_q p / c_s^2 with a global reference pressure p_ref
//                       (pressure balance keeps p close to p_ref in both
//                       phases, so no per-cell value has to travel);
//   rest direction:     rho - p / xi of the cell itself, stored in FP32 as
//                       field S_REST of the recoloring state (the rest population
//                       stays in its cell, so only the cell's own value is read).
template <typename SF>
struct Store {
  static constexpr bool SHIFT = false;
  template <typename T>
  __device__ static T get(const SF* p) { return T(__ldg(p)); }
  template <typename T>
  __device__ static SF put(T v) { return SF(v); }
};
template <>
struct Store<__half> {
  static constexpr bool SHIFT = true;
  template <typename T>
  __device__ static T get(const __half* p) { return T(__half2float(__ldg(p))); }
  template <typename T>
  __device__ static __half put(T v) { return __float2half_rn(float(v)); }
};
template <>
struct Store<__nv_bfloat16> {
  static constexpr bool SHIFT = true;
  template <typename T>
  __device__ static T get(const __nv_bfloat16* p) { return T(__bfloat162float(__ldg(p))); }
  template <typename T>
  __device__ static __nv_bfloat16 put(T v) { return __float2bfloat16_rn(float(v)); }
};

// fields of the recoloring state: rho_r/rho, rho_b/rho, R (3) [, rho - p/xi]
template <typename SF>
__host__ __device__ constexpr int ns_of() { return Store<SF>::SHIFT ? 7 : 6; }
// fields of the recoloring state after rho_r/rho, rho_b/rho and R
constexpr int S_DIVR = 5;  // sum over directions of the recoloring term of the source cells
constexpr int S_REST = 6;  // rest-direction reference of the 16-bit modes

// rest population of the rest direction of a cell
template <typename T>
__device__ __forceinline__ T rest_zero(T rho, T p) {
  return rho - p * (T(19) / T(9));  // 1/xi, xi = 9/19 for D3Q27
}

// 16-bit modes: the stored value is the deviation from the rest-state
// population divided by the lattice weight, (f_q - rest_q) / w_q, so that all
// directions use the same range of the format (the corner directions' small
// deviations stay out of the FP16 subnormals); one FMA each way.
template <bool SHIFT, typename T>
__device__ __forceinline__ T pop_decode(int q, T s, T r0, T rest1) {
  if (!SHIFT) return s;
  return s * WQ<T>(q) + (q == REST ? r0 : WQ<T>(q) * rest1);
}
template <bool SHIFT, typename T>
__device__ __forceinline__ T pop_encode(int q, T f, T r0, T rest1) {
  if (!SHIFT) return f;
  return q == REST ? (f - r0) * (T(1) / WQ<T>(q)) : f * (T(1) / WQ<T>(q)) - rest1;
}

template <typename SF>
__device__ __forceinline__ const SF* fin(const void* p) { return static_cast<const SF*>(p); }
template <typename SF>
__device__ __forceinline__ SF* fout(void* p) { return static_cast<SF*>(p); }

// ---- cell addressing -----------------------------------------------------------

struct Cell {
  int idx;
  int x, y, z;
  int xs[3], ys[3], zs[3];  // offsets of x-1, x, x+1 (etc.) with periodic wrap
};

// the cell (x, y, z), which must lie inside the domain
__device__ __forceinline__ void make_cell_at(const Geom& g, int x, int y, int z, Cell& c) {
  c.x = x;
  c.y = y;
  c.z = z;
  c.xs[0] = (x == 0 ? g.nx - 1 : x - 1);
  c.xs[1] = x;
  c.xs[2] = (x == g.nx - 1 ? 0 : x + 1);
  c.ys[0] = (y == 0 ? g.ny - 1 : y - 1) * g.nx;
  c.ys[1] = y * g.nx;
  c.ys[2] = (y == g.ny - 1 ? 0 : y + 1) * g.nx;
  c.zs[0] = (z == 0 ? g.nz - 1 : z - 1) * g.nxy;
  c.zs[1] = z * g.nxy;
  c.zs[2] = (z == g.nz - 1 ? 0 : z + 1) * g.nxy;
  c.idx = x + c.ys[1] + c.zs[1];
}

// the cell of this thread in a (x, y) block grid with one z plane per blockIdx.z
__device__ __forceinline__ bool make_cell(const Geom& g, Cell& c) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return false;
  make_cell_at(g, x, y, blockIdx.z, c);
  return true;
}

// index of the cell x + (dx, dy, dz), each in {-1, 0, 1}
__device__ __forceinline__ int nbr(const Cell& c, int dx, int dy, int dz) {
  return c.xs[dx + 1] + c.ys[dy + 1] + c.zs[dz + 1];
}

template <typename T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

// ---- where populations live: two buffers, or one buffer updated in place -------
// Stream modes of a step.  Two buffers (pull): cell x reads the population of
// direction q from the input buffer at (q, x - c_q) and writes its
// post-collision value to the output buffer at (q, x).  In place (one buffer,
// two alternating phases, the AA pattern):
//   even step: read (q, x),            write (opp q, x)
//   odd step:  read (opp q, x - c_q),  write (q, x + c_q)
// Every location is read and then written by one cell only, within the
// macroscopic pass and the collision of a step, so the update needs no second
// buffer, and the read-only load path never meets a location after its write.
// Between steps the post-collision value of direction q of cell x sits at
// (q, x + c_q) before an even step and at (opp q, x) before an odd one.
constexpr int SM_AB = 0, SM_EVEN = 1, SM_ODD = 2;
template <int SM>
__host__ __device__ constexpr int rd_dir(int q) { return SM == SM_ODD ? OPP(q) : q; }
template <int SM>
__host__ __device__ constexpr int wr_dir(int q) { return SM == SM_EVEN ? OPP(q) : q; }
// the read cell is x + rd_sign * c_q
template <int SM>
__host__ __device__ constexpr int rd_sign() { return SM == SM_EVEN ? 0 : -1; }

// element index of the population of direction q that cell c pulls at a step
// of mode sm (run-time form, for the kernels outside the step)
__device__ __forceinline__ long long pull_index(int sm, int q, long long S, const Cell& c) {
  if (sm == SM_EVEN) return q * S + c.idx;
  const int src = nbr(c, -CX(q), -CY(q), -CZ(q));
  return (sm == SM_ODD ? OPP(q) : q) * S + src;
}
// element index of the post-collision population of direction q of cell c,
// as written by a step of mode sm
__device__ __forceinline__ long long emit_index(int sm, int q, long long S, const Cell& c) {
  if (sm == SM_EVEN) return OPP(q) * S + c.idx;
  if (sm == SM_ODD) return q * S + nbr(c, CX(q), CY(q), CZ(q));
  return q * S + c.idx;
}
// stream mode of the step that follows `steps` steps
__host__ __device__ inline int next_mode(int inplace, long long steps) {
  return inplace ? ((steps & 1) ? SM_ODD : SM_EVEN) : SM_AB;
}
// stream mode of the step that left the state after `steps` steps (the
// initial state is laid out as if an odd step had written it)
__host__ __device__ inline int last_mode(int inplace, long long steps) {
  return inplace ? ((steps & 1) ? SM_EVEN : SM_ODD) : SM_AB;
}

// ---- pull of one direction with the colour split of Eq. (recoloring) -------------

// q: direction, src: the source cell x - c_q (its recoloring state), pidx: the
// element index of the population in the buffers (q * stride + src with two
// buffers)
template <typename T, typename SF, bool SOLID>
__device__ __forceinline__ void pull_colour(const Ptrs<T>& P, long long stride, int q, int src, long long pidx,
                                            uint32_t mask, T& fr, T& fb, T& ft, T ph_rest1 = T(0)) {
  static_assert(!(SOLID && Store<SF>::SHIFT), "walls are not available with 16-bit populations");
  T f = Store<SF>::template get<T>(fin<SF>(P.f_in) + pidx);
  if (Store<SF>::SHIFT)
    f = pop_decode<true>(q, f, q == REST ? ld(P.s_in + S_REST * stride + src) : T(0), ph_rest1);
  if (SOLID && ((mask >> OPP(q)) & 1u)) {
    // the source is solid: it stores the red part in F and the blue part in AUX
    fr = f;
    fb = ld(P.aux_in + pidx);
    ft = fr + fb;
  } else {
    const T a = ld(P.s_in + src);
    const T b = ld(P.s_in + stride + src);
    T t = T(0);
    if (q != REST) {
      T cR = T(0);
      if (CX(q) != 0) cR += T(CX(q)) * ld(P.s_in + 2 * stride + src);
      if (CY(q) != 0) cR += T(CY(q)) * ld(P.s_in + 3 * stride + src);
      if (CZ(q) != 0) cR += T(CZ(q)) * ld(P.s_in + 4 * stride + src);
      t = (WQ<T>(q) / Lat<T>::CS2) * cR;
    }
    fr = a * f + t;
    fb = b * f - t;
    ft = f;
  }
}

// ---- walls (Sec. IV, introduction: no-slip, slip and moving walls, fullway) ---------------
// Rule of a solid cell: returns the axes whose velocity component a slip wall
// negates (nonzero: specular reflection) or 0 for bounce-back, with uw the
// summed velocity of the cell's moving faces.  A cell is a slip cell only if
// all of its wall faces are slip walls; obstacle cells bounce back at rest.
template <typename T>
__device__ __forceinline__ int wall_rule(const Geom& g, const Phys<T>& ph, const Cell& c, T (&uw)[3]) {
  const int xyz[3] = {c.x, c.y, c.z}, n[3] = {g.nx, g.ny, g.nz};
  int slip = 0, other = 0, flip = 0;
  uw[0] = uw[1] = uw[2] = T(0);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (ph.bc[a] == BC_PERIODIC) continue;
    const int face = xyz[a] == 0 ? 2 * a : (xyz[a] == n[a] - 1 ? 2 * a + 1 : -1);
    if (face < 0) continue;
    if (ph.bc[a] == BC_SLIP) {
      ++slip;
      flip |= 1 << a;
    } else {
      ++other;
      if (ph.bc[a] == BC_MOVING)
#pragma unroll
        for (int b = 0; b < 3; ++b) uw[b] += ph.wall_u[face][b];
    }
  }
  return (other == 0 && slip > 0) ? flip : 0;
}

// direction q with the components of the axes in `flip` negated
__device__ __forceinline__ int reflect_dir(int q, int flip) {
  const int cx = (flip & 1) ? -CX(q) : CX(q);
  const int cy = (flip & 2) ? -CY(q) : CY(q);
  const int cz = (flip & 4) ? -CZ(q) : CZ(q);
  return (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1);
}

// The wall rule applied to the colour parts (fr, fb) of the population that
// arrived along c_q from the cell src: returns the direction it leaves along
// next step and adds the moving-wall term 2 w_i rho_k (c_i . u_w) / c_s^2
// (rho_k of the source cell: rr, rb) for a bounce-back cell.
template <typename T>
__device__ __forceinline__ int wall_emit(int q, int flip, const T (&uw)[3], T rr, T rb, T& fr, T& fb) {
  if (flip) return reflect_dir(q, flip);
  const T cu = T(CX(q)) * uw[0] + T(CY(q)) * uw[1] + T(CZ(q)) * uw[2];  // c_q . u_w = -c_i . u_w
  const T k = -T(2) * WQ<T>(q) * cu / Lat<T>::CS2;
  fr += k * rr;
  fb += k * rb;
  return OPP(q);
}

// ---- order parameter, Eq. (order parameter) --------------------------------------

template <typename T>
__device__ __forceinline__ T order_parameter(T rr, T rb, const Phys<T>& ph) {
  const T a = rr * ph.inv_rho_r0, b = rb * ph.inv_rho_b0;
  return (a + b > T(0)) ? (a - b) / (a + b) : T(0);
}

// ---- factorised central-moment transforms ---------------------------------------
// One axis: values at c = -1, 0, +1 <-> central moments of order 0, 1, 2 about u.
// Forward: k0 = sum f, k1 = sum f (c-u), k2 = sum f (c-u)^2.
template <typename T>
__device__ __forceinline__ void fwd3(T& fm, T& fz, T& fp, T u) {
  const T s = fp + fm, d = fp - fm;
  const T k0 = s + fz;
  const T k1 = d - u * k0;
  const T k2 = s - u * (d + k1);
  fm = k0;
  fz = k1;
  fp = k2;
}
// Inverse: raw moments m1 = k1 + u k0, m2 = k2 + 2 u k1 + u^2 k0, then the
// three-point inverse f(-1) = (m2 - m1)/2, f(0) = m0 - m2, f(1) = (m1 + m2)/2.
template <typename T>
__device__ __forceinline__ void bwd3(T& k0, T& k1, T& k2, T u) {
  const T m1 = k1 + u * k0;
  const T m2 = k2 + u * (k1 + m1);
  const T fm = T(0.5) * (m2 - m1);
  const T fz = k0 - m2;
  const T fp = T(0.5) * (m1 + m2);
  k0 = fm;
  k1 = fz;
  k2 = fp;
}

template <typename T>
__device__ __forceinline__ void forward_cm(T (&f)[27], T ux, T uy, T uz) {
#pragma unroll
  for (int l = 0; l < 9; ++l) fwd3(f[3 * l], f[3 * l + 1], f[3 * l + 2], ux);
#pragma unroll
  for (int iz = 0; iz < 3; ++iz)
#pragma unroll
    for (int a = 0; a < 3; ++a) fwd3(f[a + 9 * iz], f[a + 9 * iz + 3], f[a + 9 * iz + 6], uy);
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) fwd3(f[a + 3 * b], f[a + 3 * b + 9], f[a + 3 * b + 18], uz);
}

template <typename T>
__device__ __forceinline__ void backward_cm(T (&k)[27], T ux, T uy, T uz) {
#pragma unroll
  for (int b = 0; b < 3; ++b)
#pragma unroll
    for (int a = 0; a < 3; ++a) bwd3(k[a + 3 * b], k[a + 3 * b + 9], k[a + 3 * b + 18], uz);
#pragma unroll
  for (int iz = 0; iz < 3; ++iz)
#pragma unroll
    for (int a = 0; a < 3; ++a) bwd3(k[a + 9 * iz], k[a + 9 * iz + 3], k[a + 9 * iz + 6], uy);
#pragma unroll
  for (int l = 0; l < 9; ++l) bwd3(k[3 * l], k[3 * l + 1], k[3 * l + 2], ux);
}

// ---- equilibrium central moments (Secs. III.A-III.D) ------------------------------

template <typename T>
__device__ __forceinline__ void keq_model(int model, T rho, T p, T ux, T uy, T uz, T (&e)[27]) {
  const T cs2 = Lat<T>::CS2, cs4 = Lat<T>::CS4;
  const T d = p - rho * cs2;
  const T x2 = ux * ux, y2 = uy * uy, z2 = uz * uz;
#pragma unroll
  for (int r = 0; r < 27; ++r) e[r] = T(0);
  e[KI(0, 0, 0)] = rho;
  e[KI(2, 0, 0)] = e[KI(0, 2, 0)] = e[KI(0, 0, 2)] = p;
  if (model == 3) {  // Model D: velocity independent
    e[KI(2, 2, 0)] = e[KI(2, 0, 2)] = e[KI(0, 2, 2)] = p * cs2;
    e[KI(2, 2, 2)] = p * cs4;
  } else if (model == 2) {  // Model C
    e[KI(2, 2, 0)] = p * cs2 - d * (x2 + y2);
    e[KI(2, 0, 2)] = p * cs2 - d * (x2 + z2);
    e[KI(0, 2, 2)] = p * cs2 - d * (y2 + z2);
    e[KI(2, 1, 1)] = -d * uy * uz;
    e[KI(1, 2, 1)] = -d * ux * uz;
    e[KI(1, 1, 2)] = -d * ux * uy;
    e[KI(1, 2, 2)] = d * ux * (T(2) * y2 + T(2) * z2 + cs2);
    e[KI(2, 1, 2)] = d * uy * (T(2) * x2 + T(2) * z2 + cs2);
    e[KI(2, 2, 1)] = d * uz * (T(2) * x2 + T(2) * y2 + cs2);
    e[KI(2, 2, 2)] = p * cs4 - T(3) * d * (x2 * y2 + x2 * z2 + y2 * z2 + cs2 * (x2 + y2 + z2));
  } else {  // Models A (0) and B (1) share the terms in (p - rho cs2)
    e[KI(1, 2, 0)] = -d * ux;
    e[KI(1, 0, 2)] = -d * ux;
    e[KI(0, 1, 2)] = -d * uy;
    e[KI(2, 1, 0)] = -d * uy;
    e[KI(2, 0, 1)] = -d * uz;
    e[KI(0, 2, 1)] = -d * uz;
    e[KI(2, 2, 0)] = p * cs2 + d * (x2 + y2);
    e[KI(2, 0, 2)] = p * cs2 + d * (x2 + z2);
    e[KI(0, 2, 2)] = p * cs2 + d * (y2 + z2);
    e[KI(2, 1, 1)] = d * uy * uz;
    e[KI(1, 2, 1)] = d * ux * uz;
    e[KI(1, 1, 2)] = d * ux * uy;
    e[KI(1, 2, 2)] = -d * ux * (y2 + z2 + cs2);
    e[KI(2, 1, 2)] = -d * uy * (x2 + z2 + cs2);
    e[KI(2, 2, 1)] = -d * uz * (x2 + y2 + cs2);
    e[KI(2, 2, 2)] = p * cs4 + d * (x2 * y2 + x2 * z2 + y2 * z2 + cs2 * (x2 + y2 + z2));
    if (model == 0) {  // the extra rho u terms of Model A
      e[KI(1, 2, 0)] -= rho * ux * y2;
      e[KI(1, 0, 2)] -= rho * ux * z2;
      e[KI(0, 1, 2)] -= rho * uy * z2;
      e[KI(2, 1, 0)] -= rho * x2 * uy;
      e[KI(2, 0, 1)] -= rho * x2 * uz;
      e[KI(0, 2, 1)] -= rho * y2 * uz;
      e[KI(1, 1, 1)] = -rho * ux * uy * uz;
      e[KI(2, 2, 0)] += T(3) * rho * x2 * y2;
      e[KI(2, 0, 2)] += T(3) * rho * x2 * z2;
      e[KI(0, 2, 2)] += T(3) * rho * y2 * z2;
      e[KI(2, 1, 1)] += T(3) * rho * x2 * uy * uz;
      e[KI(1, 2, 1)] += T(3) * rho * ux * y2 * uz;
      e[KI(1, 1, 2)] += T(3) * rho * ux * uy * z2;
      e[KI(1, 2, 2)] -= rho * ux * (T(6) * y2 * z2 + cs2 * (y2 + z2));
      e[KI(2, 1, 2)] -= rho * uy * (T(6) * x2 * z2 + cs2 * (x2 + z2));
      e[KI(2, 2, 1)] -= rho * uz * (T(6) * x2 * y2 + cs2 * (x2 + y2));
      e[KI(2, 2, 2)] += rho * (T(10) * x2 * y2 * z2 + T(3) * cs2 * (x2 * y2 + x2 * z2 + y2 * z2));
    }
  }
}

// ---- collision in central-moment space ----------------------------------------------
// General form of Sec. II.B (any omega, any model), or the unit-rate Model D form
// of Sec. III.E (all omega = 1 except omega_1) when UNIT is true.  On entry f
// holds the pre-collision populations, on exit the post-collision ones.
template <typename T, bool UNIT>
__device__ __forceinline__ void collide_cm(T (&f)[27], T rho, T p, T ux, T uy, T uz,
                                           const T (&F)[3], const T (&Q)[3], T om1,
                                           const Phys<T>& ph) {
  const T cs2 = Lat<T>::CS2, cs4 = Lat<T>::CS4;
  const T third = T(1) / T(3);
  forward_cm(f, ux, uy, uz);
  T(&k)[27] = f;
  if (UNIT) {
    k[KI(1, 0, 0)] = F[0] / T(2);
    k[KI(0, 1, 0)] = F[1] / T(2);
    k[KI(0, 0, 1)] = F[2] / T(2);
    k[KI(1, 1, 0)] = (T(1) - om1) * k[KI(1, 1, 0)];
    k[KI(0, 1, 1)] = (T(1) - om1) * k[KI(0, 1, 1)];
    k[KI(1, 0, 1)] = (T(1) - om1) * k[KI(1, 0, 1)];
    const T h1 = T(1) - om1 / T(2);
    const T d1 = (T(1) - om1) * (k[KI(2, 0, 0)] - k[KI(0, 2, 0)]) + h1 * (Q[0] - Q[1]);
    const T d2 = (T(1) - om1) * (k[KI(2, 0, 0)] - k[KI(0, 0, 2)]) + h1 * (Q[0] - Q[2]);
    const T tr = T(3) * p + (Q[0] + Q[1] + Q[2]) / T(2);
    k[KI(2, 0, 0)] = (tr + d1 + d2) * third;
    k[KI(0, 2, 0)] = (tr - T(2) * d1 + d2) * third;
    k[KI(0, 0, 2)] = (tr + d1 - T(2) * d2) * third;
    k[KI(1, 2, 0)] = k[KI(1, 0, 2)] = cs2 * F[0] / T(2);
    k[KI(2, 1, 0)] = k[KI(0, 1, 2)] = cs2 * F[1] / T(2);
    k[KI(2, 0, 1)] = k[KI(0, 2, 1)] = cs2 * F[2] / T(2);
    k[KI(1, 1, 1)] = T(0);
    k[KI(2, 2, 0)] = k[KI(2, 0, 2)] = k[KI(0, 2, 2)] = p * cs2;
    k[KI(2, 1, 1)] = k[KI(1, 2, 1)] = k[KI(1, 1, 2)] = T(0);
    k[KI(1, 2, 2)] = cs4 * F[0] / T(2);
    k[KI(2, 1, 2)] = cs4 * F[1] / T(2);
    k[KI(2, 2, 1)] = cs4 * F[2] / T(2);
    k[KI(2, 2, 2)] = p * cs4;
  } else {
    T e[27];
    keq_model(ph.model, rho, p, ux, uy, uz, e);
    const T* om = ph.om;
    const T o0 = om[0], o2 = om[2], o3 = om[3], o4 = om[4], o5 = om[5], o6 = om[6],
            o7 = om[7], o8 = om[8], o9 = om[9], o10 = om[10];
    // first order
    k[KI(1, 0, 0)] = (T(1) - o0) * k[KI(1, 0, 0)] + (T(1) - o0 / T(2)) * F[0];
    k[KI(0, 1, 0)] = (T(1) - o0) * k[KI(0, 1, 0)] + (T(1) - o0 / T(2)) * F[1];
    k[KI(0, 0, 1)] = (T(1) - o0) * k[KI(0, 0, 1)] + (T(1) - o0 / T(2)) * F[2];
    // second order
    k[KI(1, 1, 0)] = (T(1) - om1) * k[KI(1, 1, 0)] + om1 * e[KI(1, 1, 0)];
    k[KI(0, 1, 1)] = (T(1) - om1) * k[KI(0, 1, 1)] + om1 * e[KI(0, 1, 1)];
    k[KI(1, 0, 1)] = (T(1) - om1) * k[KI(1, 0, 1)] + om1 * e[KI(1, 0, 1)];
    {
      const T a = k[KI(2, 0, 0)], b = k[KI(0, 2, 0)], c = k[KI(0, 0, 2)];
      const T ea = e[KI(2, 0, 0)], eb = e[KI(0, 2, 0)], ec = e[KI(0, 0, 2)];
      const T h1 = T(1) - om1 / T(2);
      const T d1 = (T(1) - om1) * (a - b) + om1 * (ea - eb) + h1 * (Q[0] - Q[1]);
      const T d2 = (T(1) - om1) * (a - c) + om1 * (ea - ec) + h1 * (Q[0] - Q[2]);
      const T tr = (T(1) - o2) * (a + b + c) + o2 * (ea + eb + ec) +
                   (T(1) - o2 / T(2)) * (Q[0] + Q[1] + Q[2]);
      k[KI(2, 0, 0)] = (tr + d1 + d2) * third;
      k[KI(0, 2, 0)] = (tr - T(2) * d1 + d2) * third;
      k[KI(0, 0, 2)] = (tr + d1 - T(2) * d2) * third;
    }
    // third order: sums relax with omega_3 (with forcing), differences with omega_4
    {
      const int p1[3] = {KI(1, 2, 0), KI(2, 1, 0), KI(2, 0, 1)};
      const int p2[3] = {KI(1, 0, 2), KI(0, 1, 2), KI(0, 2, 1)};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T k1 = k[p1[a]], k2 = k[p2[a]], e1 = e[p1[a]], e2 = e[p2[a]];
        const T s = (T(1) - o3) * (k1 + k2) + o3 * (e1 + e2) + T(2) * (T(1) - o3 / T(2)) * F[a] * cs2;
        const T dd = (T(1) - o4) * (k1 - k2) + o4 * (e1 - e2);
        k[p1[a]] = (s + dd) / T(2);
        k[p2[a]] = (s - dd) / T(2);
      }
      k[KI(1, 1, 1)] = (T(1) - o5) * k[KI(1, 1, 1)] + o5 * e[KI(1, 1, 1)];
    }
    // fourth order
    {
      const T a = k[KI(2, 2, 0)], b = k[KI(2, 0, 2)], c = k[KI(0, 2, 2)];
      const T ea = e[KI(2, 2, 0)], eb = e[KI(2, 0, 2)], ec = e[KI(0, 2, 2)];
      const T A = (T(1) - o6) * (a - T(2) * b + c) + o6 * (ea - T(2) * eb + ec);
      const T B = (T(1) - o6) * (a + b - T(2) * c) + o6 * (ea + eb - T(2) * ec);
      const T C = (T(1) - o7) * (a + b + c) + o7 * (ea + eb + ec);
      k[KI(2, 2, 0)] = (C + A + B) * third;
      k[KI(2, 0, 2)] = (C - A) * third;
      k[KI(0, 2, 2)] = (C - B) * third;
    }
    k[KI(2, 1, 1)] = (T(1) - o8) * k[KI(2, 1, 1)] + o8 * e[KI(2, 1, 1)];
    k[KI(1, 2, 1)] = (T(1) - o8) * k[KI(1, 2, 1)] + o8 * e[KI(1, 2, 1)];
    k[KI(1, 1, 2)] = (T(1) - o8) * k[KI(1, 1, 2)] + o8 * e[KI(1, 1, 2)];
    // fifth order, with forcing
    k[KI(1, 2, 2)] = (T(1) - o9) * k[KI(1, 2, 2)] + o9 * e[KI(1, 2, 2)] + (T(1) - o9 / T(2)) * F[0] * cs4;
    k[KI(2, 1, 2)] = (T(1) - o9) * k[KI(2, 1, 2)] + o9 * e[KI(2, 1, 2)] + (T(1) - o9 / T(2)) * F[1] * cs4;
    k[KI(2, 2, 1)] = (T(1) - o9) * k[KI(2, 2, 1)] + o9 * e[KI(2, 2, 1)] + (T(1) - o9 / T(2)) * F[2] * cs4;
    // sixth order
    k[KI(2, 2, 2)] = (T(1) - o10) * k[KI(2, 2, 2)] + o10 * e[KI(2, 2, 2)];
  }
  backward_cm(k, ux, uy, uz);
}

// ---- initialisation, read-back, reductions ------------------------------------------------

// self-solid flags from the user mask and the bounce-back axes (in place, bytes)
__global__ void k_solid_self(Geom g, uint8_t* solid, int has_user, int bx, int by, int bz);
// neighbour mask from the self-solid flags
__global__ void k_solid_mask(Geom g, const uint8_t* solid, uint32_t* mask);

template <typename T, typename SF, bool SOLID>
__global__ void __launch_bounds__(128) k_init(Geom g, Ptrs<T> P, Phys<T> ph, const double* in, long long lo,
                                              long long hi, int sm) {
  Cell c;
  if (!make_cell(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  if (i0 < lo || i0 >= hi) return;
  // the chunk's inputs: rho_r, rho_b, u_x, u_y, u_z, each hi - lo long
  const long long ci = i0 - lo, m = hi - lo;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
    for (int q = 0; q < 27; ++q) {
      const long long o = emit_index(sm, q, S, c);
      fout<SF>(P.f_out)[o] = Store<SF>::put(T(0));
      P.aux_out[o] = T(0);
    }
    for (int a = 0; a < 6; ++a) {
      P.s_out[a * S + i0] = T(0);
      P.mac[a * S + i0] = T(0);
    }
    for (int a = 0; a < 3; ++a) P.force[a * S + i0] = T(0);
    P.phi[i0] = T(0);
    return;
  }
  const T rr = T(in[ci]), rb = T(in[m + ci]);
  const T u[3] = {T(in[2 * m + ci]), T(in[3 * m + ci]), T(in[4 * m + ci])};
  const T rho = rr + rb;
  const T p = rr * ph.cr2 + rb * ph.cb2;
  T k[27];
  keq_model(ph.model, rho, p, u[0], u[1], u[2], k);
  backward_cm(k, u[0], u[1], u[2]);
  const T r0 = Store<SF>::SHIFT ? rest_zero(rho, p) : T(0);
#pragma unroll
  for (int q = 0; q < 27; ++q)
    fout<SF>(P.f_out)[emit_index(sm, q, S, c)] =
        Store<SF>::put(pop_encode<Store<SF>::SHIFT>(q, k[q], r0, ph.rest1));
  if (SOLID)
    for (int q = 0; q < 27; ++q) P.aux_out[emit_index(sm, q, S, c)] = T(0);
  P.s_out[i0] = rr / rho;
  P.s_out[S + i0] = rb / rho;
  P.s_out[2 * S + i0] = P.s_out[3 * S + i0] = P.s_out[4 * S + i0] = T(0);
  P.s_out[S_DIVR * S + i0] = T(0);
  if (Store<SF>::SHIFT) P.s_out[S_REST * S + i0] = r0;
  P.mac[i0] = rr;
  P.mac[S + i0] = rb;
  for (int a = 0; a < 3; ++a) {
    P.mac[(2 + a) * S + i0] = rho * u[a];
    P.force[a * S + i0] = T(0);
  }
  P.phi[i0] = order_parameter(rr, rb, ph);
}

// Initial content of the wall cells: the wall rule applied to the initial
// populations of their fluid neighbours (buffer read for fluid cells and
// written for solid cells only), with the initial colour densities that
// k_init left in mac.
template <typename T, typename SF>
__global__ void __launch_bounds__(128) k_init_walls(Geom g, Ptrs<T> P, Phys<T> ph, int sm_in, int sm_out) {
  Cell c;
  if (!make_cell(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  const uint32_t mask = ld(P.mask + i0);
  if (!((mask >> SELF_SOLID_BIT) & 1u)) return;
  T uw[3];
  const int flip = wall_rule(g, ph, c, uw);
  for (int q = 0; q < 27; ++q) {
    const int src = nbr(c, -CX(q), -CY(q), -CZ(q));
    T fr = T(0), fb = T(0), ft;
    int out;
    if (!((mask >> OPP(q)) & 1u)) {  // the source is fluid
      pull_colour<T, SF, true>(P, S, q, src, pull_index(sm_in, q, S, c), mask, fr, fb, ft);
      out = wall_emit(q, flip, uw, ld(P.mac + src), ld(P.mac + S + src), fr, fb);
    } else {
      out = flip ? reflect_dir(q, flip) : OPP(q);
    }
    const long long o = emit_index(sm_out, out, S, c);
    fout<SF>(P.f_out)[o] = Store<SF>::put(fr);
    P.aux_out[o] = fb;
  }
}

// macroscopic fields to FP64 for the cells lo <= i < hi:
// [rho_r][rho_b][u 3][p][phi], each hi - lo long
template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k_read_macros(Geom g, Ptrs<T> P, Phys<T> ph, double* out,
                                                     long long lo, long long hi) {
  Cell c;
  if (!make_cell(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  if (i0 < lo || i0 >= hi) return;
  const long long ci = i0 - lo, m = hi - lo;
  const T rr = P.mac[i0], rb = P.mac[S + i0];
  out[ci] = double(rr);
  out[m + ci] = double(rb);
  const bool solid = SOLID && ((ld(P.mask + i0) >> SELF_SOLID_BIT) & 1u);
  if (solid) {
    for (int a = 0; a < 5; ++a) out[(2 + a) * m + ci] = 0.0;
    return;
  }
  const T rho = rr + rb;
  for (int a = 0; a < 3; ++a)
    out[(2 + a) * m + ci] = double((P.mac[(2 + a) * S + i0] + P.force[a * S + i0] / T(2)) / rho);
  out[5 * m + ci] = double(rr * ph.cr2 + rb * ph.cb2);
  out[6 * m + ci] = double(order_parameter(rr, rb, ph));
}

// two-colour post-collision populations of lattice direction q to FP64
template <typename T, typename SF, bool SOLID>
__global__ void __launch_bounds__(128) k_read_pop(Geom g, Ptrs<T> P, Phys<T> ph, int q, double* out_r,
                                                  double* out_b, long long lo, long long hi, int sm) {
  Cell c;
  if (!make_cell(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  if (i0 < lo || i0 >= hi) return;
  const long long ci = i0 - lo;
  // sm: the mode of the step that wrote the state
  const long long o = emit_index(sm, q, S, c);
  T f = Store<SF>::template get<T>(fin<SF>(P.f_in) + o);
  if (Store<SF>::SHIFT) f = pop_decode<true>(q, f, P.s_in[S_REST * S + i0], ph.rest1);
  const bool solid = SOLID && ((ld(P.mask + i0) >> SELF_SOLID_BIT) & 1u);
  if (solid) {
    out_r[ci] = double(f);
    out_b[ci] = double(P.aux_in[o]);
    return;
  }
  const T cR = T(CX(q)) * P.s_in[2 * S + i0] + T(CY(q)) * P.s_in[3 * S + i0] +
               T(CZ(q)) * P.s_in[4 * S + i0];
  const T t = (q == REST) ? T(0) : (WQ<T>(q) / Lat<T>::CS2) * cR;
  out_r[ci] = double(P.s_in[i0] * f + t);
  out_b[ci] = double(P.s_in[S + i0] * f - t);
}

// FP64 block partial sums of rho_r and rho_b in a fixed order
template <typename T>
__global__ void __launch_bounds__(256) k_mass_partial(Geom g, const T* mac, long long n,
                                                      double* partial) {
  __shared__ double sr[256], sb[256];
  const long long per_block = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per_block;
  const long long hi = min(n, lo + per_block);
  double ar = 0.0, ab = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
    ar += double(mac[i]);
    ab += double(mac[g.stride + i]);
  }
  sr[threadIdx.x] = ar;
  sb[threadIdx.x] = ab;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = sr[0];
    partial[2 * blockIdx.x + 1] = sb[0];
  }
}

__global__ void k_mass_final(const double* partial, int nblocks, double* out);

}  // namespace cg27
