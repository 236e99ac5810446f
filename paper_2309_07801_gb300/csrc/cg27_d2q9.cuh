// cg27_d2q9.cuh -- the colour-gradient CM-MRT step on the D2Q9 lattice
// (App. A of arXiv 2309.07801) for the paper's two-dimensional tests.
//
// Same state layout as D3Q27 with 9 populations: F[9] (totals), S (rho_r/rho,
// rho_b/rho, R_x, R_y, 0, 0), MAC (rho_r, rho_b, j_x, j_y, 0), PHI, FORCE, WV,
// QC (z components 0).  Directions are stored lexicographically,
// q = (c_x + 1) + 3 (c_y + 1); moments use r = a + 3 b.  Two-dimensional
// domains are small, so the kernels are plain per-cell kernels (one thread per
// cell, neighbours read from global memory):
//   k2_macro   pull both colours, rho_r, rho_b, j, phi              (Sec. II.A)
//   k2_normal  grad phi (isotropic difference) and n
//   k2_force   kappa, F, u, (p - rho c_s^2) u, R, recoloring fractions
//   k2_qcorr   Q = -3 d_a[(p - rho c_s^2) u_a]                        (Sec. III.E)
//   k2_collide pull the totals, CM-MRT collision toward the generalized
//              equilibrium moments of App. A, store f^*; fullway bounce-back
// The equation of state uses (c_s^k)^2 = xi (1 - alpha_k) with xi = 3/5 (the
// value for which alpha = w_0 = 4/9 gives the lattice c_s^2 = 1/3).
#pragma once

#include "cg27_device.cuh"

namespace cg27 {

__host__ __device__ constexpr int CX2(int q) { return q % 3 - 1; }
__host__ __device__ constexpr int CY2(int q) { return q / 3 - 1; }
__host__ __device__ constexpr int OPP2(int q) { return 8 - q; }
constexpr int REST2 = 4;

template <typename T>
__host__ __device__ constexpr T W2(int q) {
  return (CX2(q) == 0 && CY2(q) == 0) ? T(4) / T(9)
                                      : ((CX2(q) == 0 || CY2(q) == 0) ? T(1) / T(9) : T(1) / T(36));
}

struct Cell2 {
  int idx, x, y;
  int xs[3], ys[3];  // x-1, x, x+1 and (y-1, y, y+1) * nx, periodic wrap
};

__device__ __forceinline__ bool make_cell2(const Geom& g, Cell2& c) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return false;
  c.x = x;
  c.y = y;
  c.xs[0] = x == 0 ? g.nx - 1 : x - 1;
  c.xs[1] = x;
  c.xs[2] = x == g.nx - 1 ? 0 : x + 1;
  c.ys[0] = (y == 0 ? g.ny - 1 : y - 1) * g.nx;
  c.ys[1] = y * g.nx;
  c.ys[2] = (y == g.ny - 1 ? 0 : y + 1) * g.nx;
  c.idx = x + c.ys[1];
  return true;
}

__device__ __forceinline__ int nbr2(const Cell2& c, int dx, int dy) { return c.xs[dx + 1] + c.ys[dy + 1]; }

// equilibrium central moments of App. A: k00 = rho, k20 = k02 = p, k22 = p c_s^2
template <typename T>
__device__ __forceinline__ void keq2(T rho, T p, T (&k)[9]) {
#pragma unroll
  for (int r = 0; r < 9; ++r) k[r] = T(0);
  k[0] = rho;
  k[2] = k[6] = p;
  k[8] = p * Lat<T>::CS2;
}

// 2D transforms: 3 lines per axis of the 3 x 3 velocity grid
template <typename T>
__device__ __forceinline__ void forward_cm2(T (&f)[9], T ux, T uy) {
#pragma unroll
  for (int l = 0; l < 3; ++l) fwd3(f[3 * l], f[3 * l + 1], f[3 * l + 2], ux);
#pragma unroll
  for (int a = 0; a < 3; ++a) fwd3(f[a], f[a + 3], f[a + 6], uy);
}
template <typename T>
__device__ __forceinline__ void backward_cm2(T (&k)[9], T ux, T uy) {
#pragma unroll
  for (int a = 0; a < 3; ++a) bwd3(k[a], k[a + 3], k[a + 6], uy);
#pragma unroll
  for (int l = 0; l < 3; ++l) bwd3(k[3 * l], k[3 * l + 1], k[3 * l + 2], ux);
}

// collision of the nine 2D central moments: first order with omega_0 and F,
// k11 and k20 - k02 with omega_1, k20 + k02 with omega_2 (Q on the diagonal),
// k21, k12 with omega_3 and c_s^2 F, k22 with omega_4
template <typename T>
__device__ __forceinline__ void collide_cm2(T (&f)[9], T rho, T p, T ux, T uy, const T (&F)[2], const T (&Q)[2],
                                            T om1, const Phys<T>& ph) {
  forward_cm2(f, ux, uy);
  T(&k)[9] = f;
  T e[9];
  keq2(rho, p, e);
  const T o0 = ph.om[0], o2 = ph.om[2], o3 = ph.om[3], o4 = ph.om[4];
  const T cs2 = Lat<T>::CS2;
  k[1] = (T(1) - o0) * k[1] + (T(1) - o0 / T(2)) * F[0];
  k[3] = (T(1) - o0) * k[3] + (T(1) - o0 / T(2)) * F[1];
  k[4] = (T(1) - om1) * k[4] + om1 * e[4];
  {
    const T d = k[2] - k[6], de = e[2] - e[6], t = k[2] + k[6], te = e[2] + e[6];
    const T ds = (T(1) - om1) * d + om1 * de + (T(1) - om1 / T(2)) * (Q[0] - Q[1]);
    const T ts = (T(1) - o2) * t + o2 * te + (T(1) - o2 / T(2)) * (Q[0] + Q[1]);
    k[2] = T(0.5) * (ts + ds);
    k[6] = T(0.5) * (ts - ds);
  }
  k[5] = (T(1) - o3) * k[5] + o3 * e[5] + (T(1) - o3 / T(2)) * F[1] * cs2;
  k[7] = (T(1) - o3) * k[7] + o3 * e[7] + (T(1) - o3 / T(2)) * F[0] * cs2;
  k[8] = (T(1) - o4) * k[8] + o4 * e[8];
  backward_cm2(k, ux, uy);
}

// colour parts of the population of direction q that streams into a cell
// from src (fluid: recoloring of Eq. (recoloring); solid: the stored parts)
template <typename T, bool SOLID>
__device__ __forceinline__ void pull_colour2(const Ptrs<T>& P, long long S, int q, int src, uint32_t mask, T& fr,
                                             T& fb) {
  const T f = ld(fin<T>(P.f_in) + q * S + src);
  if (SOLID && ((mask >> OPP2(q)) & 1u)) {
    fr = f;
    fb = ld(P.aux_in + q * S + src);
    return;
  }
  const T t = (W2<T>(q) / Lat<T>::CS2) *
              (T(CX2(q)) * ld(P.s_in + 2 * S + src) + T(CY2(q)) * ld(P.s_in + 3 * S + src));
  fr = ld(P.s_in + src) * f + t;
  fb = ld(P.s_in + S + src) * f - t;
}

// neighbour mask of a 2D cell: bit q set when x + c_q is solid, bit 27 self
__global__ void k2_solid_mask(Geom g, const uint8_t* solid, uint32_t* mask);

template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_init(Geom g, Ptrs<T> P, Phys<T> ph, const double* in, long long lo,
                                               long long hi) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  if (i0 < lo || i0 >= hi) return;
  // the chunk's inputs: rho_r, rho_b, u_x, u_y, u_z, each hi - lo long
  const long long ci = i0 - lo, m = hi - lo;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
    for (int q = 0; q < 9; ++q) {
      fout<T>(P.f_out)[q * S + i0] = T(0);
      P.aux_out[q * S + i0] = T(0);
    }
    for (int a = 0; a < 6; ++a) P.s_out[a * S + i0] = T(0);
    for (int a = 0; a < 5; ++a) P.mac[a * S + i0] = T(0);
    for (int a = 0; a < 3; ++a) P.force[a * S + i0] = T(0);
    P.phi[i0] = T(0);
    return;
  }
  const T rr = T(in[ci]), rb = T(in[m + ci]);
  const T ux = T(in[2 * m + ci]), uy = T(in[3 * m + ci]);
  const T rho = rr + rb, p = rr * ph.cr2 + rb * ph.cb2;
  T k[9];
  keq2(rho, p, k);
  backward_cm2(k, ux, uy);
  for (int q = 0; q < 9; ++q) fout<T>(P.f_out)[q * S + i0] = k[q];
  P.s_out[i0] = rr / rho;
  P.s_out[S + i0] = rb / rho;
  for (int a = 2; a < 6; ++a) P.s_out[a * S + i0] = T(0);
  P.mac[i0] = rr;
  P.mac[S + i0] = rb;
  P.mac[2 * S + i0] = rho * ux;
  P.mac[3 * S + i0] = rho * uy;
  P.mac[4 * S + i0] = T(0);
  for (int a = 0; a < 3; ++a) P.force[a * S + i0] = T(0);
  P.phi[i0] = order_parameter(rr, rb, ph);
}

// walls start with the reversed initial populations of their fluid neighbours
// (read fluid cells, write solid cells of the same buffer)
template <typename T>
__global__ void __launch_bounds__(128) k2_init_walls(Geom g, Ptrs<T> P) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  const uint32_t mask = ld(P.mask + i0);
  if (!((mask >> SELF_SOLID_BIT) & 1u)) return;
  for (int q = 0; q < 9; ++q) {
    const int src = nbr2(c, -CX2(q), -CY2(q));
    T fr = T(0), fb = T(0);
    if (!((mask >> OPP2(q)) & 1u)) pull_colour2<T, true>(P, S, q, src, mask, fr, fb);
    fout<T>(P.f_out)[OPP2(q) * S + i0] = fr;
    P.aux_out[OPP2(q) * S + i0] = fb;
  }
}

template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_macro(Geom g, Ptrs<T> P, Phys<T> ph) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  T rr = T(0), rb = T(0), jx = T(0), jy = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    T fr, fb;
    pull_colour2<T, SOLID>(P, S, q, nbr2(c, -CX2(q), -CY2(q)), mask, fr, fb);
    rr += fr;
    rb += fb;
    if (CX2(q) != 0) jx += T(CX2(q)) * (fr + fb);
    if (CY2(q) != 0) jy += T(CY2(q)) * (fr + fb);
  }
  P.mac[i0] = rr;
  P.mac[S + i0] = rb;
  P.mac[2 * S + i0] = jx;
  P.mac[3 * S + i0] = jy;
  P.mac[4 * S + i0] = T(0);
  const bool self_solid = SOLID && ((mask >> SELF_SOLID_BIT) & 1u);
  P.phi[i0] = self_solid ? T(0) : order_parameter(rr, rb, ph);
  if (!isfinite(rr + rb)) atomicOr(P.flag, 1u);
}

// isotropic difference (1/c_s^2) sum_q w_q c_q chi(x + c_q); a solid neighbour
// contributes the centre value
template <typename T, bool SOLID>
__device__ __forceinline__ void grad2(const T* chi, const Cell2& c, uint32_t mask, T (&gr)[2]) {
  const T ctr = ld(chi + c.idx);
  gr[0] = gr[1] = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (q == REST2) continue;
    T v = ld(chi + nbr2(c, CX2(q), CY2(q)));
    if (SOLID && ((mask >> q) & 1u)) v = ctr;
    if (CX2(q) != 0) gr[0] += T(CX2(q)) * W2<T>(q) * v;
    if (CY2(q) != 0) gr[1] += T(CY2(q)) * W2<T>(q) * v;
  }
  gr[0] *= T(3);
  gr[1] *= T(3);
}

// grad phi -> FORCE[0..1], n -> QC[0..1] (read by k2_force; QC is rewritten by k2_qcorr)
template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_normal(Geom g, Ptrs<T> P) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const uint32_t mask = SOLID ? ld(P.mask + c.idx) : 0u;
  T gr[2] = {T(0), T(0)};
  if (!(SOLID && ((mask >> SELF_SOLID_BIT) & 1u))) grad2<T, SOLID>(P.phi, c, mask, gr);
  const T g2 = gr[0] * gr[0] + gr[1] * gr[1];
  const T inv = g2 > T(1e-24) ? T(1) / sqrt(g2) : T(0);
  for (int a = 0; a < 2; ++a) {
    P.force[a * S + c.idx] = gr[a];
    P.qc[a * S + c.idx] = gr[a] * inv;
  }
}

template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_force(Geom g, Ptrs<T> P, Phys<T> ph) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
    for (int a = 0; a < 3; ++a) {
      P.force[a * S + i0] = T(0);
      P.wv[a * S + i0] = T(0);
    }
    for (int a = 0; a < 6; ++a) P.s_out[a * S + i0] = T(0);
    return;
  }
  T dn[2][2];  // dn[a][b] = d_a n_b
  for (int b = 0; b < 2; ++b) {
    T gb[2];
    grad2<T, SOLID>(P.qc + b * S, c, mask, gb);
    dn[0][b] = gb[0];
    dn[1][b] = gb[1];
  }
  const T nc[2] = {P.qc[i0], P.qc[S + i0]};
  T nnd = T(0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) nnd += nc[a] * nc[b] * dn[a][b];
  const T kappa = -((dn[0][0] + dn[1][1]) - nnd);
  const T rr = P.mac[i0], rb = P.mac[S + i0];
  const T rho = rr + rb, p = rr * ph.cr2 + rb * ph.cb2;
  const T inv_rho = T(1) / rho;
  const T rfac = ph.beta * rr * rb * inv_rho * inv_rho * p;
  const T grad[2] = {P.force[i0], P.force[S + i0]};
  for (int a = 0; a < 2; ++a) {
    T fb = T(0);
    if (ph.force_mode == 1) fb = ph.g[a];
    else if (ph.force_mode == 2) fb = rho * ph.g[a];
    else if (ph.force_mode == 3) fb = (rho - ph.rho_ref) * ph.g[a];
    const T Fa = T(0.5) * ph.sigma * kappa * grad[a] + fb;
    const T ua = (P.mac[(2 + a) * S + i0] + T(0.5) * Fa) * inv_rho;
    P.force[a * S + i0] = Fa;
    P.wv[a * S + i0] = (p - rho * Lat<T>::CS2) * ua;
    P.s_out[(2 + a) * S + i0] = rfac * nc[a];
  }
  P.force[2 * S + i0] = T(0);
  P.wv[2 * S + i0] = T(0);
  P.s_out[i0] = rr * inv_rho;
  P.s_out[S + i0] = rb * inv_rho;
  P.s_out[4 * S + i0] = T(0);
  P.s_out[5 * S + i0] = T(0);
}

template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_qcorr(Geom g, Ptrs<T> P, int use_Q) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const uint32_t mask = SOLID ? ld(P.mask + c.idx) : 0u;
  const bool self_solid = SOLID && ((mask >> SELF_SOLID_BIT) & 1u);
  for (int a = 0; a < 2; ++a) {
    T q = T(0);
    if (use_Q && !self_solid) {
      // no neighbour substitution: (p - rho c_s^2) u is 0 at solid cells
#pragma unroll
      for (int d = 0; d < 9; ++d) {
        const int ca = a == 0 ? CX2(d) : CY2(d);
        if (ca != 0) q += T(ca) * W2<T>(d) * ld(P.wv + a * S + nbr2(c, CX2(d), CY2(d)));
      }
      q = T(-9) * q;
    }
    P.qc[a * S + c.idx] = q;
  }
  P.qc[2 * S + c.idx] = T(0);
}

template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_collide(Geom g, Ptrs<T> P, Phys<T> ph) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
    for (int q = 0; q < 9; ++q) {
      T fr, fb;
      pull_colour2<T, SOLID>(P, S, q, nbr2(c, -CX2(q), -CY2(q)), mask, fr, fb);
      fout<T>(P.f_out)[OPP2(q) * S + i0] = fr;
      P.aux_out[OPP2(q) * S + i0] = fb;
    }
    return;
  }
  T f[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    const int src = nbr2(c, -CX2(q), -CY2(q));
    f[q] = ld(fin<T>(P.f_in) + q * S + src);
    if (SOLID && ((mask >> OPP2(q)) & 1u)) f[q] += ld(P.aux_in + q * S + src);
  }
  const T rr = P.mac[i0], rb = P.mac[S + i0];
  const T rho = rr + rb, p = rr * ph.cr2 + rb * ph.cb2;
  const T phi = order_parameter(rr, rb, ph);
  const T nu = T(0.5) * (T(1) + phi) * ph.nu_r + T(0.5) * (T(1) - phi) * ph.nu_b;
  const T om1 = p / (T(0.5) * p + rho * nu);
  const T F[2] = {P.force[i0], P.force[S + i0]};
  const T Q[2] = {P.qc[i0], P.qc[S + i0]};
  T jx = T(0), jy = T(0);
#pragma unroll
  for (int q = 0; q < 9; ++q) {
    if (CX2(q) != 0) jx += T(CX2(q)) * f[q];
    if (CY2(q) != 0) jy += T(CY2(q)) * f[q];
  }
  const T inv_rho = T(1) / rho;
  collide_cm2<T>(f, rho, p, (jx + T(0.5) * F[0]) * inv_rho, (jy + T(0.5) * F[1]) * inv_rho, F, Q, om1, ph);
#pragma unroll
  for (int q = 0; q < 9; ++q) fout<T>(P.f_out)[q * S + i0] = f[q];
}

// two-colour post-collision populations of direction q (read-back, FP64 out)
template <typename T, bool SOLID>
__global__ void __launch_bounds__(128) k2_read_pop(Geom g, Ptrs<T> P, int q, double* out_r, double* out_b,
                                                   long long lo, long long hi) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  const long long S = g.stride;
  const int i0 = c.idx;
  if (i0 < lo || i0 >= hi) return;
  const long long ci = i0 - lo;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  const T f = ld(fin<T>(P.f_in) + q * S + i0);
  if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
    out_r[ci] = double(f);
    out_b[ci] = double(ld(P.aux_in + q * S + i0));
    return;
  }
  const T t = (W2<T>(q) / Lat<T>::CS2) * (T(CX2(q)) * ld(P.s_in + 2 * S + i0) + T(CY2(q)) * ld(P.s_in + 3 * S + i0));
  out_r[ci] = double(ld(P.s_in + i0) * f + t);
  out_b[ci] = double(ld(P.s_in + S + i0) * f - t);
}

}  // namespace cg27
