// cg27_step.cuh -- the four kernels of one time step.
//
// k_macro and k_fields run one thread per (x, y) column of a TX x TY tile and
// walk a range of z planes.  Neighbour data that a stencil reads from the planes
// z-1, z, z+1 is staged in shared memory as a ring of planes (each plane loaded
// once per tile, with its x-y halo and periodic wrap applied at load time), so a
// neighbour read is one shared-memory load at a constant offset.  Populations
// (pulled once per cell) come straight from global memory, all 27 loads issued
// before they are used.
//
//   k_macro   pull both colours, sums rho_r, rho_b, j and phi        (Sec. II.A)
//   k_fields  grad phi and n on the tile plus a 1-cell halo, then
//             kappa, F, u, (p - rho c_s^2) u, R and the recoloring
//             fractions on the tile                            (Secs. II.A, III.E)
//   k_div_sep correction term Q from (p - rho c_s^2) u (Sec. III.E) and
//             the divergence of R that the next pull's colour sums need
//   k_collide one thread per cell: pull the totals, CM-MRT collision, store
//             f^*                                           (Secs. II.B, III.E)
#pragma once

#include "cg27_device.cuh"

#include <type_traits>

namespace cg27 {

constexpr int TX = 32, TY = 8, NT = TX * TY;

// Tile shapes of the z-marching passes: TX x TY threads, one per (x, y) column
// of the tile.  The single-domain kernels use ShapeA; the batch kernels are
// compiled for both, and the batch tuner chooses (block size 256 or 128, and
// the shared-memory rings sized for the tile plus its halo).
template <int X, int Y>
struct Shape {
  static constexpr int TX = X, TY = Y, NT = X * Y;
};
using ShapeA = Shape<32, 8>;
using ShapeB = Shape<32, 4>;
// tile shapes of the single-domain stencil passes (threads 32 x TY; the ring
// of the tile is recomputed, so taller tiles repeat less of it)
using FieldShape = Shape<32, 8>;
using DivShape = Shape<32, 8>;
// threads of a divergence block: 11 rows of 32 for the 32 x 8 tile, so that
// each thread loads at most one of the 340 positions of the tile plus halo
// (rows 8-10 load halo positions only): 40 registers instead of 64 with two
// positions per thread, four blocks per SM
constexpr int DIV_THREADS = 352, DIV_BLOCKS = 4;
// output rows per computing thread of the divergence pass (the x parts of the
// stencils of a shared-memory row are formed once for both rows)
constexpr int DIV_ROWS = 2;
using MacroShape = Shape<32, 4>;
// blocks per SM that a register cap aims at: `blocks256` blocks of 256 threads
template <class SH>
constexpr int blocks_of(int blocks256) { return blocks256 * 256 / SH::NT > 0 ? blocks256 * 256 / SH::NT : 1; }

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// this thread's column and its wrapped x / y neighbours
struct Col {
  int tx, ty, tid;
  int x0, y0;  // tile origin
  bool active;
  int xs[3];   // x-1, x, x+1 (wrapped)
  int ys[3];   // (y-1, y, y+1) * nx (wrapped)
};

template <class SH = ShapeA>
__device__ __forceinline__ Col make_col(const Geom& g, int bx, int by) {
  constexpr int TX = SH::TX, TY = SH::TY;
  Col c;
  c.tx = threadIdx.x;
  c.ty = threadIdx.y;
  c.tid = c.tx + TX * c.ty;
  c.x0 = bx * TX;
  c.y0 = by * TY;
  const int x = c.x0 + c.tx, y = c.y0 + c.ty;
  c.active = x < g.nx && y < g.ny;
  const int xx = c.active ? x : 0, yy = c.active ? y : 0;
  c.xs[0] = xx == 0 ? g.nx - 1 : xx - 1;
  c.xs[1] = xx;
  c.xs[2] = xx == g.nx - 1 ? 0 : xx + 1;
  c.ys[0] = (yy == 0 ? g.ny - 1 : yy - 1) * g.nx;
  c.ys[1] = yy * g.nx;
  c.ys[2] = (yy == g.ny - 1 ? 0 : yy + 1) * g.nx;
  return c;
}

__device__ __forceinline__ int ring3(int z) { return (z + 3) % 3; }

// Positions of a plane's tile-plus-halo region that this thread loads: at most
// two per thread for the regions used here; `xy` is the wrapped in-plane cell
// offset (x + nx y) of each, -1 when unused.  Computed once per block.
template <int HALO, class SH = ShapeA, int NTB = SH::NT>
struct HaloSlots {
  static constexpr int TX = SH::TX, TY = SH::TY, NT = NTB;  // NTB threads (at least the tile's)
  static constexpr int W = TX + 2 * HALO, PL = W * (TY + 2 * HALO);
  static constexpr int K = (PL + NT - 1) / NT;
  int xy[K];
  __device__ __forceinline__ void init(const Geom& g, const Col& c) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = c.tid + k * NT;
      xy[k] = -1;
      if (i < PL) {
        const int lx = i % W, ly = i / W;
        xy[k] = wrapi(c.x0 + lx - HALO, g.nx) + wrapi(c.y0 + ly - HALO, g.ny) * g.nx;
      }
    }
  }
};

__device__ __forceinline__ int zoff(const Geom& g, int z) { return wrapi(z, g.nz) * g.nxy; }

// ---- pairs of values that take the same arithmetic -----------------------------------
// Two stencils of the same shape (two fields, or two components) are carried
// as pairs, so that a pair staged in shared memory is one 8-byte access.  The
// arithmetic stays scalar: the paired FP32 instructions of sm_100 (FFMA2 and
// the like) measured slower in these passes.
template <typename T>
struct PairOf;
template <>
struct PairOf<float> { using V = float2; };
template <>
struct PairOf<double> { using V = double2; };
template <typename T>
using Pr = typename PairOf<T>::V;

__device__ __forceinline__ float2 pr(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 pr(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
}
__device__ __forceinline__ double2 fma2(double2 a, double2 b, double2 c) {
  return make_double2(fma(a.x, b.x, c.x), fma(a.y, b.y, c.y));
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 add2(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
__device__ __forceinline__ double2 mul2(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
// a - b, rounded once (b times -1 is exact)
template <typename V>
__device__ __forceinline__ V sub2(V a, V b) {
  return fma2(b, pr(decltype(a.x)(-1), decltype(a.x)(-1)), a);
}
template <typename T>
__device__ __forceinline__ Pr<T> splat(T v) { return pr(v, v); }

// ---- the pulled sums of a cell ---------------------------------------------------------
// Order in which the 27 pulled terms of a cell's colour and momentum sums are
// added: the directions with c_z = +1 (source cells in the plane below), then
// c_z = 0, then c_z = -1, each group in storage order.  A pass that builds the
// sums source plane by source plane receives the terms in this order, so every
// kernel that forms them rounds alike.
__host__ __device__ constexpr int sum_dir(int k) { return 9 * (2 - k / 9) + k % 9; }

template <typename T>
__device__ __forceinline__ T fma_rn(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_rn<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <>
__device__ __forceinline__ double fma_rn<double>(double a, double b, double c) { return __fma_rn(a, b, c); }

// sums m = (rho_r, rho_b, j_x, j_y, j_z) += the term of direction q: the total
// f pulled from a fluid source whose colour fractions are (wr, wb)
template <typename T>
__device__ __forceinline__ void add_pulled(int q, T f, T wr, T wb, T (&m)[5]) {
  m[0] = fma_rn(wr, f, m[0]);
  m[1] = fma_rn(wb, f, m[1]);
  if (CX(q) > 0) m[2] += f;
  if (CX(q) < 0) m[2] -= f;
  if (CY(q) > 0) m[3] += f;
  if (CY(q) < 0) m[3] -= f;
  if (CZ(q) > 0) m[4] += f;
  if (CZ(q) < 0) m[4] -= f;
}

// ---- pass 1 -----------------------------------------------------------------------------

// OFF32 (two buffers only, and 8 stride + nx ny < 2^31): each pulled load is
// one row base pointer per z offset (three per plane) plus a 32-bit offset per
// (c_x, c_y) column computed once per thread, instead of a 64-bit address
// formed per direction.
template <typename T, typename SF, bool SOLID, int SM = SM_AB, class SH = ShapeA, bool PAIRS = true,
          bool OFF32 = false>
__device__ __forceinline__ void macro_tile(const Geom& g, const Ptrs<T>& P, const Phys<T>& ph, int z0, int z1,
                                           int bx, int by) {
  static_assert(!OFF32 || SM == SM_AB, "32-bit column offsets are for two population buffers");
  constexpr int NT = SH::NT;
  constexpr int RS = rd_sign<SM>();
  using HS = HaloSlots<1, SH>;
  constexpr int W = HS::W, PL = HS::PL;
  constexpr int NS = 2;  // the colour fractions of the source cells
  constexpr bool SHIFT = Store<SF>::SHIFT;
  using V = Pr<T>;
  // fractions (rho_r/rho, rho_b/rho) of the planes z-1..z+1 plus the one being
  // loaded, 1-cell halo.  PAIRS: stored as pairs (two scalar stores, one
  // 8-byte load per source); else as two arrays (two 4-byte loads), which
  // needs fewer registers at the load.
  constexpr int RING = 4;
  __shared__ __align__(16) T sRaw[RING * NS * PL];
  auto slot = [&](int r, int f, int i) -> T& {
    return PAIRS ? sRaw[(r * PL + i) * NS + f] : sRaw[(r * NS + f) * PL + i];
  };
  const Col c = make_col<SH>(g, bx, by);
  const long long S = g.stride;
  HS hs;
  hs.init(g, c);
  T pre[HS::K][NS];
  auto fetch = [&](int z) {
    const int zo = zoff(g, z);
#pragma unroll
    for (int k = 0; k < HS::K; ++k)
      if (hs.xy[k] >= 0)
#pragma unroll
        for (int f = 0; f < NS; ++f) pre[k][f] = ld(P.s_in + f * S + hs.xy[k] + zo);
  };
  auto store = [&](int z) {
#pragma unroll
    for (int k = 0; k < HS::K; ++k)
      if (hs.xy[k] >= 0) {
        slot(z & (RING - 1), 0, c.tid + k * NT) = pre[k][0];
        slot(z & (RING - 1), 1, c.tid + k * NT) = pre[k][1];
      }
  };
  // OFF32: element offset of direction j = (c_x + 1) + 3 (c_y + 1) of each z
  // group from the group's row base, the source column x - c_q included
  int off[9];
  if constexpr (OFF32)
#pragma unroll
    for (int j = 0; j < 9; ++j) off[j] = j * (int)S + c.xs[1 - (j % 3 - 1)] + c.ys[1 - (j / 3 - 1)];
  fetch(z0 - 1);
  store(z0 - 1 + RING);
  fetch(z0);
  store(z0 + RING);
  fetch(z0 + 1);
  store(z0 + 1 + RING);
  __syncthreads();
  for (int z = z0; z < z1; ++z) {
    fetch(z + 2);  // in flight while this plane is computed
    if (c.active) {
      const int zo[3] = {(z == 0 ? g.nz - 1 : z - 1) * g.nxy, z * g.nxy,
                         (z == g.nz - 1 ? 0 : z + 1) * g.nxy};
      const int i0 = c.xs[1] + c.ys[1] + zo[1];
      T f[27];
      if constexpr (OFF32) {
        // z group k = c_z + 1 pulls from plane z - c_z
        const SF* base[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) base[k] = fin<SF>(P.f_in) + 9LL * k * S + zo[2 - k];
#pragma unroll
        for (int q = 0; q < 27; ++q) f[q] = Store<SF>::template get<T>(base[q / 9] + off[q % 9]);
      } else {
#pragma unroll
        for (int q = 0; q < 27; ++q)
          f[q] = Store<SF>::template get<T>(fin<SF>(P.f_in) + rd_dir<SM>(q) * S +
                                            (c.xs[1 + RS * CX(q)] + c.ys[1 + RS * CY(q)] + zo[1 + RS * CZ(q)]));
      }
      const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
      const T s_rest0 = SHIFT ? ld(P.s_in + S_REST * S + i0) : T(0);
      // sum over q of (w_q / c_s^2) c_q . R(x - c_q), from the divergence pass
      const T divr = ld(P.s_in + S_DIVR * S + i0);
      T m[5] = {divr, -divr, T(0), T(0), T(0)};  // rho_r, rho_b, j
#pragma unroll
      for (int k = 0; k < 27; ++k) {
        const int q = sum_dir(k);
        const int src = c.xs[1 - CX(q)] + c.ys[1 - CY(q)] + zo[1 - CZ(q)];
        const int rq = (z - CZ(q) + RING) & (RING - 1), iq = (c.tx + 1 - CX(q)) + W * (c.ty + 1 - CY(q));
        const V s = PAIRS ? reinterpret_cast<const V*>(sRaw)[rq * PL + iq] : pr(slot(rq, 0, iq), slot(rq, 1, iq));
        if (SHIFT) f[q] = pop_decode<true>(q, f[q], s_rest0, ph.rest1);
        if (SOLID && ((mask >> OPP(q)) & 1u)) {
          // from a wall cell: its red part sits in f, its blue part in aux
          const T fb = ld(P.aux_in + rd_dir<SM>(q) * S + (SM == SM_EVEN ? i0 : src));
          const T ft = f[q] + fb;
          m[0] += f[q];
          m[1] += fb;
          if (CX(q) != 0) m[2] += T(CX(q)) * ft;
          if (CY(q) != 0) m[3] += T(CY(q)) * ft;
          if (CZ(q) != 0) m[4] += T(CZ(q)) * ft;
        } else {
          add_pulled(q, f[q], s.x, s.y, m);
        }
      }
      const T rr = m[0], rb = m[1];
      T* const mac = P.mac + i0;  // fields S apart
#pragma unroll
      for (int a = 0; a < 5; ++a) mac[a * S] = m[a];
      const bool self_solid = SOLID && ((mask >> SELF_SOLID_BIT) & 1u);
      P.phi[i0] = self_solid ? T(0) : order_parameter(rr, rb, ph);
      if (!isfinite(rr + rb)) atomicOr(P.flag, 1u);
    }
    // plane z+2 goes to the slot of z-2, last read in the previous iteration
    store(z + 2 + RING);
    __syncthreads();
  }
}

// ---- pass 2 -----------------------------------------------------------------------------

template <typename T, bool SOLID, class SH = ShapeA>
__device__ __forceinline__ void fields_tile(const Geom& g, const Ptrs<T>& P, const Phys<T>& ph, int z0, int z1,
                                            int bx, int by) {
  constexpr int TX = SH::TX, TY = SH::TY, NT = SH::NT;
  using H2 = HaloSlots<2, SH>;  // phi, 2-cell halo
  using H1 = HaloSlots<1, SH>;  // n, 1-cell halo
  constexpr int W2 = H2::W, P2 = H2::PL, W1 = H1::W, P1 = H1::PL;
  __shared__ T sPhi[3][P2];  // phi of three planes (ring3)
  __shared__ T sN[3][3][P1];  // n of three planes (ring3)
  __shared__ T sG[2][3][NT];  // grad phi of the tile cells, planes of parity 0 and 1
  const Col c = make_col<SH>(g, bx, by);
  const long long S = g.stride;
  H2 h2;
  h2.init(g, c);
  H1 h1;
  h1.init(g, c);
  T pphi[H2::K];
  auto fetch_phi = [&](int z) {
    const int zo = zoff(g, z);
#pragma unroll
    for (int k = 0; k < H2::K; ++k)
      if (h2.xy[k] >= 0) pphi[k] = ld(P.phi + h2.xy[k] + zo);
  };
  auto store_phi = [&](int z) {
#pragma unroll
    for (int k = 0; k < H2::K; ++k)
      if (h2.xy[k] >= 0) sPhi[ring3(z)][c.tid + k * NT] = pphi[k];
  };

  // grad phi and n of plane p on the tile plus a 1-cell halo (phi of p-1..p+1 staged)
  auto normals = [&](int p) {
    const int zo = zoff(g, p);
#pragma unroll
    for (int k = 0; k < H1::K; ++k) {
      if (h1.xy[k] < 0) continue;
      const int i = c.tid + k * NT;
      const int lx = i % W1, ly = i / W1;
      T gr[3] = {T(0), T(0), T(0)};
      uint32_t mask = 0u;
      bool self_solid = false;
      if (SOLID) {
        mask = ld(P.mask + h1.xy[k] + zo);
        self_solid = (mask >> SELF_SOLID_BIT) & 1u;
      }
      if (!self_solid) {
        const int ctr = (lx + 1) + W2 * (ly + 1);
        const T pc = sPhi[ring3(p)][ctr];
#pragma unroll
        for (int q = 0; q < 27; ++q) {
          if (q == REST) continue;
          T v = sPhi[ring3(p + CZ(q))][ctr + CX(q) + W2 * CY(q)];
          if (SOLID && ((mask >> q) & 1u)) v = pc;
          const T wv = WQ<T>(q) * v;
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (CA(q, a) != 0) gr[a] += T(CA(q, a)) * wv;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) gr[a] *= T(3);  // 1 / c_s^2
      }
      const T g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
      const bool ok = g2 > T(1e-24);
      const T inv_len = ok ? T(1) / sqrt(g2) : T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) sN[ring3(p)][a][i] = gr[a] * inv_len;
      const int ix = lx - 1, iy = ly - 1;
      if (ix >= 0 && ix < TX && iy >= 0 && iy < TY)
#pragma unroll
        for (int a = 0; a < 3; ++a) sG[p & 1][a][ix + TX * iy] = gr[a];
    }
  };

  // prologue: phi of z0-2 .. z0+2 and n of z0-1, z0 (three-slot rings)
  for (int p = z0 - 2; p <= z0; ++p) {
    fetch_phi(p);
    store_phi(p);
  }
  __syncthreads();
  normals(z0 - 1);
  fetch_phi(z0 + 1);
  __syncthreads();
  store_phi(z0 + 1);  // replaces z0-2
  __syncthreads();
  normals(z0);
  fetch_phi(z0 + 2);
  __syncthreads();
  store_phi(z0 + 2);  // replaces z0-1
  __syncthreads();

  T mac[5];
  auto fetch_mac = [&](int z) {
    if (!c.active) return;
    const int i0 = c.xs[1] + c.ys[1] + zoff(g, z);
#pragma unroll
    for (int f = 0; f < 5; ++f) mac[f] = ld(P.mac + f * S + i0);
  };
  fetch_mac(z0);
  for (int z = z0; z < z1; ++z) {
    fetch_phi(z + 3);  // in flight during this plane
    normals(z + 1);
    __syncthreads();
    if (c.active) {
      const int i0 = c.xs[1] + c.ys[1] + z * g.nxy;
      const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
      if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          P.force[a * S + i0] = T(0);
          P.wv[a * S + i0] = T(0);
        }
#pragma unroll
        for (int a = 0; a < 5; ++a) P.s_out[a * S + i0] = T(0);
      } else {
        const int ctr = (c.tx + 1) + W1 * (c.ty + 1);
        const T nc[3] = {sN[ring3(z)][0][ctr], sN[ring3(z)][1][ctr], sN[ring3(z)][2][ctr]};
        T dn[3][3];  // dn[a][b] = sum_i w_i n_b(x + c_i) c_ia
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) dn[a][b] = T(0);
#pragma unroll
        for (int q = 0; q < 27; ++q) {
          if (q == REST) continue;
          const bool use_c = SOLID && ((mask >> q) & 1u);
          const int off = ctr + CX(q) + W1 * CY(q);
          T nv[3];
#pragma unroll
          for (int b = 0; b < 3; ++b) nv[b] = use_c ? nc[b] : sN[ring3(z + CZ(q))][b][off];
#pragma unroll
          for (int a = 0; a < 3; ++a)
            if (CA(q, a) != 0)
#pragma unroll
              for (int b = 0; b < 3; ++b) dn[a][b] += T(CA(q, a)) * (WQ<T>(q) * nv[b]);
        }
        T div = T(0), nnd = T(0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          div += dn[a][a];
#pragma unroll
          for (int b = 0; b < 3; ++b) nnd += nc[a] * nc[b] * dn[a][b];
        }
        const T kappa = -T(3) * (div - nnd);  // derivatives carry 1 / c_s^2
        const T rr = mac[0], rb = mac[1];
        const T rho = rr + rb;
        const T p = rr * ph.cr2 + rb * ph.cb2;
        T fbody[3] = {T(0), T(0), T(0)};
        if (ph.force_mode == 1) {
          for (int a = 0; a < 3; ++a) fbody[a] = ph.g[a];
        } else if (ph.force_mode == 2) {
          for (int a = 0; a < 3; ++a) fbody[a] = rho * ph.g[a];
        } else if (ph.force_mode == 3) {
          for (int a = 0; a < 3; ++a) fbody[a] = (rho - ph.rho_ref) * ph.g[a];
        }
        const T inv_rho = T(1) / rho;
        const T rfac = ph.beta * rr * rb * inv_rho * inv_rho * p;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const T Fa = T(0.5) * ph.sigma * kappa * sG[z & 1][a][c.tid] + fbody[a];
          const T ua = (mac[2 + a] + T(0.5) * Fa) * inv_rho;
          P.force[a * S + i0] = Fa;
          P.wv[a * S + i0] = (p - rho * Lat<T>::CS2) * ua;
          P.s_out[(2 + a) * S + i0] = rfac * nc[a];
        }
        P.s_out[i0] = rr * inv_rho;
        P.s_out[S + i0] = rb * inv_rho;
        if (ph.shift) P.s_out[S_REST * S + i0] = rest_zero(rho, p);
      }
    }
    fetch_mac(z + 1);
    // phi of z+3 replaces z, last read by normals(z+1) before the barrier above
    store_phi(z + 3);
    __syncthreads();
  }
}

// ---- pass 2, separable form (periodic domains) --------------------------------------------
// The isotropic difference of Sec. II.A factorises over the axes:
//   d_x chi = D_x S_y S_z chi,  d_y chi = S_x D_y S_z chi,  d_z chi = S_x S_y D_z chi,
// with the 1D smoothing S = (1/6, 2/3, 1/6) and difference D = (-1/2, 0, 1/2)
// (the 1/c_s^2 factor included).
//
// Positions of a tile plane with a halo of H cells are split so that slot 0 of
// every thread is its own tile cell and the other slots cover the halo ring.
// A thread keeps what it needs of its own positions in registers across
// planes: phi of three planes (for S_z phi, D_z phi), n of three planes (for
// S_z n, D_z n), and at its tile cell grad phi and n.  Shared memory holds only
// what neighbours read: the pairs (S_z phi, D_z phi) of the plane whose normals
// come next, and (S_z n_b, D_z n_b) of the output plane, each read as whole
// 8- or 16-byte records.
template <int H, class SH = ShapeA>
struct RingSlots {
  static constexpr int TX = SH::TX, TY = SH::TY, NT = SH::NT;
  static constexpr int W = TX + 2 * H, PL = W * (TY + 2 * H), NR = PL - NT;
  static constexpr int K = 1 + (NR + NT - 1) / NT;
  int at[K];   // position in the W-wide plane array, -1 when unused
  int xy[K];   // wrapped in-plane cell offset x + nx y
  __device__ __forceinline__ void init(const Geom& g, const Col& c) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      int lx = -1, ly = -1;
      if (k == 0) {
        lx = c.tx + H;
        ly = c.ty + H;
      } else {
        const int r = c.tid + (k - 1) * NT;  // index on the ring
        if (r < H * W) {
          lx = r % W;
          ly = r / W;
        } else if (r < 2 * H * W) {
          lx = (r - H * W) % W;
          ly = TY + H + (r - H * W) / W;
        } else if (r < NR) {
          const int q = r - 2 * H * W, row = q / (2 * H), col = q % (2 * H);
          lx = col < H ? col : TX + col;
          ly = H + row;
        }
      }
      at[k] = lx < 0 ? -1 : lx + W * ly;
      xy[k] = lx < 0 ? -1 : wrapi(c.x0 + lx - H, g.nx) + wrapi(c.y0 + ly - H, g.ny) * g.nx;
    }
  }
};

template <typename T>
__device__ __forceinline__ T fast_rsqrt(T v) { return T(1) / sqrt(v); }
template <>
__device__ __forceinline__ float fast_rsqrt<float>(float v) { return rsqrtf(v); }
template <typename T>
__device__ __forceinline__ T fast_rcp(T v) { return T(1) / v; }
template <>
__device__ __forceinline__ float fast_rcp<float>(float v) { return __fdividef(1.0f, v); }

template <typename T, class SH = ShapeA>
__device__ __forceinline__ void fields_sep_tile(const Geom& g, const Ptrs<T>& P, const Phys<T>& ph, int z0,
                                                int z1, int bx, int by) {
  using R2 = RingSlots<2, SH>;  // phi positions
  using R1 = RingSlots<1, SH>;  // n positions
  using V = Pr<T>;
  constexpr int W2 = R2::W, P2 = R2::PL, K2 = R2::K, W1 = R1::W, P1 = R1::PL, K1 = R1::K;
  const T S0 = T(2) / T(3), S1 = T(1) / T(6);
  __shared__ V sAB[P2];              // (S_z phi, D_z phi) of the plane whose normals come next
  __shared__ float4 sN4[P1];         // (S_z n_0, D_z n_0, S_z n_1, D_z n_1) of the output plane
  __shared__ V sN2[P1];              // (S_z n_2, D_z n_2)
  // n of three planes at the ring positions (slots k >= 1), each read only by
  // the thread that wrote it: kept in shared memory to spare registers
  __shared__ T sNr[3][K1 - 1][3][SH::NT];
  static_assert(sizeof(T) == 4, "the separable field pass is the FP32 form");
  const Col c = make_col<SH>(g, bx, by);
  const long long S = g.stride;
  R2 r2;
  r2.init(g, c);
  R1 r1;
  r1.init(g, c);
  // registers: phi of three planes at the phi positions, n of three planes at
  // the n positions, grad phi at the tile cell; each a ring of three indexed
  // by (plane - z0) mod 3, a compile-time constant in every unrolled plane
  T ph3[3][K2];
  T n3[3][1][3];  // n of three planes at the tile cell (slot 0)
  T gl3[3];  // |grad phi| at the tile cell (grad phi = |grad phi| n there)
  auto load_phi = [&](int z, auto slot) {
    constexpr int R = decltype(slot)::value;
    const int zo = zoff(g, z);
#pragma unroll
    for (int k = 0; k < K2; ++k)
      if (r2.xy[k] >= 0) ph3[R][k] = ld(P.phi + r2.xy[k] + zo);
  };
  // (S_z phi, D_z phi) of a plane at the phi positions from phi of the planes
  // below, at and above it
  auto stage_ab = [&](auto lo_, auto mid_, auto hi_) {
    constexpr int L = decltype(lo_)::value, M = decltype(mid_)::value, U = decltype(hi_)::value;
#pragma unroll
    for (int k = 0; k < K2; ++k)
      if (r2.at[k] >= 0) {
        const T lo = ph3[L][k], mid = ph3[M][k], hi = ph3[U][k];
        sAB[r2.at[k]] = pr(S1 * (lo + hi) + S0 * mid, T(0.5) * (hi - lo));
      }
  };
  // grad phi and n of the staged plane at the n positions: per row, S_x and
  // D_x of (S_z phi, D_z phi); then across the rows
  auto normals = [&](auto slot) {
    constexpr int R = decltype(slot)::value;
#pragma unroll
    for (int k = 0; k < K1; ++k) {
      if (r1.at[k] < 0) continue;
      const int lx = r1.at[k] % W1, ly = r1.at[k] / W1;
      const int ctr = (lx + 1) + W2 * (ly + 1);
      // rows y-1, y, y+1 in turn: S_y and D_y weights (1/6, 2/3, 1/6) and (-1/2, 0, 1/2)
      T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const V a = sAB[ctr + (r - 1) * W2 - 1], b = sAB[ctr + (r - 1) * W2], d = sAB[ctr + (r - 1) * W2 + 1];
        const V sx = fma2(splat(S1), add2(a, d), mul2(splat(S0), b));
        const V dx = mul2(splat(T(0.5)), sub2(d, a));
        const T ws = r == 1 ? S0 : S1, wd = T(r - 1) * T(0.5);
        gx += ws * dx.x;
        if (r != 1) gy += wd * sx.x;
        gz += ws * sx.y;
      }
      const T g2 = gx * gx + gy * gy + gz * gz;
      const T inv_len = g2 > T(1e-24) ? fast_rsqrt(g2) : T(0);
      if (k == 0) {
        n3[R][0][0] = gx * inv_len;
        n3[R][0][1] = gy * inv_len;
        n3[R][0][2] = gz * inv_len;
      } else {
        sNr[R][k - 1][0][c.tid] = gx * inv_len;
        sNr[R][k - 1][1][c.tid] = gy * inv_len;
        sNr[R][k - 1][2][c.tid] = gz * inv_len;
      }
      if (k == 0) gl3[R] = g2 * inv_len;
    }
  };
  // (S_z n_b, D_z n_b) of the output plane at the n positions
  auto stage_n = [&](auto lo_, auto mid_, auto hi_) {
    constexpr int L = decltype(lo_)::value, M = decltype(mid_)::value, U = decltype(hi_)::value;
#pragma unroll
    for (int k = 0; k < K1; ++k)
      if (r1.at[k] >= 0) {
        T a[3], d[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const T lo = k == 0 ? n3[L][0][b] : sNr[L][k - 1][b][c.tid];
          const T mid = k == 0 ? n3[M][0][b] : sNr[M][k - 1][b][c.tid];
          const T hi = k == 0 ? n3[U][0][b] : sNr[U][k - 1][b][c.tid];
          a[b] = S1 * (lo + hi) + S0 * mid;
          d[b] = T(0.5) * (hi - lo);
        }
        sN4[r1.at[k]] = make_float4(a[0], d[0], a[1], d[1]);
        sN2[r1.at[k]] = pr(a[2], d[2]);
      }
  };
  using I0 = std::integral_constant<int, 0>;
  using I1 = std::integral_constant<int, 1>;
  using I2 = std::integral_constant<int, 2>;

  // prologue (slot of plane p: (p - z0 + 3) mod 3): phi of z0-2 .. z0+2,
  // n and grad phi of z0-1 and z0
  load_phi(z0 - 2, I1{});
  load_phi(z0 - 1, I2{});
  load_phi(z0, I0{});
  stage_ab(I1{}, I2{}, I0{});  // plane z0-1
  __syncthreads();
  normals(I2{});               // n of z0-1
  load_phi(z0 + 1, I1{});      // replaces z0-2
  __syncthreads();
  stage_ab(I2{}, I0{}, I1{});  // plane z0
  __syncthreads();
  normals(I0{});               // n of z0
  load_phi(z0 + 2, I2{});      // replaces z0-1

  T mac[5];
  auto fetch_mac = [&](int z) {
    if (!c.active) return;
    const T* m = P.mac + (c.xs[1] + c.ys[1] + zoff(g, z));
#pragma unroll
    for (int f = 0; f < 5; ++f) mac[f] = ld(m + f * S);
  };
  const int cc = (c.tx + 1) + W1 * (c.ty + 1);  // this thread's tile cell among the n positions
  // one output plane z with slots A = slot of z - 1, B = slot of z, C = slot of z + 1
  auto plane = [&](int z, auto A_, auto B_, auto C_) {
    constexpr int A = decltype(A_)::value, B = decltype(B_)::value, C = decltype(C_)::value;
    using IA = std::integral_constant<int, A>;
    using IB = std::integral_constant<int, B>;
    using IC = std::integral_constant<int, C>;
    __syncthreads();               // the previous plane's reads of sN4 / sN2 are done
    stage_ab(IB{}, IC{}, IA{});    // plane z+1 from phi of z, z+1, z+2 (z+2 sits in slot A)
    load_phi(z + 3, IB{});         // phi of z is no longer needed; in flight during this plane
    __syncthreads();
    normals(IC{});                 // n of z+1
    stage_n(IA{}, IB{}, IC{});     // S_z n, D_z n of z from n of z-1, z, z+1
    fetch_mac(z);                  // in flight during the barrier and the derivatives of n
    __syncthreads();
    if (c.active) {
      const int i0 = c.xs[1] + c.ys[1] + z * g.nxy;
      const T nc[3] = {n3[B][0][0], n3[B][0][1], n3[B][0][2]};
      // dn[a][b] = d_a n_b: per row, S_x and D_x of (S_z n_b, D_z n_b)
      // accumulated row by row, so that only the nine sums stay live
      T dn[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) dn[a][b] = T(0);
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int o = cc + (r - 1) * W1;
        const float4 a4 = sN4[o - 1], b4 = sN4[o], d4 = sN4[o + 1];
        const V a2 = sN2[o - 1], b2 = sN2[o], d2 = sN2[o + 1];
        const V av[3] = {pr(a4.x, a4.y), pr(a4.z, a4.w), a2};
        const V bv[3] = {pr(b4.x, b4.y), pr(b4.z, b4.w), b2};
        const V dv[3] = {pr(d4.x, d4.y), pr(d4.z, d4.w), d2};
        const T ws = r == 1 ? S0 : S1, wd = T(r - 1) * T(0.5);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          const V sx = fma2(splat(S1), add2(av[b], dv[b]), mul2(splat(S0), bv[b]));
          const V dx = mul2(splat(T(0.5)), sub2(dv[b], av[b]));
          dn[0][b] += ws * dx.x;
          if (r != 1) dn[1][b] += wd * sx.x;
          dn[2][b] += ws * sx.y;
        }
      }
      T div = T(0), nnd = T(0);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        div += dn[a][a];
#pragma unroll
        for (int b = 0; b < 3; ++b) nnd += nc[a] * nc[b] * dn[a][b];
      }
      const T kappa = -(div - nnd);
      const T rr = mac[0], rb = mac[1];
      const T rho = rr + rb;
      const T p = rr * ph.cr2 + rb * ph.cb2;
      T fbody[3] = {T(0), T(0), T(0)};
      if (ph.force_mode == 1) {
        for (int a = 0; a < 3; ++a) fbody[a] = ph.g[a];
      } else if (ph.force_mode == 2) {
        for (int a = 0; a < 3; ++a) fbody[a] = rho * ph.g[a];
      } else if (ph.force_mode == 3) {
        for (int a = 0; a < 3; ++a) fbody[a] = (rho - ph.rho_ref) * ph.g[a];
      }
      const T inv_rho = fast_rcp(rho);
      const T rfac = ph.beta * rr * rb * inv_rho * inv_rho * p;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const T Fa = T(0.5) * ph.sigma * kappa * (gl3[B] * nc[a]) + fbody[a];
        const T ua = (mac[2 + a] + T(0.5) * Fa) * inv_rho;
        P.force[a * S + i0] = Fa;
        P.wv[a * S + i0] = (p - rho * Lat<T>::CS2) * ua;
        P.s_out[(2 + a) * S + i0] = rfac * nc[a];
      }
      P.s_out[i0] = rr * inv_rho;
      P.s_out[S + i0] = rb * inv_rho;
      if (ph.shift) P.s_out[S_REST * S + i0] = rest_zero(rho, p);
    }
  };
  // slots (z-1, z, z+1) for z - z0 = 0, 1, 2 mod 3: (2, 0, 1), (0, 1, 2), (1, 2, 0)
  for (int z = z0; z < z1; z += 3) {
    plane(z, I2{}, I0{}, I1{});
    if (z + 1 < z1) plane(z + 1, I0{}, I1{}, I2{});
    if (z + 2 < z1) plane(z + 2, I1{}, I2{}, I0{});
  }
}

// ---- pass 3: divergences, separable form ----------------------------------------------
// With the isotropic difference d_a = D_a S_b S_c (S = (1/6, 2/3, 1/6),
// D = (-1/2, 0, 1/2), the 1/c_s^2 included):
//   Q_a = -3 d_a[(p - rho c_s^2) u_a]                     (Sec. III.E), and
//   sum_q (w_q / c_s^2) c_q . R(x - c_q) = -sum_a d_a R_a, the part of the next
//   pull's colour sums that comes from the recoloring term of Eq. (recoloring).
// Each thread keeps both vector fields of planes z-1, z, z+1 at its own halo
// positions in registers and stages only their z parts (S_z for the in-plane
// components, D_z for the z component) of the output plane in shared memory
// (two buffers, one barrier per plane).
template <typename T, class SH = ShapeA, int NTB = SH::NT>
__device__ __forceinline__ void div_sep_tile(const Geom& g, const Ptrs<T>& P, int z0, int z1, int use_Q, int bx,
                                             int by) {
  constexpr int NT = NTB;
  using HS = HaloSlots<1, SH, NTB>;
  constexpr int W = HS::W, PL = HS::PL, K = HS::K;
  constexpr T S0 = T(2) / T(3), S1 = T(1) / T(6);
  __shared__ T sA[2][6][PL];
  const Col c = make_col<SH>(g, bx, by);
  const long long S = g.stride;
  HS hs;
  hs.init(g, c);
  // components 0-2: (p - rho c_s^2) u, 3-5: R; base pointers of the six
  // fields, so that each load adds one 32-bit cell index
  const T* src[6] = {P.wv, P.wv + S, P.wv + 2 * S, P.s_out + 2 * S, P.s_out + 3 * S, P.s_out + 4 * S};
  T lo[K][6], mid[K][6], hi[K][6], nx[K][6];
  auto fetch = [&](int z, T (&dst)[K][6]) {
    const int zo = zoff(g, z);
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (hs.xy[k] >= 0) {
        const int i = hs.xy[k] + zo;
#pragma unroll
        for (int f = 0; f < 3; ++f) dst[k][f] = use_Q ? ld(src[f] + i) : T(0);
#pragma unroll
        for (int f = 3; f < 6; ++f) dst[k][f] = src[f][i];
      }
  };
  T* const qc[3] = {P.qc, P.qc + S, P.qc + 2 * S};
  T* const divr = P.s_out + S_DIVR * S;
  fetch(z0 - 1, lo);
  fetch(z0, mid);
  fetch(z0 + 1, hi);
  for (int z = z0; z < z1; ++z) {
    if (z + 1 < z1) fetch(z + 2, nx);
    T(*A)[PL] = sA[z & 1];
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (hs.xy[k] >= 0) {
        const int i = c.tid + k * NT;
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          A[3 * v][i] = S1 * (lo[k][3 * v] + hi[k][3 * v]) + S0 * mid[k][3 * v];
          A[3 * v + 1][i] = S1 * (lo[k][3 * v + 1] + hi[k][3 * v + 1]) + S0 * mid[k][3 * v + 1];
          A[3 * v + 2][i] = T(0.5) * (hi[k][3 * v + 2] - lo[k][3 * v + 2]);
        }
      }
    __syncthreads();
    // ROWS output rows per computing thread: per vector and shared-memory row
    // the x parts of the three stencils (D_x, and S_x twice) once, then per
    // output row the y parts; the two vectors one after the other
    constexpr int ROWS = (SH::TY % DIV_ROWS == 0) ? DIV_ROWS : 1;
    if (c.ty < SH::TY / ROWS) {
      const int cx = c.tx + 1, x = c.x0 + c.tx;
#pragma unroll
      for (int v = 0; v < 2; ++v) {  // (p - rho c_s^2) u -> Q; R -> DIVR
        if (v == 0 && !use_Q) continue;
        T dAx[ROWS + 2], sAy[ROWS + 2], sB[ROWS + 2];
        const T* Ax = A[3 * v];
        const T* Ay = A[3 * v + 1];
        const T* B = A[3 * v + 2];
#pragma unroll
        for (int r = 0; r < ROWS + 2; ++r) {
          const int o = (ROWS * c.ty + r) * W + cx;
          dAx[r] = Ax[o + 1] - Ax[o - 1];
          sAy[r] = S1 * Ay[o - 1] + S0 * Ay[o] + S1 * Ay[o + 1];
          sB[r] = S1 * B[o - 1] + S0 * B[o] + S1 * B[o + 1];
        }
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
          const int y = c.y0 + ROWS * c.ty + i;
          if (x >= g.nx || y >= g.ny) continue;
          const T d0 = T(0.5) * (S1 * dAx[i] + S0 * dAx[i + 1] + S1 * dAx[i + 2]);
          const T d1 = T(0.5) * (sAy[i + 2] - sAy[i]);
          const T d2 = S1 * sB[i] + S0 * sB[i + 1] + S1 * sB[i + 2];
          const int i0 = x + y * g.nx + z * g.nxy;
          if (v == 0) {
            qc[0][i0] = T(-3) * d0;
            qc[1][i0] = T(-3) * d1;
            qc[2][i0] = T(-3) * d2;
          } else {
            divr[i0] = -(d0 + d1 + d2);
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int f = 0; f < 6; ++f) {
        lo[k][f] = mid[k][f];
        mid[k][f] = hi[k][f];
        hi[k][f] = nx[k][f];
      }
  }
}

// Element index of population q of cell i.  The 16-bit modes keep 27 * stride
// below 2^32 (checked when the domain is created), so their index arithmetic
// is 32-bit; it saves a tenth of the issue slots of their collision, which is
// issue-bound.  FP32/FP64 keep 64-bit indices (no measurable difference there).
template <bool IDX32>
__device__ __forceinline__ long long pop_index(int q, long long S, int i) {
  if (IDX32) return (long long)((unsigned)q * (unsigned)S + (unsigned)i);
  return q * S + i;
}

// ---- pass 4: streaming of the totals and the collision ----------------------------------
// One thread per cell: 27 pulled populations, rho_r, rho_b, F and Q in
// registers, the collision, 27 coalesced stores.  The register budget is capped
// (six 128-thread blocks per SM) so that enough warps keep loads in flight; at
// this occupancy the kernel streams at about the copy bandwidth of the device.

// The collision of a fluid cell: f holds the 27 pulled totals and becomes
// f^*; rr, rb are the colour densities of the cell, F the force and Q the
// correction term of the step.  nu(phi) and tau = 1/2 + rho nu / p
// (Sec. II.A, the relation of mu and tau), u with half the force (Sec. II.B),
// then the CM-MRT relaxation of Sec. III.E.
template <typename T, bool UNIT>
__device__ __forceinline__ void collide_pulled(T (&f)[27], T rr, T rb, const T (&F)[3], const T (&Q)[3],
                                               const Phys<T>& ph) {
  const T rho = rr + rb;
  const T p = rr * ph.cr2 + rb * ph.cb2;
  const T phi = order_parameter(rr, rb, ph);
  const T nu = T(0.5) * (T(1) + phi) * ph.nu_r + T(0.5) * (T(1) - phi) * ph.nu_b;
  // omega_1 = 1/tau with tau = 1/2 + rho nu / p (Eq. mu = (tau - 1/2) p)
  const T om1 = p / (T(0.5) * p + rho * nu);
  T j[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int q = 0; q < 27; ++q)
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (CA(q, a) != 0) j[a] += T(CA(q, a)) * f[q];
  const T inv_rho = T(1) / rho;
  T u[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) u[a] = (j[a] + T(0.5) * F[a]) * inv_rho;
  collide_cm<T, UNIT>(f, rho, p, u[0], u[1], u[2], F, Q, om1, ph);
}

template <typename T, typename SF, bool SOLID, bool UNIT, int SM = SM_AB>
__device__ __forceinline__ void collide_cell(const Geom& g, const Ptrs<T>& P, const Phys<T>& ph, const Cell& c) {
  constexpr int RS = rd_sign<SM>();
  constexpr bool SHIFT = Store<SF>::SHIFT;
  const long long S = g.stride;
  const int i0 = c.idx;
  const uint32_t mask = SOLID ? ld(P.mask + i0) : 0u;
  if (SOLID && ((mask >> SELF_SOLID_BIT) & 1u)) {
    // fullway walls: keep what streamed in, colour by colour, and send it back
    // by the cell's wall rule (bounce-back, specular, or moving)
    T uw[3];
    const int flip = wall_rule(g, ph, c, uw);
    if constexpr (SM == SM_AB) {
      for (int q = 0; q < 27; ++q) {
        const int src = nbr(c, -CX(q), -CY(q), -CZ(q));
        T fr, fb, ft;
        pull_colour<T, SF, SOLID>(P, S, q, src, pull_index(SM, q, S, c), mask, fr, fb, ft);
        const bool fluid_src = !((mask >> OPP(q)) & 1u);
        const int out = wall_emit(q, flip, uw, fluid_src ? ld(P.mac + src) : T(0),
                                  fluid_src ? ld(P.mac + S + src) : T(0), fr, fb);
        const long long o = emit_index(SM, out, S, c);
        fout<SF>(P.f_out)[o] = Store<SF>::put(fr);
        P.aux_out[o] = fb;
      }
    } else {
      // in place, the slots this cell writes are the ones it reads: read all
      // 27 first (a slip wall sends direction q into another direction's slot)
      T fr[27], fb[27];
      int out[27];
      for (int q = 0; q < 27; ++q) {
        const int src = nbr(c, -CX(q), -CY(q), -CZ(q));
        T ft;
        pull_colour<T, SF, SOLID>(P, S, q, src, pull_index(SM, q, S, c), mask, fr[q], fb[q], ft);
        const bool fluid_src = !((mask >> OPP(q)) & 1u);
        out[q] = wall_emit(q, flip, uw, fluid_src ? ld(P.mac + src) : T(0),
                           fluid_src ? ld(P.mac + S + src) : T(0), fr[q], fb[q]);
      }
      for (int q = 0; q < 27; ++q) {
        const long long o = emit_index(SM, out[q], S, c);
        fout<SF>(P.f_out)[o] = Store<SF>::put(fr[q]);
        P.aux_out[o] = fb[q];
      }
    }
    return;
  }
  T f[27];
#pragma unroll
  for (int q = 0; q < 27; ++q)
    f[q] = Store<SF>::template get<T>(fin<SF>(P.f_in) +
                                      pop_index<SHIFT>(rd_dir<SM>(q), S, nbr(c, RS * CX(q), RS * CY(q), RS * CZ(q))));
  if (SHIFT) {
    const T r0 = ld(P.s_in + S_REST * S + i0);
#pragma unroll
    for (int q = 0; q < 27; ++q) f[q] = pop_decode<true>(q, f[q], r0, ph.rest1);
  }

  if (SOLID) {
#pragma unroll
    for (int q = 0; q < 27; ++q)
      if ((mask >> OPP(q)) & 1u) f[q] += ld(P.aux_in + rd_dir<SM>(q) * S + nbr(c, RS * CX(q), RS * CY(q), RS * CZ(q)));
  }
  const T rr = ld(P.mac + i0), rb = ld(P.mac + S + i0);
  const T F[3] = {ld(P.force + i0), ld(P.force + S + i0), ld(P.force + 2 * S + i0)};
  T Q[3] = {T(0), T(0), T(0)};
  if (ph.use_Q) {
    Q[0] = ld(P.qc + i0);
    Q[1] = ld(P.qc + S + i0);
    Q[2] = ld(P.qc + 2 * S + i0);
  }
  collide_pulled<T, UNIT>(f, rr, rb, F, Q, ph);
  // the rest-direction shift is the value the field pass stored for this cell
  const T r0n = SHIFT ? P.s_out[S_REST * S + i0] : T(0);
  // In place, the slot written for direction q is the slot read for opp q:
  // opaque copies of the stride and the cell offsets make the compiler form
  // the store addresses afresh instead of keeping 27 load addresses live
  // across the collision (which spills at this register budget).
  long long Sw = S;
  Cell cw = c;
  if constexpr (SM != SM_AB) {
    asm volatile("" : "+l"(Sw));
    asm volatile("" : "+r"(cw.idx));
#pragma unroll
    for (int k = 0; k < 3; ++k) asm volatile("" : "+r"(cw.xs[k]), "+r"(cw.ys[k]), "+r"(cw.zs[k]));
  }
#pragma unroll
  for (int q = 0; q < 27; ++q)
    fout<SF>(P.f_out)[pop_index<SHIFT>(wr_dir<SM>(q), Sw, SM == SM_ODD ? nbr(cw, CX(q), CY(q), CZ(q)) : cw.idx)] =
        Store<SF>::put(pop_encode<SHIFT>(q, f[q], r0n, ph.rest1));
}

// ---- kernels of one domain ------------------------------------------------------------------
// Planes zb <= z < ze of the domain (a z slab, or the whole domain): grid (tiles
// in x, tiles in y, chunks of tz planes) of TX x TY blocks for the z-marching
// passes; one thread per cell, one z plane per blockIdx.z, for the collision.

template <typename T, typename SF, bool SOLID, int SM = SM_AB, bool OFF32 = false>
__global__ void __launch_bounds__(MacroShape::NT, blocks_of<MacroShape>((sizeof(T) == 4 && !SOLID) ? 4 : 1))
    k_macro(Geom g, Ptrs<T> P, Phys<T> ph, int tz, int zb, int ze) {
  const int z0 = zb + blockIdx.z * tz;
  macro_tile<T, SF, SOLID, SM, MacroShape, true, OFF32>(g, P, ph, z0, min(ze, z0 + tz), blockIdx.x, blockIdx.y);
}

template <typename T, bool SOLID>
__global__ void __launch_bounds__(NT) k_fields(Geom g, Ptrs<T> P, Phys<T> ph, int tz, int zb, int ze) {
  const int z0 = zb + blockIdx.z * tz;
  fields_tile<T, SOLID>(g, P, ph, z0, min(ze, z0 + tz), blockIdx.x, blockIdx.y);
}

template <typename T>
__global__ void __launch_bounds__(FieldShape::NT, blocks_of<FieldShape>(4))
    k_fields_sep(Geom g, Ptrs<T> P, Phys<T> ph, int tz, int zb, int ze) {
  const int z0 = zb + blockIdx.z * tz;
  fields_sep_tile<T, FieldShape>(g, P, ph, z0, min(ze, z0 + tz), blockIdx.x, blockIdx.y);
}

template <typename T>
__global__ void __launch_bounds__(DIV_THREADS, (sizeof(T) == 4) ? DIV_BLOCKS : 1)
    k_div_sep(Geom g, Ptrs<T> P, int tz, int use_Q, int zb, int ze) {
  const int z0 = zb + blockIdx.z * tz;
  div_sep_tile<T, DivShape, DIV_THREADS>(g, P, z0, min(ze, z0 + tz), use_Q, blockIdx.x, blockIdx.y);
}

template <typename T, typename SF, bool SOLID, bool UNIT, int SM = SM_AB>
__global__ void __launch_bounds__(128, 6) k_collide(Geom g, Ptrs<T> P, Phys<T> ph, int zb) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  if (x >= g.nx || y >= g.ny) return;
  Cell c;
  make_cell_at(g, x, y, zb + blockIdx.z, c);
  collide_cell<T, SF, SOLID, UNIT, SM>(g, P, ph, c);
}

// ---- fused pass: the collision of a step and the pulled sums of the next ------------------
// FP32, periodic, two population buffers.  A block owns a TX x TY tile of
// columns and the planes z0 <= z < z1, and walks the source planes z0-1 .. z1
// with the tile plus a one-cell ring (FW x FH = 340 positions, one thread
// each).  Every position pulls the totals of its cell, collides them
// (collide_pulled) and puts f^* in shared memory; tile cells of the planes
// z0 .. z1-1 also store f^* to the output buffer.  The tile threads then add
// the terms of that source plane to the sums of the cells above, at and below
// it in their column -- the pull of the next step, with the colour fractions
// of the source cells and DIVR (Eq. (recoloring)) as in the macroscopic pass,
// in its order (sum_dir) -- and write rho_r, rho_b, j and phi of the next step
// to mac_out and phi once a cell's third source plane is in.  The ring and the
// planes z0-1 and z1 belong to other blocks, which collide them with the same
// instructions, so the f^* summed here are bit for bit the stored ones and the
// sums equal those of the macroscopic pass on the next step.  The second
// population read of a step (the macroscopic pass) is gone: per cell the pass
// moves 152 bytes in and 132 out instead of 248 + 144 for the two passes.
// Needs 8 stride + nx ny < 2^31 (32-bit offsets of the pulled loads).
constexpr int FX = 32, FY = 8, FW = FX + 2, FH = FY + 2, FPL = FW * FH, FNT = (FPL + 31) / 32 * 32;

template <bool UNIT>
__global__ void __launch_bounds__(FNT, 2)
    k_collide_macro(Geom g, Ptrs<float> P, Phys<float> ph, int tz, int zb, int ze) {
  using T = float;
  __shared__ T sF[27][FPL];   // f^* of the source plane
  __shared__ float2 sW[FPL];  // its colour fractions (rho_r / rho, rho_b / rho)
  const int z0 = zb + blockIdx.z * tz, z1 = min(ze, z0 + tz);
  const int tid = threadIdx.x;
  const long long S = g.stride;
  // this thread's position: the tile cells, then the ring (the top row, the
  // bottom row, then both ends of the rows between)
  const bool has = tid < FPL, tile = tid < FX * FY;
  int lx = 0, ly = 0;
  if (tile) {
    lx = tid % FX + 1;
    ly = tid / FX + 1;
  } else if (has) {
    const int r = tid - FX * FY;
    if (r < FW) {
      lx = r;
    } else if (r < 2 * FW) {
      lx = r - FW;
      ly = FH - 1;
    } else {
      lx = ((r - 2 * FW) & 1) ? FW - 1 : 0;
      ly = 1 + (r - 2 * FW) / 2;
    }
  }
  const int pos = lx + FW * ly;
  const int gx = blockIdx.x * FX + lx - 1, gy = blockIdx.y * FY + ly - 1;
  const bool own = tile && gx < g.nx && gy < g.ny;
  const int x = wrapi(gx, g.nx), y = wrapi(gy, g.ny);
  const int xs[3] = {x == 0 ? g.nx - 1 : x - 1, x, x == g.nx - 1 ? 0 : x + 1};
  const int ys[3] = {(y == 0 ? g.ny - 1 : y - 1) * g.nx, y * g.nx, (y == g.ny - 1 ? 0 : y + 1) * g.nx};
  const int cxy = x + y * g.nx;
  // offset of direction j = (c_x + 1) + 3 (c_y + 1) of a z group from the
  // group's row base, the source column x - c included
  int off[9];
#pragma unroll
  for (int j = 0; j < 9; ++j) off[j] = j * (int)S + xs[1 - (j % 3 - 1)] + ys[1 - (j / 3 - 1)];
  const float* const fin = static_cast<const float*>(P.f_in);
  float* const fout = static_cast<float*>(P.f_out);
  // the inputs of this thread's cell in a source plane: 27 pulled totals;
  // rho_r, rho_b, F, Q and the colour fractions
  T f[27], in[10];
  auto fetch = [&](int z) {
    const int zo[3] = {zoff(g, z - 1), zoff(g, z), zoff(g, z + 1)};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float* const base = fin + 9LL * k * S + zo[2 - k];  // group c_z = k - 1 pulls from z - c_z
#pragma unroll
      for (int j = 0; j < 9; ++j) f[9 * k + j] = ld(base + off[j]);
    }
    const int i = cxy + zo[1];
    in[0] = ld(P.mac + i);
    in[1] = ld(P.mac + S + i);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      in[2 + a] = ld(P.force + a * S + i);
      in[5 + a] = ph.use_Q ? ld(P.qc + a * S + i) : T(0);
    }
    in[8] = ld(P.s_out + i);
    in[9] = ld(P.s_out + S + i);
  };
  // sums (rho_r, rho_b, j) of this column's cells in the planes s-1 and s
  T m_lo[5] = {T(0), T(0), T(0), T(0), T(0)}, m_mid[5] = {T(0), T(0), T(0), T(0), T(0)};
  if (has) fetch(z0 - 1);
  for (int s = z0 - 1; s <= z1; ++s) {
    // the sums of plane s+1 start from its DIVR (Eq. (recoloring) terms)
    T divr_up = T(0);
    if (tile && s + 1 < z1) divr_up = ld(P.s_out + S_DIVR * S + cxy + zoff(g, s + 1));
    if (has) {
      const T F[3] = {in[2], in[3], in[4]}, Q[3] = {in[5], in[6], in[7]};
      collide_pulled<T, UNIT>(f, in[0], in[1], F, Q, ph);
      if (own && s >= z0 && s < z1) {
        float* const o = fout + (cxy + s * g.nxy);
#pragma unroll
        for (int q = 0; q < 27; ++q) o[q * S] = f[q];
      }
#pragma unroll
      for (int q = 0; q < 27; ++q) sF[q][pos] = f[q];
      sW[pos] = make_float2(in[8], in[9]);
    }
    __syncthreads();
    if (has && s < z1) fetch(s + 1);  // in flight while the sums are formed
    if (tile) {
      // fractions of the nine source cells x - c of this plane, j = (c_x + 1) + 3 (c_y + 1)
      float2 w[9];
#pragma unroll
      for (int j = 0; j < 9; ++j) w[j] = sW[pos - (j % 3 - 1) - FW * (j / 3 - 1)];
      T m_up[5] = {divr_up, -divr_up, T(0), T(0), T(0)};
      // c_z = +1: plane s+1; c_z = 0: plane s; c_z = -1: plane s-1 (sum_dir order)
#pragma unroll
      for (int q = 18; q < 27; ++q) add_pulled(q, sF[q][pos - CX(q) - FW * CY(q)], w[q % 9].x, w[q % 9].y, m_up);
#pragma unroll
      for (int q = 9; q < 18; ++q) add_pulled(q, sF[q][pos - CX(q) - FW * CY(q)], w[q % 9].x, w[q % 9].y, m_mid);
#pragma unroll
      for (int q = 0; q < 9; ++q) add_pulled(q, sF[q][pos - CX(q) - FW * CY(q)], w[q % 9].x, w[q % 9].y, m_lo);
      if (own && s - 1 >= z0 && s - 1 < z1) {
        const int i = cxy + (s - 1) * g.nxy;
#pragma unroll
        for (int a = 0; a < 5; ++a) P.mac_out[a * S + i] = m_lo[a];
        P.phi[i] = order_parameter(m_lo[0], m_lo[1], ph);
        if (!isfinite(m_lo[0] + m_lo[1])) atomicOr(P.flag, 1u);
      }
#pragma unroll
      for (int a = 0; a < 5; ++a) {
        m_lo[a] = m_mid[a];
        m_mid[a] = m_up[a];
      }
    }
    __syncthreads();  // the next plane overwrites sF and sW
  }
}

// ---- kernels of a batch of domains -----------------------------------------------------------
// Every pass of every member domain is one launch over a work list: work item
// i of a z-marching pass (domain, tile x, tile y, z chunk) comes from a table
// written on the host, so a tile starts from one 16-byte load; collision item
// b covers cells 128 (b - cell_start[d]) ... + 127 of the domain d with
// cell_start[d] <= b < cell_start[d + 1], in storage order.  A block takes
// items blockIdx.x, blockIdx.x + gridDim.x, ...: with one block per item this
// is the plain form, with a grid of the resident blocks of the GPU it is a
// persistent kernel that walks the list.  The arithmetic of each cell is that
// of the single-domain kernels, whatever the grid.

template <typename T>
struct Dom {
  Geom g;
  Phys<T> ph;
  Ptrs<T> P[2];  // buffers of the even and odd steps of the batch
  int tz, tiles_x, tiles_y, use_Q;
  // the member takes part in the batch's steps number < stop, counted from the
  // table write; *tick is the step number at the start of the current launch
  const int* tick;
  int stop;
};

// `sp` of a batch launch: parity of its buffers in bit 0, its step offset
// within the launch (graph) above; a member past its stop sits it out
template <typename T>
__device__ __forceinline__ bool sits_out(const Dom<T>& D, int sp) {
  return __ldg(D.tick) + (sp >> 1) >= D.stop;
}

// largest d with start[d] <= b (start is non-decreasing, start[0] = 0)
__device__ __forceinline__ int find_domain(const int* __restrict__ start, int ndom, int b) {
  int lo = 0, hi = ndom - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(start + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Tiles of a z-marching batch pass: item i = (domain, tile x, tile y, z chunk).
// PERSIST = false: block b runs item b.  PERSIST = true: block b runs items b,
// b + gridDim.x, ..., waiting at a barrier before each further one, so the
// next tile's shared-memory prologue follows the last reads of the previous
// tile.  (The two forms are separate instantiations: the loop costs the
// one-item form about 5 % when it is compiled in.)
template <typename T, typename SF, bool SOLID, class SH>
__device__ __forceinline__ void macro_item(const Dom<T>* __restrict__ doms, int4 t, int sp) {
  const Dom<T>& D = doms[t.x];
  if (sits_out(D, sp)) return;
  const int par = sp & 1;
  macro_tile<T, SF, SOLID, SM_AB, SH, true, true>(D.g, D.P[par], D.ph, t.w * D.tz, min(D.g.nz, (t.w + 1) * D.tz), t.y, t.z);
}

template <typename T, bool SOLID, class SH>
__device__ __forceinline__ void fields_item(const Dom<T>* __restrict__ doms, int4 t, int sp) {
  const Dom<T>& D = doms[t.x];
  if (sits_out(D, sp)) return;
  const int par = sp & 1;
  if constexpr (!SOLID && sizeof(T) == 4)
    fields_sep_tile<T, SH>(D.g, D.P[par], D.ph, t.w * D.tz, min(D.g.nz, (t.w + 1) * D.tz), t.y, t.z);
  else
    fields_tile<T, SOLID, SH>(D.g, D.P[par], D.ph, t.w * D.tz, min(D.g.nz, (t.w + 1) * D.tz), t.y, t.z);
}

template <typename T, class SH>
__device__ __forceinline__ void div_item(const Dom<T>* __restrict__ doms, int4 t, int sp) {
  const Dom<T>& D = doms[t.x];
  if (sits_out(D, sp)) return;
  const int par = sp & 1;
  div_sep_tile<T, SH>(D.g, D.P[par], t.w * D.tz, min(D.g.nz, (t.w + 1) * D.tz), D.use_Q, t.y, t.z);
}

// blocks per SM that the register caps of the batch kernels aim at: those of
// the single-domain kernels for 256 threads, twice as many for 128
template <class SH>
constexpr int per_sm(int blocks256) { return blocks256 * (256 / SH::NT); }

template <typename T, typename SF, bool SOLID, bool PERSIST, class SH>
__global__ void __launch_bounds__(SH::NT, per_sm<SH>((sizeof(T) == 4 && !SOLID) ? 4 : 1))
    k_macro_batch(const Dom<T>* __restrict__ doms, const int4* __restrict__ items, int nitems, int sp) {
  if constexpr (!PERSIST) {
    macro_item<T, SF, SOLID, SH>(doms, __ldg(items + blockIdx.x), sp);
  } else {
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
      if (i != (int)blockIdx.x) __syncthreads();
      macro_item<T, SF, SOLID, SH>(doms, __ldg(items + i), sp);
    }
  }
}

template <typename T, bool SOLID, bool PERSIST, class SH>
__global__ void __launch_bounds__(SH::NT, per_sm<SH>((!SOLID && sizeof(T) == 4) ? 3 : 1))
    k_fields_batch(const Dom<T>* __restrict__ doms, const int4* __restrict__ items, int nitems, int sp) {
  if constexpr (!PERSIST) {
    fields_item<T, SOLID, SH>(doms, __ldg(items + blockIdx.x), sp);
  } else {
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
      if (i != (int)blockIdx.x) __syncthreads();
      fields_item<T, SOLID, SH>(doms, __ldg(items + i), sp);
    }
  }
}

template <typename T, bool PERSIST, class SH>
__global__ void __launch_bounds__(SH::NT)
    k_div_batch(const Dom<T>* __restrict__ doms, const int4* __restrict__ items, int nitems, int sp) {
  if constexpr (!PERSIST) {
    div_item<T, SH>(doms, __ldg(items + blockIdx.x), sp);
  } else {
    for (int i = blockIdx.x; i < nitems; i += gridDim.x) {
      if (i != (int)blockIdx.x) __syncthreads();
      div_item<T, SH>(doms, __ldg(items + i), sp);
    }
  }
}

// collision item blk (batch-wide numbering of start): 128 cells of one domain
template <typename T, typename SF, bool SOLID, bool UNIT>
__device__ __forceinline__ void collide_item(const Dom<T>* __restrict__ doms, const int* __restrict__ start,
                                             int ndom, int sp, int blk) {
  const int d = find_domain(start, ndom, blk);
  const Dom<T>& D = doms[d];
  if (sits_out(D, sp)) return;
  const int par = sp & 1;
  // domains hold fewer than 2^31 cells, so 32-bit unsigned index arithmetic is exact
  const unsigned i = (unsigned)(blk - __ldg(start + d)) * 128u + threadIdx.x;
  const unsigned nxy = (unsigned)D.g.nxy, nx = (unsigned)D.g.nx;
  if (i >= nxy * (unsigned)D.g.nz) return;
  const unsigned z = i / nxy, r = i - z * nxy, y = r / nx;
  Cell c;
  make_cell_at(D.g, (int)(r - y * nx), (int)y, (int)z, c);
  collide_cell<T, SF, SOLID, UNIT>(D.g, D.P[par], D.ph, c);
}

// doms and start point at the first domain of a group of members; block0 is
// that domain's first 128-cell item in the batch-wide numbering of start; the
// group has nblocks items
template <typename T, typename SF, bool SOLID, bool UNIT, bool PERSIST>
__global__ void __launch_bounds__(128, 6)
    k_collide_batch(const Dom<T>* __restrict__ doms, const int* __restrict__ start, int ndom, int sp,
                    int block0, int nblocks) {
  if constexpr (!PERSIST) {
    collide_item<T, SF, SOLID, UNIT>(doms, start, ndom, sp, (int)blockIdx.x + block0);
  } else {
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) collide_item<T, SF, SOLID, UNIT>(doms, start, ndom, sp, b + block0);
  }
}

}  // namespace cg27
