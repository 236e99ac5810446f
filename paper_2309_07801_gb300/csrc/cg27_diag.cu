// cg27_diag.cu -- diagnostics of a domain reduced on the device in FP64:
// per-colour masses, momenta and centroids, the red second-moment tensor,
// the mean pressure inside and outside a sphere (the pressure jump of the
// Laplace test, Sec. IV.A), the rise quantities of Sec. IV.D (blue centroid
// and momentum) and the largest speed.  Two passes over the cells, each a
// fixed grid of blocks with contiguous cell ranges, per-block partial sums in
// a fixed order (warp shuffles, then warps in order) and one block summing the
// partials in block order: the results are bitwise reproducible and need no
// host read-back of any field.
#include "cg27_host.cuh"

#include <cmath>
#include <string>

using namespace cg27;

namespace {

constexpr int DG_THREADS = 256;
constexpr int DG_WARPS = DG_THREADS / 32;

// slots of the first pass (summed unless noted)
enum : int {
  Q_MR, Q_MB,                   // sum rho_r, sum rho_b (all cells)
  Q_VOL,                        // sum (1 + phi) / 2 over fluid cells
  Q_JR0, Q_JR1, Q_JR2,          // sum rho_r u (fluid cells)
  Q_JB0, Q_JB1, Q_JB2,          // sum rho_b u
  Q_RC0, Q_RC1, Q_RC2,          // sum rho_r cos(2 pi x_a / n_a)
  Q_RS0, Q_RS1, Q_RS2,          // sum rho_r sin(2 pi x_a / n_a)
  Q_RX0, Q_RX1, Q_RX2,          // sum rho_r x_a
  Q_BC0, Q_BC1, Q_BC2,          // the same for rho_b
  Q_BS0, Q_BS1, Q_BS2,
  Q_BX0, Q_BX1, Q_BX2,
  Q_PIN, Q_NIN, Q_POUT, Q_NOUT, // p and cell count inside r_in / outside r_out
  Q_UMAX,                       // max |u| (a max, not a sum)
  NQ1
};
constexpr int NQ2 = 6;  // second pass: rho_r d_a d_b (xx, yy, zz, xy, xz, yz)

// result block in the workspace: the first-pass totals, the two centroids
// (red, blue), then the second-pass totals
constexpr int R_CEN = NQ1, R_M2 = NQ1 + 6, R_LEN = NQ1 + 6 + NQ2;

struct DiagArgs {
  double center[3];
  double r_in2, r_out2;
  int periodic[3];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// cells of block b: a contiguous range, the same for every call on this domain
__device__ __forceinline__ void block_range(long long n, long long& lo, long long& hi) {
  const long long per = (n + gridDim.x - 1) / gridDim.x;
  lo = (long long)blockIdx.x * per;
  hi = lo + per < n ? lo + per : n;
}

// minimum-image offset of coordinate x from c on an axis of n cells
__device__ __forceinline__ double offset(double x, double c, int n, int periodic) {
  double d = x - c;
  if (periodic) {
    d = fmod(d + 0.5 * n, (double)n);
    if (d < 0) d += n;
    d -= 0.5 * n;
  }
  return d;
}

template <int NQ>
__device__ __forceinline__ void block_reduce(double (&acc)[NQ], int max_slot, double* out) {
  __shared__ double s[DG_WARPS][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const double v = q == max_slot ? warp_max(acc[q]) : warp_sum(acc[q]);
    if (lane == 0) s[warp][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    const int q = threadIdx.x;
    double v = s[0][q];
    for (int w = 1; w < DG_WARPS; ++w) v = q == max_slot ? fmax(v, s[w][q]) : v + s[w][q];
    out[(size_t)blockIdx.x * NQ + q] = v;
  }
}

template <typename T, bool SOLID>
__global__ void __launch_bounds__(DG_THREADS) k_diag_partial(Geom g, Ptrs<T> P, Phys<T> ph, DiagArgs a,
                                                             long long n, double* partial) {
  double acc[NQ1];
#pragma unroll
  for (int q = 0; q < NQ1; ++q) acc[q] = 0.0;
  long long lo, hi;
  block_range(n, lo, hi);
  const long long S = g.stride;
  const int nn[3] = {g.nx, g.ny, g.nz};
  for (long long i = lo + threadIdx.x; i < hi; i += DG_THREADS) {
    const int ii = (int)i;
    const int z = ii / g.nxy, r = ii - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    const int xs[3] = {x, y, z};
    const T rrT = P.mac[ii], rbT = P.mac[S + ii];
    const double rr = double(rrT), rb = double(rbT);
    acc[Q_MR] += rr;
    acc[Q_MB] += rb;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double sn, cs;
      sincospi(2.0 * xs[k] / nn[k], &sn, &cs);
      acc[Q_RC0 + k] += rr * cs;
      acc[Q_RS0 + k] += rr * sn;
      acc[Q_RX0 + k] += rr * xs[k];
      acc[Q_BC0 + k] += rb * cs;
      acc[Q_BS0 + k] += rb * sn;
      acc[Q_BX0 + k] += rb * xs[k];
    }
    const bool solid = SOLID && ((ld(P.mask + ii) >> SELF_SOLID_BIT) & 1u);
    if (solid) continue;
    // the fields cg_read_macros() reports: u with F/2, p, phi (arithmetic type of the mode)
    const T rho = rrT + rbT;
    double u[3], u2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      u[k] = double((P.mac[(2 + k) * S + ii] + P.force[k * S + ii] / T(2)) / rho);
      u2 += u[k] * u[k];
      acc[Q_JR0 + k] += rr * u[k];
      acc[Q_JB0 + k] += rb * u[k];
    }
    const double p = double(rrT * ph.cr2 + rbT * ph.cb2);
    acc[Q_VOL] += 0.5 * (1.0 + double(order_parameter(rrT, rbT, ph)));
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double d = offset((double)xs[k], a.center[k], nn[k], a.periodic[k]);
      d2 += d * d;
    }
    if (d2 < a.r_in2) {
      acc[Q_PIN] += p;
      acc[Q_NIN] += 1.0;
    }
    if (d2 > a.r_out2) {
      acc[Q_POUT] += p;
      acc[Q_NOUT] += 1.0;
    }
    acc[Q_UMAX] = fmax(acc[Q_UMAX], sqrt(u2));
  }
  block_reduce<NQ1>(acc, Q_UMAX, partial);
}

// centroid of one colour along axis k from its sums: circular mean on a
// periodic axis, arithmetic mean on a wall axis
__device__ __forceinline__ double centroid(double m, double c, double s, double xm, int n, int periodic) {
  if (m <= 0.0) return 0.0;
  if (!periodic) return xm / m;
  double th = atan2(s, c);
  if (th < 0) th += 2.0 * M_PI;
  return th * n / (2.0 * M_PI);
}

template <int NQ>
__device__ __forceinline__ void final_sum(const double* partial, int nblocks, int max_slot, double* res) {
  const int q = threadIdx.x;
  if (q < NQ) {
    double v = partial[q];
    for (int b = 1; b < nblocks; ++b) {
      const double w = partial[(size_t)b * NQ + q];
      v = q == max_slot ? fmax(v, w) : v + w;
    }
    res[q] = v;
  }
}

__global__ void k_diag_final1(const double* partial, int nblocks, Geom g, DiagArgs a, double* res) {
  final_sum<NQ1>(partial, nblocks, Q_UMAX, res);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nn[3] = {g.nx, g.ny, g.nz};
    for (int k = 0; k < 3; ++k) {
      res[R_CEN + k] = centroid(res[Q_MR], res[Q_RC0 + k], res[Q_RS0 + k], res[Q_RX0 + k], nn[k], a.periodic[k]);
      res[R_CEN + 3 + k] =
          centroid(res[Q_MB], res[Q_BC0 + k], res[Q_BS0 + k], res[Q_BX0 + k], nn[k], a.periodic[k]);
    }
  }
}

// second pass: rho_r-weighted second moments about the red centroid
template <typename T>
__global__ void __launch_bounds__(DG_THREADS) k_diag_partial2(Geom g, Ptrs<T> P, DiagArgs a, long long n,
                                                              const double* res, double* partial) {
  double acc[NQ2];
#pragma unroll
  for (int q = 0; q < NQ2; ++q) acc[q] = 0.0;
  const double c[3] = {res[R_CEN], res[R_CEN + 1], res[R_CEN + 2]};
  const int nn[3] = {g.nx, g.ny, g.nz};
  long long lo, hi;
  block_range(n, lo, hi);
  for (long long i = lo + threadIdx.x; i < hi; i += DG_THREADS) {
    const int ii = (int)i;
    const int z = ii / g.nxy, r = ii - z * g.nxy, y = r / g.nx, x = r - y * g.nx;
    const int xs[3] = {x, y, z};
    const double rr = double(P.mac[ii]);
    double d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = offset((double)xs[k], c[k], nn[k], a.periodic[k]);
    acc[0] += rr * d[0] * d[0];
    acc[1] += rr * d[1] * d[1];
    acc[2] += rr * d[2] * d[2];
    acc[3] += rr * d[0] * d[1];
    acc[4] += rr * d[0] * d[2];
    acc[5] += rr * d[1] * d[2];
  }
  block_reduce<NQ2>(acc, -1, partial);
}

__global__ void k_diag_final2(const double* partial, int nblocks, double* res) {
  final_sum<NQ2>(partial, nblocks, -1, res + R_M2);
}

template <typename T, bool SOLID>
void enqueue_diag(cg_ctx* c, const DiagArgs& a, double* partial, double* res) {
  const Geom g = make_geom(c);
  const Ptrs<T> P = state_ptrs<T>(c);
  const int nb = c->L.red_blocks;
  k_diag_partial<T, SOLID><<<nb, DG_THREADS, 0, c->stream>>>(g, P, make_phys<T>(c->prm), a, c->L.n, partial);
  k_diag_final1<<<1, 64, 0, c->stream>>>(partial, nb, g, a, res);
  k_diag_partial2<T><<<nb, DG_THREADS, 0, c->stream>>>(g, P, a, c->L.n, res, partial);
  k_diag_final2<<<1, 32, 0, c->stream>>>(partial, nb, res);
}

}  // namespace

// the diagnostics scratch of a workspace (bytes), used by the layout in cg27_capi.cu
__attribute__((visibility("hidden"))) size_t cg27_diag_bytes(int red_blocks) {
  return ((size_t)red_blocks * NQ1 + R_LEN) * sizeof(double);
}

extern "C" int cg_reduce_diagnostics(cg_ctx* c, const double center[3], double r_in, double r_out,
                                     cg_diagnostics* out) {
  if (!c || !out) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  if (c->batch) CG_CUDA(cudaStreamSynchronize(c->batch_stream));
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  DiagArgs a;
  for (int k = 0; k < 3; ++k) {
    a.center[k] = center ? center[k] : 0.0;
    if (!std::isfinite(a.center[k])) return fail(CG_ERR_INVALID_ARG, "center must be finite");
    a.periodic[k] = c->prm.bc[k] == CG_BC_PERIODIC;
  }
  if (!(r_in >= 0.0) || !(r_out >= 0.0)) return fail(CG_ERR_INVALID_ARG, "r_in, r_out must be >= 0");
  a.r_in2 = r_in * r_in;
  a.r_out2 = std::isinf(r_out) ? r_out : r_out * r_out;
  double* partial = reinterpret_cast<double*>(c->ws + c->L.diag);
  double* res = partial + (size_t)c->L.red_blocks * NQ1;
  if (c->prm.precision == CG_F64) {
    if (c->L.solid) enqueue_diag<double, true>(c, a, partial, res);
    else enqueue_diag<double, false>(c, a, partial, res);
  } else {
    if (c->L.solid) enqueue_diag<float, true>(c, a, partial, res);
    else enqueue_diag<float, false>(c, a, partial, res);
  }
  CG_CUDA(cudaGetLastError());
  double h[R_LEN];
  unsigned int flag = 0;
  CG_CUDA(cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(cudaMemcpyAsync(&flag, c->ws + c->L.flag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(cudaStreamSynchronize(c->stream));
  out->mass[0] = h[Q_MR];
  out->mass[1] = h[Q_MB];
  out->red_volume = h[Q_VOL];
  for (int k = 0; k < 3; ++k) {
    out->momentum[0][k] = h[Q_JR0 + k];
    out->momentum[1][k] = h[Q_JB0 + k];
    out->centroid[0][k] = h[R_CEN + k];
    out->centroid[1][k] = h[R_CEN + 3 + k];
  }
  const double mr = h[Q_MR] > 0.0 ? h[Q_MR] : 1.0;
  for (int q = 0; q < NQ2; ++q) out->second_moment[q] = h[R_M2 + q] / mr;
  out->n_in = (int64_t)h[Q_NIN];
  out->n_out = (int64_t)h[Q_NOUT];
  out->p_in = h[Q_NIN] > 0 ? h[Q_PIN] / h[Q_NIN] : NAN;
  out->p_out = h[Q_NOUT] > 0 ? h[Q_POUT] / h[Q_NOUT] : NAN;
  out->u_max = h[Q_UMAX];
  out->nonfinite = flag ? 1 : 0;
  out->reserved = 0;
  return CG_OK;
}
