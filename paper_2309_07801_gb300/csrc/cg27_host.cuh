// cg27_host.cuh -- host-side state shared by the C-ABI translation units:
// the error text, the workspace layout of a domain, the domain context and the
// kernel argument builders.  Internal to the library (not installed).
#pragma once

#include "cg27.h"
#include "cg27_device.cuh"
#include "cg27_step.cuh"

#include <string>
#include <vector>

namespace cg27 {

inline thread_local std::string g_err;

inline int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CG_CUDA(expr)                                                              \
  do {                                                                             \
    cudaError_t e_ = (expr);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return fail(CG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

constexpr size_t ALIGN = 256;
inline size_t align_up(size_t v) { return (v + ALIGN - 1) / ALIGN * ALIGN; }

// a schedule of the step graphs: slabs of `planes` planes, tiles of `tz`
// planes, and the step form (ftz = 0: four passes; > 0: fused collision
// pass with tiles of ftz planes)
struct StepSched {
  int planes = 0, tz = 0, ftz = 0;
  bool operator==(const StepSched& o) const { return planes == o.planes && tz == o.tz && ftz == o.ftz; }
  bool operator<(const StepSched& o) const {
    return planes != o.planes ? planes < o.planes : (tz != o.tz ? tz < o.tz : ftz < o.ftz);
  }
};

struct Layout {
  long long n = 0, stride = 0;
  size_t elem = 0;      // bytes of an arithmetic value (FP64 or FP32)
  size_t pop_elem = 0;  // bytes of a stored population
  int ns = 6;           // fields of the recoloring state
  int nq = 27;          // populations per cell (27 for D3Q27, 9 for D2Q9)
  bool solid = false;
  bool inplace = false;  // one population buffer (f[1] == f[0]), updated in place
  int red_blocks = 0;
  size_t f[2] = {0, 0}, s[2] = {0, 0}, aux[2] = {0, 0};
  size_t mask = 0, phi = 0, qc = 0, force = 0, wv = 0;
  // rho_r, rho_b, j: mac[p] is written by the macroscopic pass of a step of
  // parity p, or by the fused collision pass of the step before it; the two
  // are one buffer unless the domain can take the fused pass (fusable)
  size_t mac[2] = {0, 0};
  bool fusable = false;
  size_t partial = 0, flag = 0, result = 0, diag = 0, total = 0;
};

}  // namespace cg27

// bytes of the diagnostics scratch for a reduction grid (cg27_diag.cu)
size_t cg27_diag_bytes(int red_blocks);

namespace cg27 {

}  // namespace cg27

struct cg_ctx {
  cg_params prm;
  cg_batch* batch = nullptr;  // the batch the domain is a member of, if any
  int64_t batch_stop = -1;    // step count at which it sits out the batch's steps (-1: none)
  cudaStream_t batch_stream = nullptr;  // and the stream that batch launches on
  cg27::Layout L;
  char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int64_t steps = 0;
  bool initialised = false;
  bool unit = false;  // all omega = 1 except omega_1, Model D: the Sec. III.E form
  int tz = 1;         // z planes per tile of the step kernels
  // per-pass timing: events[(CG_NUM_PASSES + 1) * s + k] brackets pass k of timed step s
  std::vector<cudaEvent_t> events;
  int64_t prof_capacity = 0, prof_used = 0;
  // graphs of the slab pipeline, [one step | a chain of steps][parity of the
  // first step], all four built by the first step that uses them
  cudaGraphExec_t sgraph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool graphs_ok = true;
  // schedule of the graphs: slabs of sched_planes planes, tiles of sched_tz
  // planes (0: not chosen yet); candidates still to time and the timings
  int sched_planes = 0, sched_tz = 0;
  std::vector<cg27::StepSched> sched_cand;
  std::vector<std::pair<float, cg27::StepSched>> sched_timed;
  int tune_phase = 0;  // 0: next chain untimed, 1..: timed chains of the candidate
  // the schedule's step form: sched_ftz = 0 runs the four passes, > 0 the
  // macroscopic pass folded into the collision of the previous step
  // (k_collide_macro, tiles of sched_ftz planes); mac_ready is the step
  // whose sums that pass has left in mac[step & 1] (-1: none)
  int sched_ftz = 0;
  int64_t mac_ready = -1;
  cudaEvent_t tev[2] = {nullptr, nullptr};
  ~cg_ctx() {
    for (cudaEvent_t e : events) cudaEventDestroy(e);
    for (cudaEvent_t e : tev)
      if (e) cudaEventDestroy(e);
    for (auto& row : sgraph)
      for (cudaGraphExec_t g : row)
        if (g) cudaGraphExecDestroy(g);
  }
};

namespace cg27 {

template <typename T>
inline Phys<T> make_phys(const cg_params& p) {
  Phys<T> ph;
  // EOS constant: (c_s^k)^2 = xi (1 - alpha_k); xi = 9/19 for D3Q27 (Sec. II.A),
  // 3/5 for D2Q9 (alpha = w_0 = 4/9 gives c_s^2 = 1/3)
  const double xi = p.lattice == CG_D2Q9 ? 3.0 / 5.0 : 9.0 / 19.0;
  ph.rho_r0 = T(p.rho_r0);
  ph.rho_b0 = T(p.rho_b0);
  ph.inv_rho_r0 = T(1.0 / p.rho_r0);
  ph.inv_rho_b0 = T(1.0 / p.rho_b0);
  ph.cr2 = T(xi * (1.0 - p.alpha_r));
  ph.cb2 = T(xi * (1.0 - p.alpha_b));
  ph.nu_r = T(p.nu_r);
  ph.nu_b = T(p.nu_b);
  ph.sigma = T(p.sigma);
  ph.beta = T(p.beta);
  for (int q = 0; q < 11; ++q) ph.om[q] = T(p.omega[q]);
  for (int a = 0; a < 3; ++a) ph.g[a] = T(p.g[a]);
  ph.rho_ref = T(p.rho_ref);
  ph.force_mode = p.force_mode;
  ph.model = p.model;
  ph.use_Q = p.use_Q;
  ph.shift = (p.precision == CG_F16S || p.precision == CG_BF16S) ? 1 : 0;
  // reference pressure of the red phase at its reference density
  ph.rest1 = T(3.0 * p.rho_r0 * xi * (1.0 - p.alpha_r));
  for (int a = 0; a < 3; ++a) ph.bc[a] = p.bc[a];
  for (int f = 0; f < 6; ++f)
    for (int b = 0; b < 3; ++b) ph.wall_u[f][b] = T(p.bc[f / 2] == CG_BC_MOVING ? p.wall_u[f][b] : 0.0);
  return ph;
}

inline Geom make_geom(const cg_ctx* c) {
  Geom g;
  g.nx = c->prm.nx;
  g.ny = c->prm.ny;
  g.nz = c->prm.nz;
  g.nxy = c->prm.nx * c->prm.ny;
  g.stride = c->L.stride;
  return g;
}

// pointers for a step that reads buffer `cur` and writes buffer 1 - cur
// (mac: the sums of that step; mac_out: of the next one)
template <typename T>
inline Ptrs<T> make_ptrs(const cg_ctx* c, int cur) {
  const Layout& L = c->L;
  Ptrs<T> P;
  char* w = c->ws;
  P.f_in = w + L.f[cur];
  P.f_out = w + L.f[1 - cur];
  P.s_in = reinterpret_cast<const T*>(w + L.s[cur]);
  P.s_out = reinterpret_cast<T*>(w + L.s[1 - cur]);
  P.aux_in = L.solid ? reinterpret_cast<const T*>(w + L.aux[cur]) : nullptr;
  P.aux_out = L.solid ? reinterpret_cast<T*>(w + L.aux[1 - cur]) : nullptr;
  P.mask = L.solid ? reinterpret_cast<const uint32_t*>(w + L.mask) : nullptr;
  P.mac = reinterpret_cast<T*>(w + L.mac[cur]);
  P.mac_out = reinterpret_cast<T*>(w + L.mac[1 - cur]);
  P.phi = reinterpret_cast<T*>(w + L.phi);
  P.qc = reinterpret_cast<T*>(w + L.qc);
  P.force = reinterpret_cast<T*>(w + L.force);
  P.wv = reinterpret_cast<T*>(w + L.wv);
  P.flag = reinterpret_cast<unsigned int*>(w + L.flag);
  return P;
}

// the sums of the last step taken (of the initial state before the first):
// what the read-back, reductions and checkpoints see
inline size_t mac_last(const cg_ctx* c) { return c->L.mac[1 - (int)(c->steps & 1)]; }

// pointers of the current state, mac pointing at the last step's sums
template <typename T>
inline Ptrs<T> state_ptrs(const cg_ctx* c) {
  Ptrs<T> P = make_ptrs<T>(c, (int)(c->steps & 1));
  P.mac = P.mac_out;
  return P;
}

}  // namespace cg27
