// cg27_capi.cu -- host side of the C ABI declared in include/cg27.h:
// workspace layout, kernel launches of one time step, initialisation,
// read-back, reductions and checkpoints.  Device code is in cg27_device.cuh.
#include "cg27_host.cuh"
#include <algorithm>
#include "cg27_d2q9.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

using namespace cg27;

namespace {

// paper velocity order (Sec. II.A) -> lexicographic storage index
int paper_to_lex(int i) {
  static const int C[27][3] = {
      {0, 0, 0},   {1, 0, 0},  {-1, 0, 0},  {0, 1, 0},   {0, -1, 0},  {0, 0, 1},   {0, 0, -1},
      {1, 1, 0},   {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},
      {0, -1, 1},  {1, 0, 1},  {-1, 0, -1}, {1, 0, -1},  {-1, 0, 1},  {1, 1, 1},   {-1, -1, -1},
      {1, 1, -1},  {-1, -1, 1}, {1, -1, 1}, {-1, 1, -1}, {-1, 1, 1},  {1, -1, -1}};
  return (C[i][0] + 1) + 3 * (C[i][1] + 1) + 9 * (C[i][2] + 1);
}

// D2Q9 velocity order of App. A -> lexicographic storage index (c_x + 1) + 3 (c_y + 1)
int paper_to_lex2(int i) {
  static const int C[9][2] = {{0, 0}, {1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, -1}, {1, -1}, {-1, 1}};
  return (C[i][0] + 1) + 3 * (C[i][1] + 1);
}

constexpr int RED_THREADS = 256;
constexpr int NUM_EVENTS_PER_STEP = CG_NUM_PASSES + 1;

// steps a batch has enqueued for a member domain complete before the
// domain's own stream reads its state
int settle(const cg_ctx* c) {
  if (c->batch) CG_CUDA(cudaStreamSynchronize(c->batch_stream));
  return CG_OK;
}

bool needs_solid(const cg_params& p) {
  return p.solid_mask != 0 || p.bc[0] != CG_BC_PERIODIC || p.bc[1] != CG_BC_PERIODIC ||
         p.bc[2] != CG_BC_PERIODIC;
}

int validate(const cg_params* p) {
  if (!p) return fail(CG_ERR_INVALID_ARG, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(CG_ERR_INVALID_ARG, "nx, ny, nz must be >= 1");
  if ((long long)p->nx * p->ny * p->nz > (1ll << 31) - 1)
    return fail(CG_ERR_INVALID_ARG, "more than 2^31-1 cells");
  if (p->nz > 65535) return fail(CG_ERR_INVALID_ARG, "nz must be <= 65535");
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a) {
    if (p->bc[a] < CG_BC_PERIODIC || p->bc[a] > CG_BC_MOVING)
      return fail(CG_ERR_INVALID_ARG, "bc must be CG_BC_PERIODIC, BOUNCEBACK, SLIP or MOVING");
    if (p->bc[a] != CG_BC_PERIODIC && n[a] < 3)
      return fail(CG_ERR_INVALID_ARG, "a wall axis needs at least 3 cells");
    for (int f = 2 * a; f < 2 * a + 2; ++f)
      for (int b = 0; b < 3; ++b) {
        if (!std::isfinite(p->wall_u[f][b])) return fail(CG_ERR_INVALID_ARG, "wall_u must be finite");
        if (p->bc[a] == CG_BC_MOVING && b == a && p->wall_u[f][b] != 0.0)
          return fail(CG_ERR_INVALID_ARG, "a moving wall moves in its own plane (normal component 0)");
      }
  }
  if (!(p->rho_r0 > 0) || !(p->rho_b0 > 0)) return fail(CG_ERR_INVALID_ARG, "rho_r0, rho_b0 must be > 0");
  if (!(p->alpha_r >= 0 && p->alpha_r < 1) || !(p->alpha_b >= 0 && p->alpha_b < 1))
    return fail(CG_ERR_INVALID_ARG, "alpha_r, alpha_b must be in [0, 1)");
  if (!(p->nu_r >= 0) || !(p->nu_b >= 0)) return fail(CG_ERR_INVALID_ARG, "viscosities must be >= 0");
  if (!std::isfinite(p->sigma) || !std::isfinite(p->beta)) return fail(CG_ERR_INVALID_ARG, "sigma, beta must be finite");
  for (int q = 0; q < 11; ++q)
    if (!std::isfinite(p->omega[q])) return fail(CG_ERR_INVALID_ARG, "omega must be finite");
  if (p->force_mode < CG_FORCE_NONE || p->force_mode > CG_FORCE_BUOYANCY)
    return fail(CG_ERR_INVALID_ARG, "unknown force_mode");
  if (p->model < CG_MODEL_A || p->model > CG_MODEL_D) return fail(CG_ERR_INVALID_ARG, "unknown model");
  if (p->precision != CG_F64 && p->precision != CG_F32 && p->precision != CG_F16S &&
      p->precision != CG_BF16S)
    return fail(CG_ERR_UNSUPPORTED, "precision must be CG_F64, CG_F32, CG_F16S or CG_BF16S");
  if ((p->precision == CG_F16S || p->precision == CG_BF16S) && needs_solid(*p))
    return fail(CG_ERR_UNSUPPORTED, "walls are not available with 16-bit population storage");
  if ((p->precision == CG_F16S || p->precision == CG_BF16S) &&
      27.0 * (((double)p->nx * p->ny * p->nz + 63) / 64 * 64) >= 4294967296.0)
    return fail(CG_ERR_UNSUPPORTED, "16-bit population storage is limited to 159 million cells");
  if (p->lattice != CG_D3Q27 && p->lattice != CG_D2Q9) return fail(CG_ERR_INVALID_ARG, "unknown lattice");
  if (p->streaming != CG_STREAM_TWO_BUFFERS && p->streaming != CG_STREAM_IN_PLACE)
    return fail(CG_ERR_INVALID_ARG, "streaming must be CG_STREAM_TWO_BUFFERS or CG_STREAM_IN_PLACE");
  if (p->reserved0 != 0) return fail(CG_ERR_INVALID_ARG, "reserved0 must be 0");
  if (p->streaming == CG_STREAM_IN_PLACE && p->lattice != CG_D3Q27)
    return fail(CG_ERR_UNSUPPORTED, "in-place streaming is implemented for D3Q27");
  if (p->lattice == CG_D2Q9) {
    if (p->nz != 1) return fail(CG_ERR_INVALID_ARG, "a D2Q9 domain has nz = 1");
    if (p->bc[2] != CG_BC_PERIODIC) return fail(CG_ERR_INVALID_ARG, "a D2Q9 domain has bc[2] = CG_BC_PERIODIC");
    if (p->bc[0] > CG_BC_BOUNCEBACK || p->bc[1] > CG_BC_BOUNCEBACK)
      return fail(CG_ERR_UNSUPPORTED, "D2Q9 supports periodic and bounce-back axes");
    if (p->solid_mask) return fail(CG_ERR_UNSUPPORTED, "D2Q9 takes no solid mask");
    if (p->model != CG_MODEL_D) return fail(CG_ERR_UNSUPPORTED, "D2Q9 implements the generalized equilibria (Model D) of App. A");
    if (p->precision != CG_F64 && p->precision != CG_F32) return fail(CG_ERR_UNSUPPORTED, "D2Q9 runs in FP64 or FP32");
  }
  return CG_OK;
}

Layout make_layout(const cg_params& p) {
  Layout L;
  L.n = (long long)p.nx * p.ny * p.nz;
  L.stride = (L.n + 63) / 64 * 64;
  L.elem = (p.precision == CG_F64) ? 8 : 4;
  L.pop_elem = (p.precision == CG_F64) ? 8 : (p.precision == CG_F32 ? 4 : 2);
  L.ns = (p.precision == CG_F16S || p.precision == CG_BF16S) ? 7 : 6;
  L.solid = needs_solid(p);
  L.nq = p.lattice == CG_D2Q9 ? 9 : 27;
  L.red_blocks = (int)std::min<long long>(1024, (L.n + RED_THREADS - 1) / RED_THREADS);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align_up(off + bytes);
    return at;
  };
  const size_t field = (size_t)L.stride * L.elem;
  // in place: one population buffer (and one wall buffer), named twice
  L.inplace = p.streaming == CG_STREAM_IN_PLACE;
  for (int b = 0; b < 2; ++b) L.f[b] = (b && L.inplace) ? L.f[0] : take(L.nq * (size_t)L.stride * L.pop_elem);
  for (int b = 0; b < 2; ++b) L.s[b] = take(L.ns * field);
  if (L.solid) {
    for (int b = 0; b < 2; ++b) L.aux[b] = (b && L.inplace) ? L.aux[0] : take(L.nq * field);
    L.mask = take((size_t)L.stride * 4);
  }
  // the fused collision pass (FP32, periodic, two buffers, 32-bit pulled
  // offsets) writes the next step's sums while the current ones are read
  L.fusable = p.lattice == CG_D3Q27 && p.precision == CG_F32 && !L.solid && !L.inplace &&
              8LL * L.stride + (long long)p.nx * p.ny < (1LL << 31);
  L.mac[0] = take(5 * field);
  L.mac[1] = L.fusable ? take(5 * field) : L.mac[0];
  L.phi = take(field);
  L.qc = take(3 * field);
  L.force = take(3 * field);
  L.wv = take(3 * field);
  L.partial = take((size_t)L.red_blocks * 2 * sizeof(double));
  L.flag = take(sizeof(unsigned int));
  L.result = take(2 * sizeof(double));
  L.diag = take(cg27_diag_bytes(L.red_blocks));
  L.total = off;
  return L;
}

dim3 block_of(const cg_params& p) {
  int bx = p.nx >= 128 ? 128 : (p.nx >= 64 ? 64 : 32);
  return dim3(bx, 128 / bx, 1);
}


dim3 grid_of(const cg_params& p, dim3 b) {
  return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz);
}

// The step graphs cut the domain into z slabs of `planes` planes whose tiles
// march `tz` planes (the schedule).  Thin slabs let the passes of
// neighbouring slabs overlap but repeat the z halo of the stencil passes at
// every tile start; thick ones do the opposite.  16 planes in tiles of 8
// measured best at 128^3 (among 16/24/32/48 planes and 4/8/12/16 per tile);
// at 512^3 the kernels fill the GPU on their own and the halo repeats cost
// more than the overlap gains.  So the first chained steps of a domain time
// the candidates below and keep the fastest (results do not depend on the
// schedule).  Graphs are used from SLAB_MIN_NZ planes on.
constexpr int SLAB_MIN_NZ = 32;
// steps chained in one graph (8: +6 % over one step per graph at 128^3,
// 16 gains 0.3 % more)
constexpr int GRAPH_STEPS = 8;
// chains of each candidate: one untimed, then TUNE_CHAINS timed
constexpr int TUNE_CHAINS = 2;

// candidate schedules of a domain with nz >= SLAB_MIN_NZ: thin slabs where the
// domain holds at least two, and whole-domain kernels with the domain's
// default depth, all with the four passes.  (The fused form is not among
// them: its recomputed ring and planes repeat the issue-bound collision --
// 1617 instructions per cell against 862 + 425 for the collision and the
// macroscopic pass -- and it measured 9.4 ms per 512^3 step against 8.0 for
// the two passes; cg_set_schedule_form still selects it.)
std::vector<StepSched> schedule_candidates(const cg_ctx* c) {
  std::vector<StepSched> v;
  const int nz = c->prm.nz;
  for (auto pt : {std::make_pair(16, 8), std::make_pair(32, 16), std::make_pair(64, 32)})
    if (nz >= 2 * pt.first) v.push_back({pt.first, pt.second, 0});
  v.push_back({nz, std::min(c->tz, nz), 0});
  return v;
}

void drop_graphs(cg_ctx* c) {
  for (auto& row : c->sgraph)
    for (cudaGraphExec_t& g : row)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
}

// switch the graph path to schedule sc; its graphs are built at the next step
void set_schedule(cg_ctx* c, const StepSched& sc) {
  if (c->sched_planes != sc.planes || c->sched_tz != sc.tz || c->sched_ftz != sc.ftz) drop_graphs(c);
  c->sched_planes = sc.planes;
  c->sched_tz = sc.tz;
  c->sched_ftz = sc.ftz;
}

// (re)start tuning: the candidates are timed by the next chained steps
void start_tuning(cg_ctx* c) {
  c->sched_cand = schedule_candidates(c);
  c->sched_timed.clear();
  c->tune_phase = 0;
  set_schedule(c, c->sched_cand.front());
  if (c->sched_cand.size() == 1) c->sched_cand.clear();  // nothing to choose
}

// the macroscopic pass and the collision of a step of stream mode sm
// (with two buffers and 8 stride + nx ny < 2^31, the form with 32-bit column
// offsets: 512^3 fits)
template <typename T, typename SF, bool SOLID>
void* macro_kernel(const cg_ctx* c, int sm) {
  if (sm == SM_EVEN) return (void*)k_macro<T, SF, SOLID, SM_EVEN>;
  if (sm == SM_ODD) return (void*)k_macro<T, SF, SOLID, SM_ODD>;
  if (8LL * c->L.stride + (long long)c->prm.nx * c->prm.ny < (1LL << 31))
    return (void*)k_macro<T, SF, SOLID, SM_AB, true>;
  return (void*)k_macro<T, SF, SOLID, SM_AB, false>;
}
template <typename T, typename SF, bool SOLID>
void* collide_kernel(int sm, bool unit) {
  if (sm == SM_EVEN)
    return unit ? (void*)k_collide<T, SF, SOLID, true, SM_EVEN> : (void*)k_collide<T, SF, SOLID, false, SM_EVEN>;
  if (sm == SM_ODD)
    return unit ? (void*)k_collide<T, SF, SOLID, true, SM_ODD> : (void*)k_collide<T, SF, SOLID, false, SM_ODD>;
  return unit ? (void*)k_collide<T, SF, SOLID, true, SM_AB> : (void*)k_collide<T, SF, SOLID, false, SM_AB>;
}

// block and grid of a z-marching pass with tiles of shape SH over `planes`
// planes in tiles of tz planes
template <class SH>
dim3 shape_block() { return dim3(SH::TX, SH::TY, 1); }
template <class SH>
dim3 shape_grid(const cg_ctx* c, int planes, int tz) {
  return dim3((c->prm.nx + SH::TX - 1) / SH::TX, (c->prm.ny + SH::TY - 1) / SH::TY, (planes + tz - 1) / tz);
}

// whether the steps of the domain take the fused collision pass now
template <typename T, typename SF, bool SOLID>
bool fused_now(const cg_ctx* c) {
  if constexpr (std::is_same<T, float>::value && std::is_same<SF, float>::value && !SOLID)
    return c->L.fusable && c->sched_ftz > 0;
  return false;
}

// the fused collision pass over planes zb <= z < ze in tiles of ftz planes
void* fused_kernel(const cg_ctx* c) {
  return c->unit ? (void*)k_collide_macro<true> : (void*)k_collide_macro<false>;
}
dim3 fused_grid(const cg_ctx* c, int planes, int ftz) {
  return dim3((c->prm.nx + FX - 1) / FX, (c->prm.ny + FY - 1) / FY, (planes + ftz - 1) / ftz);
}

// the macroscopic pass of the whole domain for the step that reads buffer
// `cur` (the first step of the fused form after anything else)
template <typename T, typename SF, bool SOLID>
void launch_macro(cg_ctx* c, int cur) {
  const Geom g = make_geom(c);
  int zb = 0, ze = c->prm.nz, tz = std::min(c->tz, ze);
  const Ptrs<T> P = make_ptrs<T>(c, cur);
  const Phys<T> ph = make_phys<T>(c->prm);
  void* args[] = {(void*)&g, (void*)&P, (void*)&ph, (void*)&tz, (void*)&zb, (void*)&ze};
  cudaLaunchKernel(macro_kernel<T, SF, SOLID>(c, next_mode(c->L.inplace, cur)), shape_grid<MacroShape>(c, ze, tz),
                   shape_block<MacroShape>(), args, 0, c->stream);
}

// One step of the whole domain as plain launches: the four passes, or with
// the fused form fields, div and the fused collision pass (preceded by the
// macroscopic pass when no fused step left this step's sums).
template <typename T, typename SF, bool SOLID>
void launch_passes(cg_ctx* c, int cur, cudaEvent_t* ev, int zb, int ze) {
  const Geom g = make_geom(c);
  const dim3 b(TX, TY, 1);
  const bool fused = fused_now<T, SF, SOLID>(c);
  const int tz = std::min(c->tz, ze - zb);
  const dim3 gr((c->prm.nx + TX - 1) / TX, (c->prm.ny + TY - 1) / TY, (ze - zb + tz - 1) / tz);
  const dim3 bc = block_of(c->prm);
  const dim3 gc((c->prm.nx + bc.x - 1) / bc.x, (c->prm.ny + bc.y - 1) / bc.y, ze - zb);
  const Ptrs<T> P = make_ptrs<T>(c, cur);
  const Phys<T> ph = make_phys<T>(c->prm);
  const int sm = next_mode(c->L.inplace, cur);
  if (ev) cudaEventRecord(ev[0], c->stream);
  if (!fused || c->mac_ready != c->steps) {
    int tz_ = tz;
    void* args[] = {(void*)&g, (void*)&P, (void*)&ph, (void*)&tz_, (void*)&zb, (void*)&ze};
    cudaLaunchKernel(macro_kernel<T, SF, SOLID>(c, sm), shape_grid<MacroShape>(c, ze - zb, tz),
                     shape_block<MacroShape>(), args, 0, c->stream);
  }
  if (ev) cudaEventRecord(ev[1], c->stream);
  if constexpr (!SOLID && sizeof(T) == 4)
    k_fields_sep<T><<<shape_grid<FieldShape>(c, ze - zb, tz), shape_block<FieldShape>(), 0, c->stream>>>(
        g, P, ph, tz, zb, ze);
  else
    k_fields<T, SOLID><<<gr, b, 0, c->stream>>>(g, P, ph, tz, zb, ze);
  if (ev) cudaEventRecord(ev[2], c->stream);
  k_div_sep<T><<<shape_grid<DivShape>(c, ze - zb, tz), dim3(32, DIV_THREADS / 32, 1), 0, c->stream>>>(
      g, P, tz, c->prm.use_Q, zb, ze);
  if (ev) cudaEventRecord(ev[3], c->stream);
  if (fused) {
    int ftz = std::min(c->sched_ftz, ze - zb);
    void* args[] = {(void*)&g, (void*)&P, (void*)&ph, (void*)&ftz, (void*)&zb, (void*)&ze};
    cudaLaunchKernel(fused_kernel(c), fused_grid(c, ze - zb, ftz), dim3(FNT, 1, 1), args, 0, c->stream);
    c->mac_ready = c->steps + 1;
  } else {
    void* args[] = {(void*)&g, (void*)&P, (void*)&ph, (void*)&zb};
    cudaLaunchKernel(collide_kernel<T, SF, SOLID>(sm, c->unit), gc, bc, args, 0, c->stream);
    c->mac_ready = -1;
  }
  if (ev) cudaEventRecord(ev[4], c->stream);
}

// Slab pipeline: the four passes of each z slab of SLAB_PLANES planes are
// graph nodes with their true dependencies -- fields(i) after macro(i-1..i+1)
// (phi with a two-plane halo), div(i) after fields(i-1..i+1), collide(i) after
// div(i) -- so the passes of different slabs overlap on the GPU (the
// issue-bound stencil passes with the bandwidth-bound population passes, and
// the tail of one pass with the head of the next).  `nsteps` consecutive steps
// go into one graph, chained by macro(t+1, i) after collide(t, i-1..i+1): that
// edge covers every cross-step hazard (the pulls of F and of the colour state
// from slabs i+-1, and the overwrites of mac, phi, force and the recoloring
// state that step t still reads), so the start of a step overlaps the end of
// the previous one.  Results do not depend on the slabs or the chaining.
// The fused form has three passes per slab: fields(i) after fused(t-1,
// i-1..i+1) (it writes mac and phi of step t), div(i) after fields(i-1..i+1),
// fused(i) after div(i-1..i+1) (its ring planes read F and Q of the slabs
// beside it); the same edges cover the cross-step hazards, and the graph
// assumes that the step before it left its sums (mac_ready).
template <typename T, typename SF, bool SOLID>
cudaGraphExec_t build_slab_graph(cg_ctx* c, int cur0, int nsteps) {
  const int slab = c->sched_planes;
  const int nz = c->prm.nz, ns = (nz + slab - 1) / slab;
  const Geom g = make_geom(c);
  const Ptrs<T> P[2] = {make_ptrs<T>(c, 0), make_ptrs<T>(c, 1)};
  const Phys<T> ph = make_phys<T>(c->prm);
  cudaGraph_t gph;
  if (cudaGraphCreate(&gph, 0) != cudaSuccess) return nullptr;
  std::vector<cudaGraphNode_t> M(ns), F(ns), D(ns), C(ns), Cprev;
  const dim3 b(TX, TY, 1);
  const dim3 bc = block_of(c->prm);
  int use_Q = c->prm.use_Q;
  bool ok = true;
  auto deps3 = [&](const std::vector<cudaGraphNode_t>& v, int i, std::vector<cudaGraphNode_t>& out) {
    out.clear();
    for (int d = -1; d <= 1; ++d) {
      cudaGraphNode_t n = v[(i + d + ns) % ns];
      if (std::find(out.begin(), out.end(), n) == out.end()) out.push_back(n);
    }
  };
  std::vector<int> zb(ns), ze(ns), tzs(ns);
  for (int i = 0; i < ns; ++i) {
    zb[i] = i * slab;
    ze[i] = std::min(nz, zb[i] + slab);
    tzs[i] = std::min(c->sched_tz, ze[i] - zb[i]);
  }
  auto add = [&](cudaGraphNode_t* node, void* func, dim3 gr, dim3 blk, void** args,
                 const std::vector<cudaGraphNode_t>& dv) {
    cudaKernelNodeParams kp = {};
    kp.func = func;
    kp.gridDim = gr;
    kp.blockDim = blk;
    kp.kernelParams = args;
    if (cudaGraphAddKernelNode(node, gph, dv.empty() ? nullptr : dv.data(), dv.size(), &kp) != cudaSuccess)
      ok = false;
  };
  std::vector<cudaGraphNode_t> dv;
  const bool fused = fused_now<T, SF, SOLID>(c);
  std::vector<int> ftz(ns);
  for (int i = 0; i < ns; ++i) ftz[i] = std::min(c->sched_ftz, ze[i] - zb[i]);
  for (int s = 0; s < nsteps && ok; ++s) {
    const Ptrs<T>& Pc = P[(cur0 + s) & 1];
    const int sm = next_mode(c->L.inplace, cur0 + s);
    for (int i = 0; i < ns && !fused; ++i) {
      const dim3 gr((c->prm.nx + TX - 1) / TX, (c->prm.ny + TY - 1) / TY, (ze[i] - zb[i] + tzs[i] - 1) / tzs[i]);
      void* args[] = {(void*)&g, (void*)&Pc, (void*)&ph, (void*)&tzs[i], (void*)&zb[i], (void*)&ze[i]};
      if (s > 0) deps3(Cprev, i, dv); else dv.clear();
      add(&M[i], macro_kernel<T, SF, SOLID>(c, sm), shape_grid<MacroShape>(c, ze[i] - zb[i], tzs[i]),
          shape_block<MacroShape>(), args, dv);
    }
    for (int i = 0; i < ns; ++i) {
      const dim3 gr((c->prm.nx + TX - 1) / TX, (c->prm.ny + TY - 1) / TY, (ze[i] - zb[i] + tzs[i] - 1) / tzs[i]);
      void* args[] = {(void*)&g, (void*)&Pc, (void*)&ph, (void*)&tzs[i], (void*)&zb[i], (void*)&ze[i]};
      void* fn;
      dim3 grf = gr, bf = b;
      if constexpr (!SOLID && sizeof(T) == 4) {
        fn = (void*)k_fields_sep<T>;
        grf = shape_grid<FieldShape>(c, ze[i] - zb[i], tzs[i]);
        bf = shape_block<FieldShape>();
      } else {
        fn = (void*)k_fields<T, SOLID>;
      }
      if (!fused) deps3(M, i, dv);
      else if (s > 0) deps3(Cprev, i, dv);
      else dv.clear();
      add(&F[i], fn, grf, bf, args, dv);
    }
    for (int i = 0; i < ns; ++i) {
      const dim3 gr((c->prm.nx + TX - 1) / TX, (c->prm.ny + TY - 1) / TY, (ze[i] - zb[i] + tzs[i] - 1) / tzs[i]);
      void* args[] = {(void*)&g, (void*)&Pc, (void*)&tzs[i], (void*)&use_Q, (void*)&zb[i], (void*)&ze[i]};
      deps3(F, i, dv);
      add(&D[i], (void*)k_div_sep<T>, shape_grid<DivShape>(c, ze[i] - zb[i], tzs[i]), dim3(32, DIV_THREADS / 32, 1),
          args, dv);
    }
    for (int i = 0; i < ns; ++i) {
      if (fused) {
        void* args[] = {(void*)&g, (void*)&Pc, (void*)&ph, (void*)&ftz[i], (void*)&zb[i], (void*)&ze[i]};
        deps3(D, i, dv);
        add(&C[i], fused_kernel(c), fused_grid(c, ze[i] - zb[i], ftz[i]), dim3(FNT, 1, 1), args, dv);
        continue;
      }
      const dim3 gc((c->prm.nx + bc.x - 1) / bc.x, (c->prm.ny + bc.y - 1) / bc.y, ze[i] - zb[i]);
      void* args[] = {(void*)&g, (void*)&Pc, (void*)&ph, (void*)&zb[i]};
      dv.assign(1, D[i]);
      add(&C[i], collide_kernel<T, SF, SOLID>(sm, c->unit), gc, bc, args, dv);
    }
    Cprev = C;
  }
  cudaGraphExec_t ex = nullptr;
  if (!ok || cudaGraphInstantiate(&ex, gph, 0) != cudaSuccess) ex = nullptr;
  cudaGraphDestroy(gph);
  return ex;
}

// One step of the tuning of the schedule when a chain is launched: an untimed
// chain of the current candidate, then TUNE_CHAINS chains between two events
// (waiting for them); after the last candidate the fastest is kept.
// Returns false when the chain could not be launched.
bool launch_chain_tuned(cg_ctx* c, cudaGraphExec_t gx) {
  if (c->sched_cand.empty()) return cudaGraphLaunch(gx, c->stream) == cudaSuccess;
  if (!c->tev[0]) {
    if (cudaEventCreate(&c->tev[0]) != cudaSuccess || cudaEventCreate(&c->tev[1]) != cudaSuccess) return false;
  }
  if (c->tune_phase == 1) cudaEventRecord(c->tev[0], c->stream);
  if (cudaGraphLaunch(gx, c->stream) != cudaSuccess) return false;
  if (c->tune_phase == 0) {
    c->tune_phase = 1;
    return true;
  }
  if (++c->tune_phase <= TUNE_CHAINS) return true;  // more chains of this candidate
  cudaEventRecord(c->tev[1], c->stream);
  if (cudaEventSynchronize(c->tev[1]) != cudaSuccess) return false;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->tev[0], c->tev[1]);
  c->sched_timed.push_back({ms, c->sched_cand.front()});
  c->sched_cand.erase(c->sched_cand.begin());
  c->tune_phase = 0;
  if (!c->sched_cand.empty()) {
    set_schedule(c, c->sched_cand.front());
  } else {
    const auto best = std::min_element(c->sched_timed.begin(), c->sched_timed.end());
    set_schedule(c, best->second);
  }
  return true;
}

// Enqueues up to `remaining` steps (at least one) and returns how many.
template <typename T, typename SF, bool SOLID>
int enqueue_steps(cg_ctx* c, int64_t remaining) {
  const int cur = (int)(c->steps & 1);
  cudaEvent_t* ev = nullptr;
  if (c->prof_used < c->prof_capacity) ev = &c->events[NUM_EVENTS_PER_STEP * c->prof_used++];
  // the step graphs when the domain has at least SLAB_MIN_NZ planes, no
  // per-pass timing is requested and the stream is not being captured
  if (!ev && c->prm.nz >= SLAB_MIN_NZ && c->graphs_ok) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      if (c->sched_planes == 0) start_tuning(c);
      // all four graphs of the schedule (one step and a chain, both parities)
      // at its first use, so that no later call pays for an instantiation
      for (int kk = 0; kk < 2; ++kk)
        for (int par = 0; par < 2; ++par)
          if (!c->sgraph[kk][par]) c->sgraph[kk][par] = build_slab_graph<T, SF, SOLID>(c, par, kk ? GRAPH_STEPS : 1);
      const int k = remaining >= GRAPH_STEPS ? 1 : 0;
      const int n = k ? GRAPH_STEPS : 1;
      // a single step inside a timed window would falsify it: time again
      if (!k && !c->sched_cand.empty() && c->tune_phase > 1) c->tune_phase = 1;
      cudaGraphExec_t gx = c->sgraph[k][cur];
      const bool fused = fused_now<T, SF, SOLID>(c);
      // the fused graphs start from the sums that the step before left
      if (gx && fused && c->mac_ready != c->steps) launch_macro<T, SF, SOLID>(c, cur);
      if (gx && (k ? launch_chain_tuned(c, gx) : cudaGraphLaunch(gx, c->stream) == cudaSuccess)) {
        c->mac_ready = fused ? c->steps + n : -1;
        return n;
      }
      (void)cudaGetLastError();
      c->graphs_ok = false;  // graphs unavailable here: plain launches from now on
    }
  }
  launch_passes<T, SF, SOLID>(c, cur, ev, 0, c->prm.nz);
  return 1;
}

// one D2Q9 step: five per-cell kernels (the normal and force kernels are
// timed together as the field pass)
template <typename T, bool SOLID>
void enqueue_step2(cg_ctx* c) {
  const int cur = (int)(c->steps & 1);
  const Geom g = make_geom(c);
  const dim3 b = block_of(c->prm), gr = grid_of(c->prm, b);
  const Ptrs<T> P = make_ptrs<T>(c, cur);
  const Phys<T> ph = make_phys<T>(c->prm);
  cudaEvent_t* ev = nullptr;
  if (c->prof_used < c->prof_capacity) ev = &c->events[NUM_EVENTS_PER_STEP * c->prof_used++];
  if (ev) cudaEventRecord(ev[0], c->stream);
  k2_macro<T, SOLID><<<gr, b, 0, c->stream>>>(g, P, ph);
  if (ev) cudaEventRecord(ev[1], c->stream);
  k2_normal<T, SOLID><<<gr, b, 0, c->stream>>>(g, P);
  k2_force<T, SOLID><<<gr, b, 0, c->stream>>>(g, P, ph);
  if (ev) cudaEventRecord(ev[2], c->stream);
  k2_qcorr<T, SOLID><<<gr, b, 0, c->stream>>>(g, P, c->prm.use_Q);
  if (ev) cudaEventRecord(ev[3], c->stream);
  k2_collide<T, SOLID><<<gr, b, 0, c->stream>>>(g, P, ph);
  if (ev) cudaEventRecord(ev[4], c->stream);
}

int enqueue_step_any(cg_ctx* c, int64_t remaining) {
  if (c->prm.lattice == CG_D2Q9) {
    if (c->prm.precision == CG_F64) {
      if (c->L.solid) enqueue_step2<double, true>(c); else enqueue_step2<double, false>(c);
    } else {
      if (c->L.solid) enqueue_step2<float, true>(c); else enqueue_step2<float, false>(c);
    }
    return 1;
  }
  switch (c->prm.precision) {
    case CG_F64:
      return c->L.solid ? enqueue_steps<double, double, true>(c, remaining)
                        : enqueue_steps<double, double, false>(c, remaining);
    case CG_F32:
      return c->L.solid ? enqueue_steps<float, float, true>(c, remaining)
                        : enqueue_steps<float, float, false>(c, remaining);
    case CG_F16S: return enqueue_steps<float, __half, false>(c, remaining);
    default: return enqueue_steps<float, __nv_bfloat16, false>(c, remaining);
  }
}

// The first cell whose densities are not finite and >= 0, or -1: the host
// arrays are scanned in parallel slices (one per hardware thread, at most 32),
// so that a 512^3 upload does not wait for one core to read 2 GB.
long long first_invalid_density(const double* rr, const double* rb, long long n) {
  auto scan = [rr, rb](long long lo, long long hi) -> long long {
    for (long long i = lo; i < hi; ++i)
      if (!(std::isfinite(rr[i]) && std::isfinite(rb[i]) && rr[i] >= 0 && rb[i] >= 0)) return i;
    return -1;
  };
  const int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < (1LL << 20) || nt == 1) return scan(0, n);
  std::vector<long long> found(nt, -1);
  std::vector<std::thread> pool;
  const long long per = (n + nt - 1) / nt;
  for (int t = 0; t < nt; ++t)
    pool.emplace_back([&, t] { found[t] = scan(std::min(n, t * per), std::min(n, (t + 1) * per)); });
  for (std::thread& th : pool) th.join();
  for (long long f : found)
    if (f >= 0) return f;  // slices are in cell order: the first hit is the first invalid cell
  return -1;
}

// Device memory free between steps, for staging host transfers: the
// population buffer the next step writes, or with in-place streaming the
// recoloring-state buffer the next step writes.  Transfers go through it in
// chunks of cells, so it may be smaller than what a whole transfer needs.
struct Stage {
  char* p;
  size_t bytes;
};
Stage stage_of(const cg_ctx* c) {
  const Layout& L = c->L;
  const int spare = 1 - (int)(c->steps & 1);
  if (L.inplace) return {c->ws + L.s[spare], L.ns * (size_t)L.stride * L.elem};
  return {c->ws + L.f[spare], L.nq * (size_t)L.stride * L.pop_elem};
}
// cells per chunk when each cell needs `per_cell` bytes of staging
long long chunk_cells(const Stage& st, size_t per_cell) {
  return std::max<long long>(1, (long long)(st.bytes / per_cell));
}

template <typename T, bool SOLID>
void enqueue_init2(cg_ctx* c, const double* d_in, long long lo, long long hi) {
  const Geom g = make_geom(c);
  const dim3 b = block_of(c->prm), gr = grid_of(c->prm, b);
  Ptrs<T> P = make_ptrs<T>(c, 1);  // the initial state goes to buffer 0
  k2_init<T, SOLID><<<gr, b, 0, c->stream>>>(g, P, make_phys<T>(c->prm), d_in, lo, hi);
  if (hi < c->L.n) return;  // walls once every fluid cell is in place
  if constexpr (SOLID) {
    Ptrs<T> W = make_ptrs<T>(c, 0);
    W.f_out = const_cast<void*>(W.f_in);
    W.aux_out = const_cast<T*>(W.aux_in);
    k2_init_walls<T><<<gr, b, 0, c->stream>>>(g, W);
  }
}

template <typename T, typename SF, bool SOLID>
void enqueue_init(cg_ctx* c, const double* d_in, long long lo, long long hi) {
  const Geom g = make_geom(c);
  const dim3 b = block_of(c->prm), gr = grid_of(c->prm, b);
  // the initial state is written to buffer 0 (read by the first step)
  Ptrs<T> P = make_ptrs<T>(c, 1);
  // laid out as if an odd step had written it (in place) or in buffer 0
  k_init<T, SF, SOLID><<<gr, b, 0, c->stream>>>(g, P, make_phys<T>(c->prm), d_in, lo, hi,
                                                last_mode(c->L.inplace, 0));
  if (hi < c->L.n) return;  // walls once every fluid cell is in place
  if constexpr (SOLID) {
    // walls from the fluid cells of the same buffer (read fluid, write solid)
    Ptrs<T> W = make_ptrs<T>(c, 0);
    W.f_out = const_cast<void*>(W.f_in);
    W.aux_out = const_cast<T*>(W.aux_in);
    W.mac = P.mac;
    k_init_walls<T, SF><<<gr, b, 0, c->stream>>>(g, W, make_phys<T>(c->prm), next_mode(c->L.inplace, 0),
                                                 last_mode(c->L.inplace, 0));
  }
}

}  // namespace

// ---- solid flags (non-template kernels) -------------------------------------------

namespace cg27 {
__global__ void k_solid_self(Geom g, uint8_t* solid, int has_user, int bx, int by, int bz) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= g.nx || y >= g.ny) return;
  const int i = x + g.nx * y + g.nxy * z;
  uint8_t s = has_user ? (solid[i] != 0) : 0;
  if (bx && (x == 0 || x == g.nx - 1)) s = 1;
  if (by && (y == 0 || y == g.ny - 1)) s = 1;
  if (bz && (z == 0 || z == g.nz - 1)) s = 1;
  solid[i] = s;
}

__global__ void k2_solid_mask(Geom g, const uint8_t* solid, uint32_t* mask) {
  Cell2 c;
  if (!make_cell2(g, c)) return;
  uint32_t m = solid[c.idx] ? (1u << SELF_SOLID_BIT) : 0u;
  for (int q = 0; q < 9; ++q)
    if (solid[nbr2(c, CX2(q), CY2(q))]) m |= (1u << q);
  mask[c.idx] = m;
}

__global__ void k_solid_mask(Geom g, const uint8_t* solid, uint32_t* mask) {
  Cell c;
  if (!make_cell(g, c)) return;
  uint32_t m = solid[c.idx] ? (1u << SELF_SOLID_BIT) : 0u;
#pragma unroll
  for (int q = 0; q < 27; ++q)
    if (solid[nbr(c, CX(q), CY(q), CZ(q))]) m |= (1u << q);
  mask[c.idx] = m;
}

__global__ void k_mass_final(const double* partial, int nblocks, double* out) {
  __shared__ double sr[256], sb[256];
  double ar = 0.0, ab = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
    ar += partial[2 * i];
    ab += partial[2 * i + 1];
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
    out[0] = sr[0];
    out[1] = sb[0];
  }
}
}  // namespace cg27

// error recording shared with the other translation units of the library
__attribute__((visibility("hidden"))) int cg27_internal_fail(int code, const char* msg) {
  return fail(code, msg);
}

// ---- C ABI --------------------------------------------------------------------------

extern "C" {

int cg_abi_version(void) { return CG27_ABI_VERSION; }

const char* cg_last_error(void) { return g_err.c_str(); }

int cg_params_default(cg_params* p, int32_t nx, int32_t ny, int32_t nz) {
  if (!p) return fail(CG_ERR_INVALID_ARG, "params is NULL");
  std::memset(p, 0, sizeof(*p));
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->rho_r0 = p->rho_b0 = 1.0;
  p->alpha_r = p->alpha_b = 8.0 / 27.0;
  p->nu_r = p->nu_b = 0.1;
  p->sigma = 0.0;
  p->beta = 0.7;
  for (int q = 0; q < 11; ++q) p->omega[q] = 1.0;
  p->force_mode = CG_FORCE_NONE;
  p->model = CG_MODEL_D;
  p->use_Q = 1;
  p->precision = CG_F32;
  return CG_OK;
}

int cg_workspace_bytes(const cg_params* p, size_t* bytes) {
  int rc = validate(p);
  if (rc) return rc;
  if (!bytes) return fail(CG_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = make_layout(*p).total;
  return CG_OK;
}

int cg_create(const cg_params* p, void* d_workspace, size_t bytes, void* cuda_stream, cg_ctx** out) {
  int rc = validate(p);
  if (rc) return rc;
  if (!out) return fail(CG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  Layout L = make_layout(*p);
  if (!d_workspace) return fail(CG_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(d_workspace) % ALIGN != 0)
    return fail(CG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < L.total)
    return fail(CG_ERR_WORKSPACE, "workspace too small: need " + std::to_string(L.total) + " bytes");
  cudaPointerAttributes attr;
  CG_CUDA(cudaPointerGetAttributes(&attr, d_workspace));
  if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
    return fail(CG_ERR_WORKSPACE, "workspace is not device memory");
  cg_ctx* c = new cg_ctx;
  c->prm = *p;
  c->L = L;
  c->ws = static_cast<char*>(d_workspace);
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  bool unit = (p->model == CG_MODEL_D);
  for (int q = 0; q < 11; ++q)
    if (q != 1 && p->omega[q] != 1.0) unit = false;
  c->unit = unit;
  // z planes per tile: enough tiles for about eight per SM
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles_xy = (long long)((p->nx + TX - 1) / TX) * ((p->ny + TY - 1) / TY);
  const long long chunks = std::max(1LL, std::min<long long>(p->nz, (8LL * sms + tiles_xy - 1) / tiles_xy));
  c->tz = (int)((p->nz + chunks - 1) / chunks);
  *out = c;
  return CG_OK;
}

int cg_destroy(cg_ctx* c) {
  if (c && c->batch) return fail(CG_ERR_INVALID_ARG, "the domain is a member of a batch: remove it first");
  delete c;
  return CG_OK;
}

int cg_init_fields(cg_ctx* c, const double* rho_r, const double* rho_b, const double* u,
                   const uint8_t* solid) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (c->batch) return fail(CG_ERR_INVALID_ARG, "the domain is a member of a batch: remove it first");
  if (!rho_r || !rho_b || !u) return fail(CG_ERR_INVALID_ARG, "rho_r, rho_b, u must be non-NULL");
  if (solid && !c->L.solid)
    return fail(CG_ERR_INVALID_ARG, "a solid mask needs params.solid_mask = 1 or a bounce-back axis");
  const long long n = c->L.n;
  const long long bad = first_invalid_density(rho_r, rho_b, n);
  if (bad >= 0)
    return fail(CG_ERR_INVALID_ARG, "densities must be finite and >= 0 (cell " + std::to_string(bad) + ")");
  c->steps = 0;  // the state goes to buffer 0, the staging to buffer 1
  c->mac_ready = -1;
  const Stage st = stage_of(c);
  double* d_in = reinterpret_cast<double*>(st.p);
  const Geom g = make_geom(c);
  const dim3 b = block_of(c->prm), gr = grid_of(c->prm, b);
  if (c->L.solid) {
    // the solid flags are staged in the phi field, which the init kernels
    // write only after the neighbour mask has been built
    uint8_t* d_solid = reinterpret_cast<uint8_t*>(c->ws + c->L.phi);
    if (solid)
      CG_CUDA(cudaMemcpyAsync(d_solid, solid, (size_t)n, cudaMemcpyHostToDevice, c->stream));
    k_solid_self<<<gr, b, 0, c->stream>>>(g, d_solid, solid ? 1 : 0, c->prm.bc[0] != CG_BC_PERIODIC,
                                          c->prm.bc[1] != CG_BC_PERIODIC, c->prm.bc[2] != CG_BC_PERIODIC);
    if (c->prm.lattice == CG_D2Q9)
      k2_solid_mask<<<gr, b, 0, c->stream>>>(g, d_solid, reinterpret_cast<uint32_t*>(c->ws + c->L.mask));
    else
      k_solid_mask<<<gr, b, 0, c->stream>>>(g, d_solid, reinterpret_cast<uint32_t*>(c->ws + c->L.mask));
  }
  // chunks of cells: rho_r, rho_b, u_x, u_y, u_z of each chunk staged together
  const long long chunk = chunk_cells(st, 5 * sizeof(double));
  for (long long lo = 0; lo < n; lo += chunk) {
    const long long hi = std::min(n, lo + chunk), m = hi - lo;
    const size_t mb = (size_t)m * sizeof(double);
    const double* src[5] = {rho_r + lo, rho_b + lo, u + lo, u + n + lo, u + 2 * n + lo};
    for (int a = 0; a < 5; ++a)
      CG_CUDA(cudaMemcpyAsync(d_in + a * m, src[a], mb, cudaMemcpyHostToDevice, c->stream));
    if (c->prm.lattice == CG_D2Q9) {
      if (c->prm.precision == CG_F64) {
        if (c->L.solid) enqueue_init2<double, true>(c, d_in, lo, hi); else enqueue_init2<double, false>(c, d_in, lo, hi);
      } else {
        if (c->L.solid) enqueue_init2<float, true>(c, d_in, lo, hi); else enqueue_init2<float, false>(c, d_in, lo, hi);
      }
    } else
    switch (c->prm.precision) {
      case CG_F64:
        if (c->L.solid) enqueue_init<double, double, true>(c, d_in, lo, hi);
        else enqueue_init<double, double, false>(c, d_in, lo, hi);
        break;
      case CG_F32:
        if (c->L.solid) enqueue_init<float, float, true>(c, d_in, lo, hi);
        else enqueue_init<float, float, false>(c, d_in, lo, hi);
        break;
      case CG_F16S: enqueue_init<float, __half, false>(c, d_in, lo, hi); break;
      default: enqueue_init<float, __nv_bfloat16, false>(c, d_in, lo, hi); break;
    }
  }
  CG_CUDA(cudaMemsetAsync(c->ws + c->L.flag, 0, sizeof(unsigned int), c->stream));
  CG_CUDA(cudaGetLastError());
  // the host arrays may be pageable and reused by the caller: finish the copies
  CG_CUDA(cudaStreamSynchronize(c->stream));
  c->initialised = true;
  return CG_OK;
}

int cg_step(cg_ctx* c, int64_t nsteps) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (c->batch) return fail(CG_ERR_INVALID_ARG, "the domain is a member of a batch: remove it first");
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  if (nsteps < 0) return fail(CG_ERR_INVALID_ARG, "nsteps must be >= 0");
  for (int64_t s = 0; s < nsteps;) {
    const int n = enqueue_step_any(c, nsteps - s);
    c->steps += n;
    s += n;
  }
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

int cg_read_macros(cg_ctx* c, double* rho_r, double* rho_b, double* u, double* p, double* phi) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (int rc_ = settle(c)) return rc_;
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  const long long n = c->L.n;
  const Stage st = stage_of(c);
  double* d_out = reinterpret_cast<double*>(st.p);
  const Geom g = make_geom(c);
  const dim3 b = block_of(c->prm), gr = grid_of(c->prm, b);
  // chunks of cells, the seven fields of each chunk staged together
  const long long chunk = chunk_cells(st, 7 * sizeof(double));
  for (long long lo = 0; lo < n; lo += chunk) {
    const long long hi = std::min(n, lo + chunk), m = hi - lo;
    if (c->prm.precision == CG_F64) {
      auto P = state_ptrs<double>(c);
      if (c->L.solid)
        k_read_macros<double, true><<<gr, b, 0, c->stream>>>(g, P, make_phys<double>(c->prm), d_out, lo, hi);
      else
        k_read_macros<double, false><<<gr, b, 0, c->stream>>>(g, P, make_phys<double>(c->prm), d_out, lo, hi);
    } else {
      auto P = state_ptrs<float>(c);
      if (c->L.solid)
        k_read_macros<float, true><<<gr, b, 0, c->stream>>>(g, P, make_phys<float>(c->prm), d_out, lo, hi);
      else
        k_read_macros<float, false><<<gr, b, 0, c->stream>>>(g, P, make_phys<float>(c->prm), d_out, lo, hi);
    }
    CG_CUDA(cudaGetLastError());
    const size_t mb = (size_t)m * sizeof(double);
    double* dst[7] = {rho_r ? rho_r + lo : nullptr, rho_b ? rho_b + lo : nullptr,
                      u ? u + lo : nullptr,         u ? u + n + lo : nullptr,
                      u ? u + 2 * n + lo : nullptr, p ? p + lo : nullptr,
                      phi ? phi + lo : nullptr};
    for (int a = 0; a < 7; ++a)
      if (dst[a]) CG_CUDA(cudaMemcpyAsync(dst[a], d_out + a * m, mb, cudaMemcpyDeviceToHost, c->stream));
  }
  CG_CUDA(cudaStreamSynchronize(c->stream));
  return CG_OK;
}

int cg_read_populations(cg_ctx* c, double* fr, double* fb) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (int rc_ = settle(c)) return rc_;
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  const long long n = c->L.n;
  const Stage st = stage_of(c);
  double* d_out = reinterpret_cast<double*>(st.p);
  const Geom g = make_geom(c);
  const dim3 b = block_of(c->prm), gr = grid_of(c->prm, b);
  // the current state sits in buffer `cur`: read it through the "input" pointers
  const int cur = (int)(c->steps & 1);
  const long long chunk = chunk_cells(st, 2 * sizeof(double));
  const int sm = last_mode(c->L.inplace, c->steps);  // where the last step left the populations
  for (int i = 0; i < c->L.nq; ++i)
  for (long long lo = 0; lo < n; lo += chunk) {
    const long long hi = std::min(n, lo + chunk), m = hi - lo;
    const size_t mb = (size_t)m * sizeof(double);
    if (c->prm.lattice == CG_D2Q9) {
      const int q = paper_to_lex2(i);
      if (c->prm.precision == CG_F64) {
        auto P = make_ptrs<double>(c, cur);
        if (c->L.solid) k2_read_pop<double, true><<<gr, b, 0, c->stream>>>(g, P, q, d_out, d_out + m, lo, hi);
        else k2_read_pop<double, false><<<gr, b, 0, c->stream>>>(g, P, q, d_out, d_out + m, lo, hi);
      } else {
        auto P = make_ptrs<float>(c, cur);
        if (c->L.solid) k2_read_pop<float, true><<<gr, b, 0, c->stream>>>(g, P, q, d_out, d_out + m, lo, hi);
        else k2_read_pop<float, false><<<gr, b, 0, c->stream>>>(g, P, q, d_out, d_out + m, lo, hi);
      }
    } else if (c->prm.precision == CG_F64) {
      const int q = paper_to_lex(i);
      auto P = make_ptrs<double>(c, cur);
      if (c->L.solid) k_read_pop<double, double, true><<<gr, b, 0, c->stream>>>(g, P, make_phys<double>(c->prm), q, d_out, d_out + m, lo, hi, sm);
      else k_read_pop<double, double, false><<<gr, b, 0, c->stream>>>(g, P, make_phys<double>(c->prm), q, d_out, d_out + m, lo, hi, sm);
    } else {
      const int q = paper_to_lex(i);
      auto P = make_ptrs<float>(c, cur);
      if (c->prm.precision == CG_F16S)
        k_read_pop<float, __half, false><<<gr, b, 0, c->stream>>>(g, P, make_phys<float>(c->prm), q, d_out, d_out + m, lo, hi, sm);
      else if (c->prm.precision == CG_BF16S)
        k_read_pop<float, __nv_bfloat16, false><<<gr, b, 0, c->stream>>>(g, P, make_phys<float>(c->prm), q, d_out, d_out + m, lo, hi, sm);
      else if (c->L.solid)
        k_read_pop<float, float, true><<<gr, b, 0, c->stream>>>(g, P, make_phys<float>(c->prm), q, d_out, d_out + m, lo, hi, sm);
      else
        k_read_pop<float, float, false><<<gr, b, 0, c->stream>>>(g, P, make_phys<float>(c->prm), q, d_out, d_out + m, lo, hi, sm);
    }
    CG_CUDA(cudaGetLastError());
    if (fr) CG_CUDA(cudaMemcpyAsync(fr + (size_t)i * n + lo, d_out, mb, cudaMemcpyDeviceToHost, c->stream));
    if (fb) CG_CUDA(cudaMemcpyAsync(fb + (size_t)i * n + lo, d_out + m, mb, cudaMemcpyDeviceToHost, c->stream));
  }
  CG_CUDA(cudaStreamSynchronize(c->stream));
  return CG_OK;
}

int cg_reduce(cg_ctx* c, double out_mass[2], int32_t* nonfinite) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (int rc_ = settle(c)) return rc_;
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  const Geom g = make_geom(c);
  double* partial = reinterpret_cast<double*>(c->ws + c->L.partial);
  double* result = reinterpret_cast<double*>(c->ws + c->L.result);
  if (c->prm.precision == CG_F64)
    k_mass_partial<double><<<c->L.red_blocks, RED_THREADS, 0, c->stream>>>(
        g, reinterpret_cast<const double*>(c->ws + mac_last(c)), c->L.n, partial);
  else
    k_mass_partial<float><<<c->L.red_blocks, RED_THREADS, 0, c->stream>>>(
        g, reinterpret_cast<const float*>(c->ws + mac_last(c)), c->L.n, partial);
  k_mass_final<<<1, RED_THREADS, 0, c->stream>>>(partial, c->L.red_blocks, result);
  CG_CUDA(cudaGetLastError());
  double m[2];
  unsigned int flag = 0;
  CG_CUDA(cudaMemcpyAsync(m, result, sizeof(m), cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(cudaMemcpyAsync(&flag, c->ws + c->L.flag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
  CG_CUDA(cudaStreamSynchronize(c->stream));
  if (out_mass) {
    out_mass[0] = m[0];
    out_mass[1] = m[1];
  }
  if (nonfinite) *nonfinite = flag ? 1 : 0;
  return CG_OK;
}

int cg_profile_enable(cg_ctx* c, int64_t max_steps) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (max_steps < 0 || max_steps > (1 << 20)) return fail(CG_ERR_INVALID_ARG, "max_steps out of range");
  CG_CUDA(cudaStreamSynchronize(c->stream));
  while ((int64_t)c->events.size() < NUM_EVENTS_PER_STEP * max_steps) {
    cudaEvent_t e;
    CG_CUDA(cudaEventCreate(&e));
    c->events.push_back(e);
  }
  c->prof_capacity = max_steps;
  c->prof_used = 0;
  return CG_OK;
}

int cg_profile_read(cg_ctx* c, double ms[CG_NUM_PASSES], int64_t* steps) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  CG_CUDA(cudaStreamSynchronize(c->stream));
  double acc[CG_NUM_PASSES] = {0};
  for (int64_t s = 0; s < c->prof_used; ++s)
    for (int k = 0; k < CG_NUM_PASSES; ++k) {
      float t = 0.f;
      CG_CUDA(cudaEventElapsedTime(&t, c->events[NUM_EVENTS_PER_STEP * s + k],
                                   c->events[NUM_EVENTS_PER_STEP * s + k + 1]));
      acc[k] += t;
    }
  if (ms)
    for (int k = 0; k < CG_NUM_PASSES; ++k) ms[k] = acc[k];
  if (steps) *steps = c->prof_used;
  return CG_OK;
}

int cg_set_schedule_form(cg_ctx* c, int32_t planes, int32_t tz, int32_t fused_tz) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (c->batch) return fail(CG_ERR_INVALID_ARG, "the domain is a member of a batch: remove it first");
  if (planes == 0 && tz == 0 && fused_tz == 0) {
    CG_CUDA(cudaStreamSynchronize(c->stream));  // graphs of the old schedule may be in flight
    c->sched_planes = 0;  // tune again at the next graph step
    c->sched_ftz = 0;
    drop_graphs(c);
    return CG_OK;
  }
  if (planes < 1 || planes > c->prm.nz || tz < 1 || tz > planes || fused_tz < 0 || fused_tz > planes)
    return fail(CG_ERR_INVALID_ARG,
                "need 1 <= planes <= nz, 1 <= tz <= planes and 0 <= fused_tz <= planes (or all 0)");
  if (fused_tz > 0 && !c->L.fusable)
    return fail(CG_ERR_UNSUPPORTED, "the fused collision pass needs FP32, two buffers, no walls and a D3Q27 "
                                    "domain with 8 * stride + nx * ny < 2^31");
  CG_CUDA(cudaStreamSynchronize(c->stream));  // graphs of the old schedule may be in flight
  c->sched_cand.clear();
  c->sched_timed.clear();
  set_schedule(c, StepSched{planes, tz, fused_tz});
  return CG_OK;
}

int cg_set_schedule(cg_ctx* c, int32_t planes, int32_t tz) { return cg_set_schedule_form(c, planes, tz, 0); }

int cg_schedule_form(cg_ctx* c, int32_t* planes, int32_t* tz, int32_t* fused_tz, int32_t* tuning) {
  if (!c) return fail(CG_ERR_INVALID_ARG, "ctx is NULL");
  if (planes) *planes = c->sched_planes;
  if (tz) *tz = c->sched_tz;
  if (fused_tz) *fused_tz = c->sched_ftz;
  if (tuning)
    *tuning = c->graphs_ok && c->prm.lattice == CG_D3Q27 &&
              ((c->sched_planes == 0 && c->prm.nz >= SLAB_MIN_NZ) || !c->sched_cand.empty());
  return CG_OK;
}

int cg_schedule(cg_ctx* c, int32_t* planes, int32_t* tz, int32_t* tuning) {
  return cg_schedule_form(c, planes, tz, nullptr, tuning);
}

int cg_steps_taken(cg_ctx* c, int64_t* steps) {
  if (!c || !steps) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  *steps = c->steps;
  return CG_OK;
}

// ---- checkpoints -------------------------------------------------------------------------

namespace {
struct StateHeader {
  char magic[8];
  int32_t abi, nx, ny, nz, precision, solid, lattice, streaming;
  int64_t steps;
  uint64_t payload;
};

// (offset, bytes) of each region saved in a checkpoint, for the current buffer
int state_regions(const cg_ctx* c, size_t off[6], size_t len[6]) {
  const Layout& L = c->L;
  const int cur = (int)(c->steps & 1);
  const size_t field = (size_t)L.stride * L.elem;
  int k = 0;
  off[k] = L.f[cur]; len[k++] = L.nq * (size_t)L.stride * L.pop_elem;
  off[k] = L.s[cur]; len[k++] = L.ns * field;
  off[k] = mac_last(c); len[k++] = 5 * field;
  off[k] = L.force; len[k++] = 3 * field;
  if (L.solid) {
    off[k] = L.aux[cur]; len[k++] = L.nq * field;
    off[k] = L.mask; len[k++] = (size_t)L.stride * 4;
  }
  return k;
}
}  // namespace

int cg_state_bytes(cg_ctx* c, size_t* bytes) {
  if (!c || !bytes) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  size_t off[6], len[6];
  int k = state_regions(c, off, len);
  size_t total = sizeof(StateHeader);
  for (int i = 0; i < k; ++i) total += len[i];
  *bytes = total;
  return CG_OK;
}

int cg_save_state(cg_ctx* c, void* host, size_t bytes) {
  if (!c || !host) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  if (int rc_ = settle(c)) return rc_;
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  size_t need = 0;
  cg_state_bytes(c, &need);
  if (bytes < need) return fail(CG_ERR_INVALID_ARG, "buffer too small: need " + std::to_string(need));
  StateHeader h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, "CG27STAT", 8);
  h.abi = CG27_ABI_VERSION;
  h.nx = c->prm.nx; h.ny = c->prm.ny; h.nz = c->prm.nz;
  h.precision = c->prm.precision;
  h.solid = c->L.solid;
  h.lattice = c->prm.lattice;
  h.streaming = c->prm.streaming;
  h.steps = c->steps;
  h.payload = need - sizeof(StateHeader);
  std::memcpy(host, &h, sizeof(h));
  size_t off[6], len[6];
  int k = state_regions(c, off, len);
  char* dst = static_cast<char*>(host) + sizeof(h);
  for (int i = 0; i < k; ++i) {
    CG_CUDA(cudaMemcpyAsync(dst, c->ws + off[i], len[i], cudaMemcpyDeviceToHost, c->stream));
    dst += len[i];
  }
  CG_CUDA(cudaStreamSynchronize(c->stream));
  return CG_OK;
}

int cg_load_state(cg_ctx* c, const void* host, size_t bytes) {
  if (!c || !host) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  if (c->batch) return fail(CG_ERR_INVALID_ARG, "the domain is a member of a batch: remove it first");
  if (bytes < sizeof(StateHeader)) return fail(CG_ERR_INVALID_ARG, "buffer too small");
  StateHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (std::memcmp(h.magic, "CG27STAT", 8) != 0 || h.abi != CG27_ABI_VERSION)
    return fail(CG_ERR_INVALID_ARG, "not a checkpoint of this library version");
  if (h.nx != c->prm.nx || h.ny != c->prm.ny || h.nz != c->prm.nz || h.precision != c->prm.precision ||
      h.solid != (int)c->L.solid || h.lattice != c->prm.lattice || h.streaming != c->prm.streaming)
    return fail(CG_ERR_INVALID_ARG, "checkpoint does not match the domain parameters");
  c->steps = h.steps;  // selects the buffer the regions go to
  c->mac_ready = -1;
  size_t off[6], len[6];
  int k = state_regions(c, off, len);
  size_t need = sizeof(h);
  for (int i = 0; i < k; ++i) need += len[i];
  if (bytes < need || h.payload != need - sizeof(h)) return fail(CG_ERR_INVALID_ARG, "checkpoint size mismatch");
  const char* src = static_cast<const char*>(host) + sizeof(h);
  for (int i = 0; i < k; ++i) {
    CG_CUDA(cudaMemcpyAsync(c->ws + off[i], src, len[i], cudaMemcpyHostToDevice, c->stream));
    src += len[i];
  }
  CG_CUDA(cudaMemsetAsync(c->ws + c->L.flag, 0, sizeof(unsigned int), c->stream));
  CG_CUDA(cudaStreamSynchronize(c->stream));
  c->initialised = true;
  return CG_OK;
}

}  // extern "C"
