// cg27_batch.cu -- batches of domains advanced in shared launches.
//
// A batch holds up to max_domains initialised domains of one precision and
// one kernel variant (walls or none; unit-rate Model D or the general
// collision).  One batch step is four launches per group of members, whatever
// the number of members: each pass runs over a work list that concatenates the
// tiles of the group's members (cg27_step.cuh, "kernels of a batch of domains").  The descriptor
// table and the work lists live in the caller's batch workspace.  The members
// form up to BATCH_GROUPS contiguous groups of about equal cell counts, and a
// CUDA graph holds the four passes of every group as independent chains (the
// passes of one group wait only for that group), so the issue-bound stencil
// passes of one group overlap the bandwidth-bound population passes of another;
// BATCH_CHAIN consecutive steps go into one graph, each group's step t+1 after
// its step t.  Graphs are built per step parity and replayed.  The z depth of the tiles is tuned online: the first steps after
// the member set has changed noticeably are timed for three depths and the
// fastest is kept (the results of a cell do not depend on the depth, so the
// tuning steps are ordinary steps of the simulation).
#include "cg27_host.cuh"

#include <algorithm>
#include <cstring>

using namespace cg27;

namespace {

constexpr int TUNE_STEPS = 3;  // timed steps per candidate depth
constexpr int BATCH_GROUPS = 4;  // member groups whose passes run concurrently (4..32 within 1 %)
constexpr int BATCH_CHAIN = 8;   // steps per graph when enough steps are requested

size_t dom_bytes(int precision) {
  return precision == CG_F64 ? sizeof(Dom<double>) : sizeof(Dom<float>);
}

struct BatchLayout {
  size_t doms = 0, items = 0, cell_start = 0, tick = 0, total = 0;
  long long max_items = 0;
};

// the tile table holds up to max_items (domain, tile x, tile y, z chunk) items
BatchLayout batch_layout(int max_domains, int precision, long long max_items) {
  BatchLayout L;
  size_t off = 0;
  L.doms = off;
  off = align_up(off + (size_t)max_domains * dom_bytes(precision));
  L.cell_start = off;
  off = align_up(off + (size_t)(max_domains + 1) * sizeof(int));
  L.items = off;
  L.max_items = max_items;
  off = align_up(off + (size_t)max_items * sizeof(int4));
  L.tick = off;  // step number of the current launch, counted from the table write
  off = align_up(off + sizeof(int));
  L.total = off;
  return L;
}

// capacity of the tile table (1 MiB or more): a 128^3 member needs 8192 items
// at depth 1; larger members get deeper tiles when the table would overflow
long long table_items(int max_domains) { return std::max<long long>(1 << 16, 64LL * max_domains); }

bool has_solid(const cg_ctx* c) { return c->L.solid; }

// tile shapes of the z-marching batch kernels (cg27_step.cuh): 0 = ShapeA
// (32 x 8 threads), 1 = ShapeB (32 x 4)
constexpr int NUM_SHAPES = 2;
int tile_x(int shape) { return shape ? ShapeB::TX : ShapeA::TX; }
int tile_y(int shape) { return shape ? ShapeB::TY : ShapeA::TY; }

// advances the step number of a batch after a launch of n steps
__global__ void k_batch_tick(int* tick, int n) { *tick += n; }

// a schedule of the batch: tile depth, grid form, tile shape
struct Sched {
  int tz, persist, shape;
};

}  // namespace

struct cg_batch {
  int max_domains = 0, precision = 0;
  char* ws = nullptr;
  BatchLayout L;
  cudaStream_t stream = nullptr;
  std::vector<cg_ctx*> members;
  int solid = -1, unit = -1;  // kernel variant of the members (-1: no member yet)
  // work lists of the current table
  int tz = 0;            // z planes per tile of the current table
  int tiles = 0, cell_blocks = 0;
  bool dirty = true;     // member set or depth changed since the table was written
  int64_t table_steps = 0;  // batch steps since the table was written (selects the parity)
  // member groups of the current table: members gdom[k] .. gdom[k+1]-1, tile
  // items gitem[k] .. gitem[k+1]-1, collision blocks cs[gdom[k]] .. cs[gdom[k+1]]-1
  std::vector<int> gdom, gitem, cs;
  // graphs [one step | BATCH_CHAIN steps][parity of the first step]; a stale
  // graph is refreshed in place when the new one has the same shape
  cudaGraphExec_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
  bool stale[2][2] = {{false, false}, {false, false}};
  bool use_graphs = true;
  // launch schedule: tile depth, grid form (0: one block per work item,
  // 1: persistent, a grid of the blocks the GPU holds at once walking the
  // list) and tile shape of the z-marching passes
  int persist = 0;
  int shape = 0;
  int resident[NUM_SHAPES][4] = {};  // blocks per SM of the four batch kernels, per shape
  int sms = 0;
  // tuning of the schedule
  int fixed_tz = 0;              // > 0: set by the caller, not tuned
  int fixed_persist = -1;        // >= 0: set by the caller, not tuned
  int fixed_shape = -1;          // >= 0: set by the caller, not tuned
  long long tuned_cells = 0;     // cell count the current choice was tuned for
  std::vector<Sched> cand;       // schedules still to time
  std::vector<std::pair<double, Sched>> timed;  // (ms per step, schedule)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int64_t steps = 0;

  ~cg_batch() {
    for (auto& row : graph)
      for (auto& g : row)
        if (g) cudaGraphExecDestroy(g);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    for (cg_ctx* c : members) {
      c->batch = nullptr;
      c->batch_stop = -1;
      c->batch_stream = nullptr;
    }
  }

  // the member set or the schedule changed: graphs are rebuilt at their next use
  void drop_graphs() {
    for (auto& row : stale)
      for (bool& st : row) st = true;
  }
};

namespace {

long long total_cells(const cg_batch* b) {
  long long n = 0;
  for (const cg_ctx* c : b->members) n += c->L.n;
  return n;
}

int max_nz(const cg_batch* b) {
  int m = 1;
  for (const cg_ctx* c : b->members) m = std::max(m, c->prm.nz);
  return m;
}

// depth with about eight tiles of the current shape per SM over the whole batch
int heuristic_tz(const cg_batch* b) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tx = tile_x(b->shape), ty = tile_y(b->shape);
  long long col_planes = 0;  // sum over members of tiles_xy * nz
  for (const cg_ctx* c : b->members)
    col_planes += (long long)((c->prm.nx + tx - 1) / tx) * ((c->prm.ny + ty - 1) / ty) * c->prm.nz;
  const long long want = 8LL * sms;
  return (int)std::max(1LL, std::min<long long>(max_nz(b), (col_planes + want - 1) / want));
}

// tile items of the members at depth tz (each member's depth capped by its nz)
long long count_items(const cg_batch* b, int tz) {
  const int tx = tile_x(b->shape), ty = tile_y(b->shape);
  long long n = 0;
  for (const cg_ctx* c : b->members) {
    const int t = std::min(tz, c->prm.nz);
    n += (long long)((c->prm.nx + tx - 1) / tx) * ((c->prm.ny + ty - 1) / ty) * ((c->prm.nz + t - 1) / t);
  }
  return n;
}

template <typename T>
int write_table(cg_batch* b) {
  const int nd = (int)b->members.size();
  // a deeper tile when the item table would overflow
  int tz = b->tz;
  while (count_items(b, tz) > b->L.max_items && tz < max_nz(b)) tz = std::min(max_nz(b), 2 * tz);
  if (count_items(b, tz) > b->L.max_items) return fail(CG_ERR_UNSUPPORTED, "batch tile table too small");
  b->tz = tz;
  std::vector<Dom<T>> doms(nd);
  std::vector<int> cs(nd + 1), istart(nd + 1);
  std::vector<int4> items;
  items.reserve((size_t)count_items(b, tz));
  cs[0] = 0;
  for (int d = 0; d < nd; ++d) {
    const cg_ctx* c = b->members[d];
    Dom<T>& D = doms[d];
    D.g = make_geom(c);
    D.ph = make_phys<T>(c->prm);
    const int cur = (int)(c->steps & 1);
    D.P[0] = make_ptrs<T>(c, cur);
    D.P[1] = make_ptrs<T>(c, 1 - cur);
    D.tz = std::min(tz, c->prm.nz);
    D.tiles_x = (c->prm.nx + tile_x(b->shape) - 1) / tile_x(b->shape);
    D.tiles_y = (c->prm.ny + tile_y(b->shape) - 1) / tile_y(b->shape);
    D.use_Q = c->prm.use_Q;
    D.tick = reinterpret_cast<const int*>(b->ws + b->L.tick);
    const long long left = c->batch_stop < 0 ? (1LL << 30) : std::max<long long>(0, c->batch_stop - c->steps);
    D.stop = (int)std::min<long long>(left, 1LL << 30);
    const int chunks = (c->prm.nz + D.tz - 1) / D.tz;
    istart[d] = (int)items.size();
    for (int bz = 0; bz < chunks; ++bz)
      for (int by = 0; by < D.tiles_y; ++by)
        for (int bx = 0; bx < D.tiles_x; ++bx) items.push_back(make_int4(d, bx, by, bz));
    const long long cblocks = (c->L.n + 127) / 128;
    if (cs[d] + cblocks > (1LL << 31) - 1) return fail(CG_ERR_UNSUPPORTED, "batch longer than 2^31-1 blocks");
    cs[d + 1] = cs[d] + (int)cblocks;
  }
  b->tiles = (int)items.size();
  b->cell_blocks = cs[nd];
  istart[nd] = b->tiles;
  // contiguous member groups of about total / BATCH_GROUPS cells each
  long long total = 0;
  for (const cg_ctx* c : b->members) total += c->L.n;
  b->gdom.assign(1, 0);
  long long cum = 0;
  for (int d = 0; d < nd; ++d) {
    cum += b->members[d]->L.n;
    const int k = (int)b->gdom.size();
    if (k < BATCH_GROUPS && d + 1 < nd && cum * BATCH_GROUPS >= k * total) b->gdom.push_back(d + 1);
  }
  b->gdom.push_back(nd);
  b->gitem.clear();
  for (int g : b->gdom) b->gitem.push_back(istart[g]);
  b->cs = cs;
  if (nd > 0) {
    CG_CUDA(cudaMemcpyAsync(b->ws + b->L.doms, doms.data(), nd * sizeof(Dom<T>), cudaMemcpyHostToDevice,
                            b->stream));
    CG_CUDA(cudaMemcpyAsync(b->ws + b->L.items, items.data(), items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, b->stream));
    CG_CUDA(cudaMemcpyAsync(b->ws + b->L.cell_start, cs.data(), (nd + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream));
    CG_CUDA(cudaMemsetAsync(b->ws + b->L.tick, 0, sizeof(int), b->stream));
    CG_CUDA(cudaStreamSynchronize(b->stream));  // the host vectors end here
  }
  b->table_steps = 0;
  b->dirty = false;
  b->drop_graphs();
  return CG_OK;
}

// launch shape and arguments of the four passes of member group k
template <typename T>
struct GroupPass {
  const Dom<T>* doms;   // all members (the tile items name their domain)
  const Dom<T>* cdoms;  // from the group's first member (the collision)
  const int4* items;
  const int* cs;
  int ndom, block0;
  int ntiles, nblocks;  // work items of the tile passes and of the collision
  dim3 grid[4];         // grids of macro, fields, div, collide
};

// grid of a pass over `items` work items in one of ngroups concurrent groups:
// one block per item, or the group's share of the blocks the GPU holds at once
unsigned pass_grid(const cg_batch* b, int items, int kernel) {
  if (!b->persist) return (unsigned)items;
  const int ng = (int)b->gdom.size() - 1;
  const long long share =
      std::max(1LL, (long long)b->sms * std::max(1, b->resident[b->shape][kernel]) / std::max(1, ng));
  return (unsigned)std::min<long long>(items, share);
}

template <typename T>
GroupPass<T> group_pass(const cg_batch* b, int k) {
  GroupPass<T> g;
  const int d0 = b->gdom[k], d1 = b->gdom[k + 1];
  g.doms = reinterpret_cast<const Dom<T>*>(b->ws + b->L.doms);
  g.cdoms = g.doms + d0;
  g.items = reinterpret_cast<const int4*>(b->ws + b->L.items) + b->gitem[k];
  g.cs = reinterpret_cast<const int*>(b->ws + b->L.cell_start) + d0;
  g.ndom = d1 - d0;
  g.block0 = b->cs[d0];
  g.ntiles = b->gitem[k + 1] - b->gitem[k];
  g.nblocks = b->cs[d1] - b->cs[d0];
  for (int p = 0; p < 4; ++p) g.grid[p] = dim3(pass_grid(b, p < 3 ? g.ntiles : g.nblocks, p));
  return g;
}

// the four batch kernels of a variant in one grid form and tile shape
template <typename T, typename SF, bool SOLID, bool UNIT, bool PERSIST, class SH>
void batch_kernels_of(void* fn[4]) {
  fn[0] = (void*)k_macro_batch<T, SF, SOLID, PERSIST, SH>;
  fn[1] = (void*)k_fields_batch<T, SOLID, PERSIST, SH>;
  fn[2] = (void*)k_div_batch<T, PERSIST, SH>;
  fn[3] = (void*)k_collide_batch<T, SF, SOLID, UNIT, PERSIST>;
}
template <typename T, typename SF, bool SOLID, bool UNIT>
void batch_kernels(bool persist, int shape, void* fn[4]) {
  if (persist) {
    if (shape) batch_kernels_of<T, SF, SOLID, UNIT, true, ShapeB>(fn);
    else batch_kernels_of<T, SF, SOLID, UNIT, true, ShapeA>(fn);
  } else {
    if (shape) batch_kernels_of<T, SF, SOLID, UNIT, false, ShapeB>(fn);
    else batch_kernels_of<T, SF, SOLID, UNIT, false, ShapeA>(fn);
  }
}

template <typename T, typename SF, bool SOLID, bool UNIT>
void launch_step(cg_batch* b, int par) {
  const dim3 blk(tile_x(b->shape), tile_y(b->shape), 1), cblk(128, 1, 1);
  void* fn[4];
  batch_kernels<T, SF, SOLID, UNIT>(b->persist != 0, b->shape, fn);
  for (int k = 0; k + 1 < (int)b->gdom.size(); ++k) {
    GroupPass<T> g = group_pass<T>(b, k);
    void* a_tile[] = {(void*)&g.doms, (void*)&g.items, (void*)&g.ntiles, (void*)&par};
    void* a_coll[] = {(void*)&g.cdoms, (void*)&g.cs, (void*)&g.ndom, (void*)&par, (void*)&g.block0,
                      (void*)&g.nblocks};
    for (int p = 0; p < 4; ++p)
      cudaLaunchKernel(fn[p], g.grid[p], p < 3 ? blk : cblk, p < 3 ? a_tile : a_coll, 0, b->stream);
  }
  k_batch_tick<<<1, 1, 0, b->stream>>>(reinterpret_cast<int*>(b->ws + b->L.tick), 1);
}

// nsteps steps from parity par0: per group a chain of its four passes per step
template <typename T, typename SF, bool SOLID, bool UNIT>
cudaGraph_t build_batch_graph(const cg_batch* b, int par0, int nsteps) {
  cudaGraph_t gph;
  if (cudaGraphCreate(&gph, 0) != cudaSuccess) return nullptr;
  bool ok = true;
  const dim3 blk(tile_x(b->shape), tile_y(b->shape), 1), cblk(128, 1, 1);
  const int ng = (int)b->gdom.size() - 1;
  std::vector<cudaGraphNode_t> last(ng, nullptr);
  void* fn[4];
  batch_kernels<T, SF, SOLID, UNIT>(b->persist != 0, b->shape, fn);
  for (int s = 0; s < nsteps && ok; ++s) {
    int sp = (s << 1) | ((par0 + s) & 1);  // step offset within the graph, parity
    for (int k = 0; k < ng && ok; ++k) {
      GroupPass<T> g = group_pass<T>(b, k);
      void* a_tile[] = {(void*)&g.doms, (void*)&g.items, (void*)&g.ntiles, (void*)&sp};
      void* a_coll[] = {(void*)&g.cdoms, (void*)&g.cs, (void*)&g.ndom, (void*)&sp, (void*)&g.block0,
                        (void*)&g.nblocks};
      for (int p = 0; p < 4 && ok; ++p) {
        cudaKernelNodeParams kp = {};
        kp.func = fn[p];
        kp.gridDim = g.grid[p];
        kp.blockDim = p < 3 ? blk : cblk;
        kp.kernelParams = p < 3 ? a_tile : a_coll;
        cudaGraphNode_t node = nullptr;
        if (cudaGraphAddKernelNode(&node, gph, last[k] ? &last[k] : nullptr, last[k] ? 1 : 0, &kp) != cudaSuccess)
          ok = false;
        last[k] = node;
      }
    }
  }
  // the step number advances once every group's last pass is done
  if (ok) {
    int* tick = reinterpret_cast<int*>(b->ws + b->L.tick);
    int n = nsteps;
    void* a_tick[] = {(void*)&tick, (void*)&n};
    cudaKernelNodeParams kp = {};
    kp.func = (void*)k_batch_tick;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1);
    kp.kernelParams = a_tick;
    std::vector<cudaGraphNode_t> dv;
    for (cudaGraphNode_t n_ : last)
      if (n_) dv.push_back(n_);
    cudaGraphNode_t node = nullptr;
    if (cudaGraphAddKernelNode(&node, gph, dv.data(), dv.size(), &kp) != cudaSuccess) ok = false;
  }
  if (!ok) {
    cudaGraphDestroy(gph);
    return nullptr;
  }
  return gph;
}

// the executable graph of slot (k, par) for the current table: refreshed in
// place (cudaGraphExecUpdate: same nodes and edges, new grids and arguments)
// when the member groups keep their number, else instantiated anew
template <typename T, typename SF, bool SOLID, bool UNIT>
bool ready_graph(cg_batch* b, int k, int par, int nsteps) {
  cudaGraphExec_t& ex = b->graph[k][par];
  if (ex && !b->stale[k][par]) return true;
  cudaGraph_t g = build_batch_graph<T, SF, SOLID, UNIT>(b, par, nsteps);
  if (!g) return false;
  if (ex) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ex, g, &info) != cudaSuccess) {
      (void)cudaGetLastError();
      cudaGraphExecDestroy(ex);
      ex = nullptr;
    }
  }
  if (!ex && cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) ex = nullptr;
  cudaGraphDestroy(g);
  b->stale[k][par] = false;
  return ex != nullptr;
}

template <typename T, typename SF, bool SOLID, bool UNIT>
int run_steps(cg_batch* b, int64_t n) {
  if (b->resident[b->shape][0] == 0) {
    // blocks per SM of the four kernels of this variant and shape (the persistent grids)
    int dev = 0;
    CG_CUDA(cudaGetDevice(&dev));
    CG_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
    void* fn[4];
    batch_kernels<T, SF, SOLID, UNIT>(true, b->shape, fn);
    const int nt = tile_x(b->shape) * tile_y(b->shape);
    for (int p = 0; p < 4; ++p)
      CG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b->resident[b->shape][p], fn[p], p < 3 ? nt : 128, 0));
  }
  for (int64_t s = 0; s < n;) {
    const int par = (int)(b->table_steps & 1);
    const int k = (n - s >= BATCH_CHAIN) ? 1 : 0;
    const int m = k ? BATCH_CHAIN : 1;
    if (b->use_graphs && !ready_graph<T, SF, SOLID, UNIT>(b, k, par, m)) {
      (void)cudaGetLastError();
      b->use_graphs = false;  // graphs unavailable here: plain launches from now on
    }
    if (b->use_graphs)
      CG_CUDA(cudaGraphLaunch(b->graph[k][par], b->stream));
    else
      for (int i = 0; i < m; ++i) launch_step<T, SF, SOLID, UNIT>(b, (par + i) & 1);
    b->table_steps += m;
    b->steps += m;
    for (cg_ctx* c : b->members)
      c->steps += c->batch_stop < 0 ? m : std::max<int64_t>(0, std::min<int64_t>(m, c->batch_stop - c->steps));
    s += m;
  }
  CG_CUDA(cudaGetLastError());
  return CG_OK;
}

template <typename T, typename SF>
int run_any(cg_batch* b, int64_t n) {
  if (b->solid)
    return b->unit ? run_steps<T, SF, true, true>(b, n) : run_steps<T, SF, true, false>(b, n);
  return b->unit ? run_steps<T, SF, false, true>(b, n) : run_steps<T, SF, false, false>(b, n);
}

int run(cg_batch* b, int64_t n) {
  switch (b->precision) {
    case CG_F64: return run_any<double, double>(b, n);
    case CG_F32: return run_any<float, float>(b, n);
    case CG_F16S: return b->solid ? fail(CG_ERR_UNSUPPORTED, "walls with 16-bit storage")
                                  : (b->unit ? run_steps<float, __half, false, true>(b, n)
                                             : run_steps<float, __half, false, false>(b, n));
    default: return b->solid ? fail(CG_ERR_UNSUPPORTED, "walls with 16-bit storage")
                             : (b->unit ? run_steps<float, __nv_bfloat16, false, true>(b, n)
                                        : run_steps<float, __nv_bfloat16, false, false>(b, n));
  }
}

int write_table_any(cg_batch* b) {
  return b->precision == CG_F64 ? write_table<double>(b) : write_table<float>(b);
}

// Start tuning when the member set has changed by more than a factor two in
// cells: the candidates are three depths (the heuristic h, h/2, 2h of each
// tile shape) times the two grid forms times the two tile shapes, less what
// the caller has fixed.
void maybe_retune(cg_batch* b) {
  if (b->members.empty()) return;
  const long long n = total_cells(b);
  if (b->tuned_cells > 0 && n <= 2 * b->tuned_cells && 2 * n >= b->tuned_cells) return;
  std::vector<int> forms, shapes;
  if (b->fixed_persist >= 0) forms.push_back(b->fixed_persist);
  else forms = {0, 1};
  if (b->fixed_shape >= 0) shapes.push_back(b->fixed_shape);
  else shapes = {0, 1};
  const int keep = b->shape;
  b->cand.clear();
  for (int sh : shapes) {
    std::vector<int> depths;
    if (b->fixed_tz > 0) {
      depths.push_back(b->fixed_tz);
    } else {
      b->shape = sh;  // the heuristic counts tiles of this shape
      const int h = heuristic_tz(b), mz = max_nz(b);
      for (int t : {h, std::max(1, h / 2), std::min(mz, 2 * h)})
        if (std::find(depths.begin(), depths.end(), t) == depths.end()) depths.push_back(t);
    }
    for (int t : depths)
      for (int f : forms) b->cand.push_back({t, f, sh});
  }
  b->shape = keep;
  if (b->cand.size() == 1) {  // nothing left to choose
    b->tz = b->cand[0].tz;
    b->persist = b->cand[0].persist;
    b->shape = b->cand[0].shape;
    b->cand.clear();
    b->dirty = true;
  }
  b->timed.clear();
  b->tuned_cells = n;
}

}  // namespace

extern "C" {

int cg_batch_workspace_bytes(int32_t max_domains, int32_t precision, size_t* bytes) {
  if (!bytes) return fail(CG_ERR_INVALID_ARG, "bytes is NULL");
  if (max_domains < 1 || max_domains > (1 << 20)) return fail(CG_ERR_INVALID_ARG, "max_domains must be in [1, 2^20]");
  if (precision != CG_F64 && precision != CG_F32 && precision != CG_F16S && precision != CG_BF16S)
    return fail(CG_ERR_UNSUPPORTED, "unknown precision");
  *bytes = batch_layout(max_domains, precision, table_items(max_domains)).total;
  return CG_OK;
}

int cg_batch_create(int32_t max_domains, int32_t precision, void* d_workspace, size_t bytes, void* cuda_stream,
                    cg_batch** out) {
  if (!out) return fail(CG_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  size_t need = 0;
  int rc = cg_batch_workspace_bytes(max_domains, precision, &need);
  if (rc) return rc;
  if (!d_workspace) return fail(CG_ERR_WORKSPACE, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(d_workspace) % ALIGN != 0)
    return fail(CG_ERR_WORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < need) return fail(CG_ERR_WORKSPACE, "workspace smaller than cg_batch_workspace_bytes()");
  cg_batch* b = new cg_batch();
  b->max_domains = max_domains;
  b->precision = precision;
  b->ws = static_cast<char*>(d_workspace);
  b->L = batch_layout(max_domains, precision, table_items(max_domains));
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->use_graphs = b->stream != nullptr;  // plain launches on the legacy default stream
  if (cudaEventCreate(&b->ev[0]) != cudaSuccess || cudaEventCreate(&b->ev[1]) != cudaSuccess) {
    delete b;
    return fail(CG_ERR_CUDA, "cudaEventCreate failed");
  }
  *out = b;
  return CG_OK;
}

int cg_batch_add(cg_batch* b, cg_ctx* c) {
  if (!b || !c) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  if (!c->initialised) return fail(CG_ERR_INVALID_ARG, "cg_init_fields() has not been called");
  if (c->batch) return fail(CG_ERR_INVALID_ARG, "the domain is already in a batch");
  if (c->prm.precision != b->precision) return fail(CG_ERR_UNSUPPORTED, "precision differs from the batch's");
  if (c->prm.lattice != CG_D3Q27) return fail(CG_ERR_UNSUPPORTED, "batches hold D3Q27 domains");
  if (c->prm.streaming != CG_STREAM_TWO_BUFFERS)
    return fail(CG_ERR_UNSUPPORTED, "batches hold domains with two population buffers");
  if ((int)b->members.size() >= b->max_domains) return fail(CG_ERR_INVALID_ARG, "the batch is full");
  // the batch kernels address populations with 32-bit column offsets
  if (8LL * c->L.stride + (long long)c->prm.nx * c->prm.ny >= (1LL << 31))
    return fail(CG_ERR_UNSUPPORTED, "batch members hold at most about 238 million cells");
  const int solid = has_solid(c) ? 1 : 0, unit = c->unit ? 1 : 0;
  if (!b->members.empty() && (solid != b->solid || unit != b->unit))
    return fail(CG_ERR_UNSUPPORTED,
                "kernel variant (walls, unit-rate Model D) differs from the batch's members");
  // the domain's own stream may still hold its initialisation
  CG_CUDA(cudaStreamSynchronize(c->stream));
  b->solid = solid;
  b->unit = unit;
  b->members.push_back(c);
  c->batch = b;
  c->batch_stop = -1;
  c->batch_stream = b->stream;
  b->dirty = true;
  maybe_retune(b);
  return CG_OK;
}

int cg_batch_remove(cg_batch* b, cg_ctx* c) {
  if (!b || !c) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  auto it = std::find(b->members.begin(), b->members.end(), c);
  if (it == b->members.end()) return fail(CG_ERR_INVALID_ARG, "the domain is not in this batch");
  CG_CUDA(cudaStreamSynchronize(b->stream));  // its last steps are complete
  b->members.erase(it);
  c->batch = nullptr;
  c->batch_stop = -1;
  c->batch_stream = nullptr;
  b->dirty = true;
  if (b->members.empty()) {
    b->solid = b->unit = -1;
    b->tuned_cells = 0;
    for (auto& r : b->resident) r[0] = 0;  // the next member may bring another kernel variant
  } else {
    maybe_retune(b);
  }
  return CG_OK;
}

int cg_batch_size(cg_batch* b, int32_t* n) {
  if (!b || !n) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  *n = (int32_t)b->members.size();
  return CG_OK;
}

int cg_batch_set_depth(cg_batch* b, int32_t tz) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "batch is NULL");
  if (tz < 0) return fail(CG_ERR_INVALID_ARG, "depth must be >= 0");
  b->fixed_tz = tz;
  b->tuned_cells = 0;
  b->cand.clear();
  b->timed.clear();
  if (tz > 0) {
    b->tz = tz;
    b->dirty = true;
  }
  maybe_retune(b);
  return CG_OK;
}

int cg_batch_set_persistent(cg_batch* b, int32_t mode) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "batch is NULL");
  if (mode < -1 || mode > 1) return fail(CG_ERR_INVALID_ARG, "mode must be -1 (tuned), 0 or 1");
  b->fixed_persist = mode;
  b->tuned_cells = 0;
  b->cand.clear();
  b->timed.clear();
  if (mode >= 0) {
    b->persist = mode;
    b->dirty = true;
  }
  maybe_retune(b);
  return CG_OK;
}

int cg_batch_set_stop(cg_batch* b, cg_ctx* c, int64_t total_steps) {
  if (!b || !c) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  if (std::find(b->members.begin(), b->members.end(), c) == b->members.end())
    return fail(CG_ERR_INVALID_ARG, "the domain is not in this batch");
  CG_CUDA(cudaStreamSynchronize(b->stream));  // the table being replaced may be in use
  c->batch_stop = total_steps < 0 ? -1 : total_steps;
  b->dirty = true;
  return CG_OK;
}

int cg_batch_set_tile(cg_batch* b, int32_t shape) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "batch is NULL");
  if (shape < -1 || shape >= NUM_SHAPES) return fail(CG_ERR_INVALID_ARG, "tile must be -1 (tuned), 0 or 1");
  b->fixed_shape = shape;
  b->tuned_cells = 0;
  b->cand.clear();
  b->timed.clear();
  if (shape >= 0) {
    b->shape = shape;
    b->dirty = true;
  }
  maybe_retune(b);
  return CG_OK;
}

int cg_batch_tile(cg_batch* b, int32_t* tile_nx, int32_t* tile_ny) {
  if (!b || !tile_nx || !tile_ny) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  *tile_nx = tile_x(b->shape);
  *tile_ny = tile_y(b->shape);
  return CG_OK;
}

int cg_batch_persistent(cg_batch* b, int32_t* mode) {
  if (!b || !mode) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  *mode = b->persist;
  return CG_OK;
}

int cg_batch_depth(cg_batch* b, int32_t* tz, int32_t* tuning) {
  if (!b || !tz || !tuning) return fail(CG_ERR_INVALID_ARG, "NULL argument");
  *tz = b->tz;
  *tuning = b->cand.empty() ? 0 : 1;
  return CG_OK;
}

int cg_batch_step(cg_batch* b, int64_t nsteps) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "batch is NULL");
  if (nsteps < 0) return fail(CG_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (b->members.empty() || nsteps == 0) return CG_OK;
  int rc;
  if (b->fixed_tz > 0 && b->tz != b->fixed_tz) {
    b->tz = b->fixed_tz;
    b->dirty = true;
  }
  if (b->fixed_persist >= 0 && b->persist != b->fixed_persist) {
    b->persist = b->fixed_persist;
    b->dirty = true;
  }
  if (b->fixed_shape >= 0 && b->shape != b->fixed_shape) {
    b->shape = b->fixed_shape;
    b->dirty = true;
  }
  if (b->tz == 0) b->tz = heuristic_tz(b);
  // tuning: time TUNE_STEPS steps per candidate schedule (one untimed step
  // first, for the table write and the graph build)
  while (!b->cand.empty() && nsteps >= TUNE_STEPS + 1) {
    const Sched t = b->cand.back();
    b->cand.pop_back();
    b->tz = t.tz;
    b->persist = t.persist;
    b->shape = t.shape;
    if ((rc = write_table_any(b))) return rc;
    if ((rc = run(b, 1))) return rc;
    CG_CUDA(cudaEventRecord(b->ev[0], b->stream));
    if ((rc = run(b, TUNE_STEPS))) return rc;
    CG_CUDA(cudaEventRecord(b->ev[1], b->stream));
    CG_CUDA(cudaEventSynchronize(b->ev[1]));
    float ms = 0.f;
    CG_CUDA(cudaEventElapsedTime(&ms, b->ev[0], b->ev[1]));
    b->timed.push_back({ms / TUNE_STEPS, t});
    nsteps -= TUNE_STEPS + 1;
    if (b->cand.empty()) {
      const Sched best = std::min_element(b->timed.begin(), b->timed.end(),
                                          [](const std::pair<double, Sched>& x, const std::pair<double, Sched>& y) {
                                            return x.first < y.first;
                                          })->second;
      b->tz = best.tz;
      b->persist = best.persist;
      b->shape = best.shape;
      b->dirty = true;
    }
  }
  if (b->dirty && (rc = write_table_any(b))) return rc;
  return run(b, nsteps);
}

int cg_batch_sync(cg_batch* b) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "batch is NULL");
  CG_CUDA(cudaStreamSynchronize(b->stream));
  return CG_OK;
}

int cg_batch_destroy(cg_batch* b) {
  if (!b) return fail(CG_ERR_INVALID_ARG, "batch is NULL");
  cudaStreamSynchronize(b->stream);
  delete b;
  return CG_OK;
}

}  // extern "C"
