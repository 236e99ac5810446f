// cg27_batch.cu -- batches of domains advanced in shared launches.
//
// A batch holds up to max_domains initialised domains of one precision and
// one kernel variant (walls or none; unit-rate Model D or the general
// collision).  One batch step is four launches whatever the number of
// members: each pass runs over a work list that concatenates the tiles of all
// members (cg27_step.cuh, "kernels of a batch of domains").  The descriptor
// table and the work lists live in the caller's batch workspace; the four
// launches of a step are captured once per step parity into CUDA graphs and
// replayed.  The z depth of the tiles is tuned online: the first steps after
// the member set has changed noticeably are timed for three depths and the
// fastest is kept (the results of a cell do not depend on the depth, so the
// tuning steps are ordinary steps of the simulation).
#include "cg27_host.cuh"

#include <algorithm>
#include <cstring>

using namespace cg27;

namespace {

constexpr int TUNE_STEPS = 3;  // timed steps per candidate depth

size_t dom_bytes(int precision) {
  return precision == CG_F64 ? sizeof(Dom<double>) : sizeof(Dom<float>);
}

struct BatchLayout {
  size_t doms = 0, items = 0, cell_start = 0, total = 0;
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
  L.total = off;
  return L;
}

// capacity of the tile table (1 MiB or more): a 128^3 member needs 8192 items
// at depth 1; larger members get deeper tiles when the table would overflow
long long table_items(int max_domains) { return std::max<long long>(1 << 16, 64LL * max_domains); }

bool has_solid(const cg_ctx* c) { return c->L.solid; }

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
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  bool use_graphs = true;
  // depth tuning
  int fixed_tz = 0;              // > 0: set by the caller, no tuning
  long long tuned_cells = 0;     // cell count the current choice was tuned for
  std::vector<int> cand;         // candidates still to time
  std::vector<std::pair<double, int>> timed;  // (ms per cell-update, depth)
  cudaEvent_t ev[2] = {nullptr, nullptr};
  int64_t steps = 0;

  ~cg_batch() {
    for (auto& g : graph)
      if (g) cudaGraphExecDestroy(g);
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
    for (cg_ctx* c : members) {
      c->batch = nullptr;
      c->batch_stream = nullptr;
    }
  }

  void drop_graphs() {
    for (auto& g : graph)
      if (g) {
        cudaGraphExecDestroy(g);
        g = nullptr;
      }
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

// depth with about eight tiles per SM over the whole batch
int heuristic_tz(const cg_batch* b) {
  int dev = 0, sms = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long col_planes = 0;  // sum over members of tiles_xy * nz
  for (const cg_ctx* c : b->members)
    col_planes += (long long)((c->prm.nx + TX - 1) / TX) * ((c->prm.ny + TY - 1) / TY) * c->prm.nz;
  const long long want = 8LL * sms;
  return (int)std::max(1LL, std::min<long long>(max_nz(b), (col_planes + want - 1) / want));
}

// tile items of the members at depth tz (each member's depth capped by its nz)
long long count_items(const cg_batch* b, int tz) {
  long long n = 0;
  for (const cg_ctx* c : b->members) {
    const int t = std::min(tz, c->prm.nz);
    n += (long long)((c->prm.nx + TX - 1) / TX) * ((c->prm.ny + TY - 1) / TY) * ((c->prm.nz + t - 1) / t);
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
  std::vector<int> cs(nd + 1);
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
    D.tiles_x = (c->prm.nx + TX - 1) / TX;
    D.tiles_y = (c->prm.ny + TY - 1) / TY;
    D.use_Q = c->prm.use_Q;
    const int chunks = (c->prm.nz + D.tz - 1) / D.tz;
    for (int bz = 0; bz < chunks; ++bz)
      for (int by = 0; by < D.tiles_y; ++by)
        for (int bx = 0; bx < D.tiles_x; ++bx) items.push_back(make_int4(d, bx, by, bz));
    const long long cblocks = (c->L.n + 127) / 128;
    if (cs[d] + cblocks > (1LL << 31) - 1) return fail(CG_ERR_UNSUPPORTED, "batch longer than 2^31-1 blocks");
    cs[d + 1] = cs[d] + (int)cblocks;
  }
  b->tiles = (int)items.size();
  b->cell_blocks = cs[nd];
  if (nd > 0) {
    CG_CUDA(cudaMemcpyAsync(b->ws + b->L.doms, doms.data(), nd * sizeof(Dom<T>), cudaMemcpyHostToDevice,
                            b->stream));
    CG_CUDA(cudaMemcpyAsync(b->ws + b->L.items, items.data(), items.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, b->stream));
    CG_CUDA(cudaMemcpyAsync(b->ws + b->L.cell_start, cs.data(), (nd + 1) * sizeof(int),
                            cudaMemcpyHostToDevice, b->stream));
    CG_CUDA(cudaStreamSynchronize(b->stream));  // the host vectors end here
  }
  b->table_steps = 0;
  b->dirty = false;
  b->drop_graphs();
  return CG_OK;
}

template <typename T, typename SF, bool SOLID, bool UNIT>
void launch_step(cg_batch* b, int par) {
  const Dom<T>* doms = reinterpret_cast<const Dom<T>*>(b->ws + b->L.doms);
  const int4* items = reinterpret_cast<const int4*>(b->ws + b->L.items);
  const int* cs = reinterpret_cast<const int*>(b->ws + b->L.cell_start);
  const int nd = (int)b->members.size();
  const dim3 blk(TX, TY, 1);
  k_macro_batch<T, SF, SOLID><<<b->tiles, blk, 0, b->stream>>>(doms, items, par);
  k_fields_batch<T, SOLID><<<b->tiles, blk, 0, b->stream>>>(doms, items, par);
  k_div_batch<T><<<b->tiles, blk, 0, b->stream>>>(doms, items, par);
  k_collide_batch<T, SF, SOLID, UNIT><<<b->cell_blocks, 128, 0, b->stream>>>(doms, cs, nd, par);
}

template <typename T, typename SF, bool SOLID, bool UNIT>
int run_steps(cg_batch* b, int64_t n) {
  for (int64_t s = 0; s < n; ++s) {
    const int par = (int)(b->table_steps & 1);
    if (b->use_graphs) {
      if (!b->graph[par]) {
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          launch_step<T, SF, SOLID, UNIT>(b, par);
          e = cudaStreamEndCapture(b->stream, &g);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[par], g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          // capture is not available on this stream: plain launches from now on
          (void)cudaGetLastError();
          b->graph[par] = nullptr;
          b->use_graphs = false;
        }
      }
    }
    if (b->use_graphs)
      CG_CUDA(cudaGraphLaunch(b->graph[par], b->stream));
    else
      launch_step<T, SF, SOLID, UNIT>(b, par);
    ++b->table_steps;
    ++b->steps;
    for (cg_ctx* c : b->members) ++c->steps;
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

// start tuning when the member set has changed by more than a factor two in cells
void maybe_retune(cg_batch* b) {
  if (b->fixed_tz > 0 || b->members.empty()) return;
  const long long n = total_cells(b);
  if (b->tuned_cells > 0 && n <= 2 * b->tuned_cells && 2 * n >= b->tuned_cells) return;
  const int h = heuristic_tz(b), mz = max_nz(b);
  b->cand.clear();
  for (int t : {h, std::max(1, h / 2), std::min(mz, 2 * h)})
    if (std::find(b->cand.begin(), b->cand.end(), t) == b->cand.end()) b->cand.push_back(t);
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
  b->use_graphs = b->stream != nullptr;  // the legacy default stream cannot be captured
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
  c->batch_stream = nullptr;
  b->dirty = true;
  if (b->members.empty()) {
    b->solid = b->unit = -1;
    b->tuned_cells = 0;
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
  } else {
    maybe_retune(b);
  }
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
  if (b->tz == 0) b->tz = heuristic_tz(b);
  // tuning: time TUNE_STEPS steps per candidate depth (one untimed step first,
  // for the table write and the graph capture)
  while (!b->cand.empty() && nsteps >= TUNE_STEPS + 1) {
    const int t = b->cand.back();
    b->cand.pop_back();
    b->tz = t;
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
      b->tz = std::min_element(b->timed.begin(), b->timed.end())->second;
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
