// Host driver and C ABI: context lifetime, the step-iteration launch
// sequence (Sec. 2 of the paper: the CPU issues one kernel per action per
// step iteration), the device-side loop in a CUDA graph, primaries in,
// tallies out. All copies are stream ordered on the context's stream
// (Sec. 3.4: no device-wide synchronisation from blocking memcpy).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include "celer_gb.h"
#include "launch.h"
#include "tables.h"
#include "fastmath.cuh"

using namespace celer;

namespace {

constexpr double kNA = 6.02214076e23;
constexpr double kNeWater = 3.343e23;  // reference electron density of the photon model
constexpr double kZWater = 7.42;       // reference effective Z of the photon model
constexpr int kTimingPool = 8192;

uint64_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}

}  // namespace

struct celer_ctx {
  celer_problem prob{};
  bool ctl_fresh = false;  // h_ctl equals the device control block (no head/tail-moving work since)
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  Params p{};
  LaunchShape shape{};
  std::vector<void*> dev_allocs;
  std::vector<void*> host_allocs;
  std::vector<double> zb;
  std::vector<int> layer_mat;
  std::vector<double> h_mtab;  // log/exp reduction tables (host copy, source of the device copy)
  std::unordered_map<uint32_t, uint64_t> next_tid;
  uint64_t next_history = 0;
  StagedPrimary* h_stage = nullptr;
  StagedPrimary* d_stage = nullptr;
  uint64_t stage_cap = 0;
  cudaEvent_t stage_done = nullptr;
  Ctl* h_ctl = nullptr;          // pinned mirror of the control block
  double* h_bounce = nullptr;    // pinned bounce buffer for tallies / history
  size_t bounce_bytes = 0;
  unsigned int* h_cont = nullptr;  // pinned loop-condition slots
  cudaEvent_t cont_ev[2] = {nullptr, nullptr};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_policy = -1;
  int graph_split = -1;
  int split_actions = 0;
  std::string last_error;
  // kernel timing
  bool timing = false;
  std::vector<cudaEvent_t> t_start, t_stop;
  std::vector<int> t_kid;
  int t_used = 0;
  uint32_t* ring_state = nullptr;  // buffer entry states, set in the Params of asynchronous runs only
  bool tiles_stale = false;  // the per-tile vacancy prefix predates the last block-local iterations
  // per-iteration hit readout of the host loop: 0 off, 1 stream-ordered, 2 synchronous
  int hit_mode = 0;
  double* h_hits = nullptr;
  double t_total_ms[KID_COUNT] = {};
  uint64_t t_launches[KID_COUNT] = {};
};

namespace {

celer_status fail(celer_ctx* ctx, celer_status s, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return s;
}

celer_status cuda_fail(celer_ctx* ctx, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(ctx, CELER_ERR_CUDA, m);
}

#define CELER_CUDA(ctx, call)                                  \
  do {                                                         \
    cudaError_t err_ = (call);                                 \
    if (err_ != cudaSuccess) return cuda_fail(ctx, err_, #call); \
  } while (0)

template <class T>
cudaError_t dalloc(celer_ctx* ctx, T** out, size_t n) {
  void* ptr = nullptr;
  const size_t bytes = (n ? n : 1) * sizeof(T);
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) return e;
  ctx->dev_allocs.push_back(ptr);
  e = cudaMemsetAsync(ptr, 0, bytes, ctx->stream);
  *out = static_cast<T*>(ptr);
  return e;
}

template <class T>
cudaError_t halloc(celer_ctx* ctx, T** out, size_t n) {
  void* ptr = nullptr;
  cudaError_t e = cudaMallocHost(&ptr, (n ? n : 1) * sizeof(T));
  if (e != cudaSuccess) return e;
  ctx->host_allocs.push_back(ptr);
  std::memset(ptr, 0, (n ? n : 1) * sizeof(T));
  *out = static_cast<T*>(ptr);
  return cudaSuccess;
}

// Layer containing z: the largest i <= L-1 with z_i <= z (z at the far end
// belongs to the last layer); a track exactly on an inner plane and moving
// backwards belongs to the layer behind it.
int layer_of(const std::vector<double>& zb, double z, double uz) {
  const int L = (int)zb.size() - 1;
  if (z >= zb[L]) return L - 1;
  int lo = 0, hi = L - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (zb[mid] <= z)
      lo = mid;
    else
      hi = mid - 1;
  }
  if (z == zb[lo] && uz < 0.0 && lo > 0) --lo;
  return lo;
}

bool policy_sorted(int policy) { return global_partition(policy); }

int keys_of(int policy) {
  return policy == POLICY_ACTION ? kKeysAlong : (policy == POLICY_ACTION_TYPE ? kKeysFull : 0);
}

// ---- kernel timing (plain loop only)
void timing_resolve(celer_ctx* ctx) {
  if (ctx->t_used == 0) return;
  cudaStreamSynchronize(ctx->stream);
  for (int i = 0; i < ctx->t_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->t_start[i], ctx->t_stop[i]) == cudaSuccess) {
      ctx->t_total_ms[ctx->t_kid[i]] += ms;
      ctx->t_launches[ctx->t_kid[i]] += 1;
    }
  }
  ctx->t_used = 0;
}

template <class F>
void timed(celer_ctx* ctx, cudaStream_t s, int kid, F&& launch, bool allow_timing) {
  if (!(ctx->timing && allow_timing)) {
    launch();
    return;
  }
  if (ctx->t_used == (int)ctx->t_start.size()) timing_resolve(ctx);
  const int i = ctx->t_used++;
  ctx->t_kid[i] = kid;
  cudaEventRecord(ctx->t_start[i], s);
  launch();
  cudaEventRecord(ctx->t_stop[i], s);
}

// One step iteration as a sequence of launches on stream s. Phase-merged:
// fill + step limit (+ bookkeeping), scatter, along-step + interactions (+
// end of iteration). Per action (split_actions), as in the paper's loop over
// actions: fill, step limit, scatter, one along-step kernel per particle kind,
// one kernel per interaction, end of iteration.
// The block-pass policies (LOCAL, DATA) run one launch per iteration in the
// phase-merged modes; they need the per-block vacancy scan at the start of
// each run.
bool fused_local(const celer_ctx* ctx) { return !ctx->split_actions && block_pass(ctx->p.policy); }

// Start of a run (or a single step): the block-local iterations start from a
// fresh per-block vacancy scan; the others, after block-local ones, from a
// fresh per-tile scan.
void begin_policy_run(celer_ctx* ctx) {
  if (fused_local(ctx)) {
    launch_local_prepare(ctx->p, ctx->shape, ctx->stream);
    ctx->tiles_stale = true;
  } else if (ctx->tiles_stale) {
    launch_scan_tiles(ctx->p, ctx->stream);
    ctx->tiles_stale = false;
  }
}

void launch_iteration(celer_ctx* ctx, cudaStream_t s, unsigned long long handle, int use_handle) {
  const Params& p = ctx->p;
  const LaunchShape& sh = ctx->shape;
  const bool t = use_handle == 0;
  const bool sorted = policy_sorted(p.policy);
  if (!ctx->split_actions && block_pass(p.policy)) {
    timed(ctx, s, KID_LOCAL, [&] { launch_local(p, sh, handle, use_handle, s); }, t);
    return;
  }
  if (!ctx->split_actions) {
    timed(ctx, s, KID_FILL_STEP, [&] { launch_fill_step(p, sh, s); }, t);
    if (sorted) timed(ctx, s, KID_SCATTER, [&] { launch_scatter(p, sh, s); }, t);
    timed(ctx, s, KID_STEP, [&] { launch_step(p, sh, handle, use_handle, s); }, t);
    return;
  }
  timed(ctx, s, KID_FILL, [&] { launch_fill(p, sh, s); }, t);
  timed(ctx, s, KID_PRE_STEP, [&] { launch_pre_step(p, sh, s); }, t);
  if (sorted) timed(ctx, s, KID_SCATTER, [&] { launch_scatter(p, sh, s); }, t);
  timed(ctx, s, KID_ALONG_NEUTRAL, [&] { launch_along(p, 0, sh, s); }, t);
  timed(ctx, s, KID_ALONG_CHARGED, [&] { launch_along(p, 1, sh, s); }, t);
  const int P = p.processes;
  if (P & PROC_COMPTON) timed(ctx, s, KID_POST_COMPTON, [&] { launch_post(p, A_COMPTON, sh, s); }, t);
  if (P & PROC_PE) timed(ctx, s, KID_POST_PE, [&] { launch_post(p, A_PE, sh, s); }, t);
  if (P & PROC_PAIR) timed(ctx, s, KID_POST_PAIR, [&] { launch_post(p, A_PAIR, sh, s); }, t);
  if (P & PROC_MOLLER) timed(ctx, s, KID_POST_MOLLER, [&] { launch_post(p, A_MOLLER, sh, s); }, t);
  if (P & PROC_BREMS) timed(ctx, s, KID_POST_BREMS, [&] { launch_post(p, A_BREMS, sh, s); }, t);
  timed(ctx, s, KID_LOOP_CTL, [&] { launch_loop_ctl(p, handle, use_handle, s); }, t);
}

void destroy_graph(celer_ctx* ctx) {
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->graph) cudaGraphDestroy(ctx->graph);
  ctx->graph_exec = nullptr;
  ctx->graph = nullptr;
  ctx->graph_policy = -1;
}

// The whole step loop as one CUDA graph: a conditional while-node whose body
// is one iteration; the last kernel of the body sets the condition.
celer_status build_graph(celer_ctx* ctx) {
  destroy_graph(ctx);
  cudaGraph_t g = nullptr;
  CELER_CUDA(ctx, cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle handle;
  cudaError_t e = cudaGraphConditionalHandleCreate(&handle, g, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "cudaGraphConditionalHandleCreate");
  }
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = handle;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "cudaGraphAddNode(conditional)");
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(ctx->capture_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "cudaStreamBeginCaptureToGraph");
  }
  launch_iteration(ctx, ctx->capture_stream, (unsigned long long)handle, 1);
  cudaGraph_t captured = nullptr;
  e = cudaStreamEndCapture(ctx->capture_stream, &captured);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "cudaStreamEndCapture");
  }
  cudaGraphExec_t exec = nullptr;
  e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(ctx, e, "cudaGraphInstantiate");
  }
  ctx->graph = g;
  ctx->graph_exec = exec;
  ctx->graph_policy = ctx->p.policy;
  ctx->graph_split = ctx->split_actions;
  return CELER_OK;
}

celer_status read_ctl(celer_ctx* ctx) {
  CELER_CUDA(ctx, cudaMemcpyAsync(ctx->h_ctl, ctx->p.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  ctx->ctl_fresh = true;
  return CELER_OK;
}

void fill_stats(const Ctl& c, celer_step_stats* s) {
  s->iteration = c.iteration;
  s->alive = c.alive;
  s->queued = c.tail - c.head;
  s->steps = c.last_steps_iter;
  s->steps_total = c.steps_total;
  s->deferred = c.last_n_deferred;
  s->error = c.error;
  for (int k = 0; k < 16; ++k) s->action_count[k] = k < kMaxKeys ? c.last_action_count[k] : 0;
}

celer_status status_from_error(celer_ctx* ctx, unsigned err) {
  if (err & ERR_ITERATIONS) return fail(ctx, CELER_ERR_TIMEOUT, "iteration limit reached");
  if (err & ERR_NO_PROGRESS)
    return fail(ctx, CELER_ERR_CAPACITY, "initializer buffer full and no track can make progress");
  if (err & ERR_PRIMARIES_REJECTED)
    return fail(ctx, CELER_ERR_INVALID, "device primaries rejected (invalid record or buffer full)");
  if (err & ERR_BARRIER_TIMEOUT) return fail(ctx, CELER_ERR_TIMEOUT, "persistent loop: a bounded wait (grid barrier or buffer entry) timed out");
  if (err & ERR_VACANCY) return fail(ctx, CELER_ERR_STATE, "vacancy bookkeeping inconsistent");
  if (err & ERR_SAMPLING) return fail(ctx, CELER_ERR_STATE, "rejection sampling hit its attempt limit");
  if (err) return fail(ctx, CELER_ERR_STATE, "device error flag set");
  return CELER_OK;
}

celer_status validate_problem(const celer_problem* pb, std::string& why) {
  if (!pb) return why = "null problem", CELER_ERR_INVALID;
  if (pb->n_materials < 1 || pb->n_materials > kMaxMaterials || !pb->materials)
    return why = "n_materials must be in [1, 8]", CELER_ERR_INVALID;
  for (int m = 0; m < pb->n_materials; ++m) {
    const celer_material& M = pb->materials[m];
    const bool ne_ok = M.ne > 0.0 || (M.A > 0.0 && M.rho > 0.0 && M.Z > 0.0);
    if (!ne_ok || !(M.Z > 0.0) || !(M.X0 > 0.0) || !(M.I > 0.0))
      return why = "material " + std::to_string(m) + " has non-positive parameters", CELER_ERR_INVALID;
  }
  if (pb->n_layers < 1 || pb->n_periods < 1 || !pb->layer_material || !pb->layer_thickness)
    return why = "empty layer stack", CELER_ERR_INVALID;
  if ((long)pb->n_layers * pb->n_periods > kMaxLayers) return why = "more than 1024 layers", CELER_ERR_INVALID;
  for (int i = 0; i < pb->n_layers; ++i) {
    if (pb->layer_material[i] < 0 || pb->layer_material[i] >= pb->n_materials)
      return why = "layer material index out of range", CELER_ERR_INVALID;
    if (!(pb->layer_thickness[i] > 0.0) || !std::isfinite(pb->layer_thickness[i]))
      return why = "layer thickness must be positive", CELER_ERR_INVALID;
  }
  if (!(pb->half_x > 0.0) || !(pb->half_y > 0.0)) return why = "half widths must be positive", CELER_ERR_INVALID;
  if (!std::isfinite(pb->Bz)) return why = "Bz must be finite", CELER_ERR_INVALID;
  if (pb->field_substep_cap < 0) return why = "field_substep_cap must be >= 0", CELER_ERR_INVALID;
  if (!(pb->cut_track >= kGridEmin) || !(pb->cut_track < kGridEmax))
    return why = "cut_track must be in [1 keV, 10 GeV)", CELER_ERR_INVALID;
  if (!(pb->cut_moller > 0.0) || !(pb->cut_brems > 0.0)) return why = "production cuts must be positive", CELER_ERR_INVALID;
  if (pb->processes & ~63) return why = "unknown process bits", CELER_ERR_INVALID;
  if (pb->tally_mode != CELER_TALLY_ZBINS && pb->tally_mode != CELER_TALLY_LAYERS)
    return why = "unknown tally mode", CELER_ERR_INVALID;
  if (pb->tally_mode == CELER_TALLY_ZBINS && pb->n_zbins < 1) return why = "n_zbins must be >= 1", CELER_ERR_INVALID;
  if (pb->n_slots < 1 || pb->n_slots > (1ull << 30)) return why = "n_slots must be in [1, 2^30]", CELER_ERR_INVALID;
  if (pb->init_capacity < 1 || pb->init_capacity > (1ull << 34)) return why = "bad init_capacity", CELER_ERR_INVALID;
  if (pb->max_events < 1) return why = "max_events must be >= 1", CELER_ERR_INVALID;
  if (pb->sort_policy < 0 || pb->sort_policy >= kPolicyCount) return why = "unknown sort policy", CELER_ERR_INVALID;
  if (pb->block_size != 0 && pb->block_size != 128 && pb->block_size != 256 && pb->block_size != 512)
    return why = "block_size must be 128, 256 or 512", CELER_ERR_INVALID;
  return CELER_OK;
}

}  // namespace

extern "C" {

const char* celer_status_string(celer_status s) {
  switch (s) {
    case CELER_OK: return "ok";
    case CELER_ERR_INVALID: return "invalid argument";
    case CELER_ERR_CAPACITY: return "capacity exceeded";
    case CELER_ERR_CUDA: return "CUDA error";
    case CELER_ERR_TIMEOUT: return "iteration limit reached";
    case CELER_ERR_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* celer_last_error(const celer_ctx* ctx) { return ctx ? ctx->last_error.c_str() : ""; }

void celer_destroy(celer_ctx* ctx) {
  if (!ctx) return;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  destroy_graph(ctx);
  for (auto& e : ctx->t_start) cudaEventDestroy(e);
  for (auto& e : ctx->t_stop) cudaEventDestroy(e);
  if (ctx->stage_done) cudaEventDestroy(ctx->stage_done);
  for (auto& e : ctx->cont_ev)
    if (e) cudaEventDestroy(e);
  for (void* ptr : ctx->dev_allocs) cudaFree(ptr);
  for (void* ptr : ctx->host_allocs) cudaFreeHost(ptr);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
}

celer_status celer_create(const celer_problem* pb, celer_ctx** out) {
  if (!out) return CELER_ERR_INVALID;
  *out = nullptr;
  std::string why;
  if (validate_problem(pb, why) != CELER_OK) {
    fprintf(stderr, "celer_create: %s\n", why.c_str());
    return CELER_ERR_INVALID;
  }
  celer_ctx* ctx = new celer_ctx();
  ctx->prob = *pb;
  ctx->prob.materials = nullptr;
  ctx->prob.layer_material = nullptr;
  ctx->prob.layer_thickness = nullptr;
  ctx->stream = (cudaStream_t)pb->cuda_stream;
  auto bail = [&](celer_status s) {
    if (s != CELER_OK) {
      fprintf(stderr, "celer_create: %s\n", ctx->last_error.c_str());
      celer_destroy(ctx);
    }
    return s;
  };
#define CREATE_CUDA(call)                                   \
  do {                                                      \
    cudaError_t err_ = (call);                              \
    if (err_ != cudaSuccess) return bail(cuda_fail(ctx, err_, #call)); \
  } while (0)

  CREATE_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));

  // geometry: boundaries by cumulative sum from z = 0, one material per layer
  const int L = pb->n_layers * pb->n_periods;
  ctx->zb.assign(L + 1, 0.0);
  ctx->layer_mat.assign(L, 0);
  for (int i = 0; i < L; ++i) {
    const int j = i % pb->n_layers;
    ctx->layer_mat[i] = pb->layer_material[j];
    ctx->zb[i + 1] = ctx->zb[i] + pb->layer_thickness[j];
  }
  const int n_bins = pb->tally_mode == CELER_TALLY_LAYERS ? L : pb->n_zbins;

  // materials: electron density and photon-model scale factors
  std::vector<MaterialData> mats(pb->n_materials);
  for (int m = 0; m < pb->n_materials; ++m) {
    const celer_material& M = pb->materials[m];
    MaterialData& d = mats[m];
    d.ne = M.ne > 0.0 ? M.ne : kNA * M.rho * M.Z / M.A;
    d.Z = M.Z;
    d.X0 = M.X0;
    d.I = M.I;
    const double zr = M.Z / kZWater;
    d.f_pe = d.ne / kNeWater * zr * zr * zr;
    d.f_pair = d.ne / kNeWater * zr;
  }

  Params& p = ctx->p;
  const uint32_t N = (uint32_t)pb->n_slots;
  const uint64_t C = next_pow2(pb->init_capacity);
  p.n_slots = N;
  p.n_tiles = (N + kTile - 1) / kTile;
  p.ring_capacity = C;
  p.ring_mask = C - 1;
  p.policy = pb->sort_policy;
  p.n_keys = keys_of(p.policy);
  p.n_layers = L;
  p.n_materials = pb->n_materials;
  p.hx = pb->half_x;
  p.hy = pb->half_y;
  p.Bz = pb->Bz;
  p.field_cap = pb->field_substep_cap;
  p.async_warps = 1;  // the asynchronous loop schedules per warp for the block-local policy
  p.cut_track = pb->cut_track;
  p.cut_moller = pb->cut_moller;
  p.cut_brems = pb->cut_brems;
  p.processes = pb->processes;
  p.lnEmin = std::log(kGridEmin);
  p.dl = std::log(kGridEmax / kGridEmin) / (kGrid - 1);
  p.inv_dl = 1.0 / p.dl;
  p.seed = pb->seed;
  p.tally_mode = pb->tally_mode;
  p.n_bins = n_bins;
  p.z0 = ctx->zb[0];
  p.zscale = (double)n_bins / (ctx->zb[L] - ctx->zb[0]);
  p.max_events = pb->max_events;
  p.hist_cap = pb->history_capacity;

  Tracks& t = p.trk;
  CREATE_CUDA(dalloc(ctx, &t.x, N));
  CREATE_CUDA(dalloc(ctx, &t.y, N));
  CREATE_CUDA(dalloc(ctx, &t.z, N));
  CREATE_CUDA(dalloc(ctx, &t.ux, N));
  CREATE_CUDA(dalloc(ctx, &t.uy, N));
  CREATE_CUDA(dalloc(ctx, &t.uz, N));
  CREATE_CUDA(dalloc(ctx, &t.E, N));
  CREATE_CUDA(dalloc(ctx, &t.nmfp, N));
  CREATE_CUDA(dalloc(ctx, &t.step, N));
  CREATE_CUDA(dalloc(ctx, &t.rpost, N));
  CREATE_CUDA(dalloc(ctx, &t.gfrac, N));
  CREATE_CUDA(dalloc(ctx, &t.gbin, N));
  CREATE_CUDA(dalloc(ctx, &t.tid, N));
  CREATE_CUDA(dalloc(ctx, &t.ctr, N));
  CREATE_CUDA(dalloc(ctx, &t.event, N));
  CREATE_CUDA(dalloc(ctx, &t.primary, N));
  CREATE_CUDA(dalloc(ctx, &t.layer, N));
  CREATE_CUDA(dalloc(ctx, &t.ptype, N));
  CREATE_CUDA(dalloc(ctx, &t.status, N));
  CREATE_CUDA(dalloc(ctx, &t.action, N));
  CREATE_CUDA(dalloc(ctx, &t.key, N));
  Ring& r = p.ring;
  CREATE_CUDA(dalloc(ctx, &r.x, C));
  CREATE_CUDA(dalloc(ctx, &r.y, C));
  CREATE_CUDA(dalloc(ctx, &r.z, C));
  CREATE_CUDA(dalloc(ctx, &r.ux, C));
  CREATE_CUDA(dalloc(ctx, &r.uy, C));
  CREATE_CUDA(dalloc(ctx, &r.uz, C));
  CREATE_CUDA(dalloc(ctx, &r.E, C));
  CREATE_CUDA(dalloc(ctx, &r.tid, C));
  CREATE_CUDA(dalloc(ctx, &r.event, C));
  CREATE_CUDA(dalloc(ctx, &r.primary, C));
  CREATE_CUDA(dalloc(ctx, &r.layer, C));
  CREATE_CUDA(dalloc(ctx, &r.ptype, C));
  CREATE_CUDA(dalloc(ctx, &p.ctl, 1));
  p.n_chunks = (N + 31) / 32;
  CREATE_CUDA(dalloc(ctx, &p.vacant, p.n_chunks));
  CREATE_CUDA(dalloc(ctx, &p.filled, p.n_chunks));
  CREATE_CUDA(dalloc(ctx, &p.tile_vacant, p.n_tiles));
  CREATE_CUDA(dalloc(ctx, &p.tile_prefix, p.n_tiles));
  CREATE_CUDA(dalloc(ctx, &p.chunk_dirty, p.n_chunks));
  CREATE_CUDA(cudaMemsetAsync(p.chunk_dirty, 1, p.n_chunks, ctx->stream));  // every key starts unset
  CREATE_CUDA(dalloc(ctx, &p.barrier, 4));
  {
    // every slot starts vacant
    std::vector<uint32_t> vac(p.n_chunks), tvac(p.n_tiles, 0);
    std::vector<unsigned long long> pre(p.n_tiles);
    for (uint32_t g = 0; g < p.n_chunks; ++g) {
      const uint64_t lo = (uint64_t)g * 32;
      vac[g] = (uint32_t)((N - lo) < 32ull ? (N - lo) : 32ull);
      tvac[g >> 3] += vac[g];
    }
    unsigned long long run = 0;
    for (uint32_t t = 0; t < p.n_tiles; ++t) {
      pre[t] = run;
      run += tvac[t];
    }
    CREATE_CUDA(cudaMemcpy(p.vacant, vac.data(), sizeof(uint32_t) * p.n_chunks, cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemcpy(p.tile_vacant, tvac.data(), sizeof(uint32_t) * p.n_tiles, cudaMemcpyHostToDevice));
    CREATE_CUDA(cudaMemcpy(p.tile_prefix, pre.data(), sizeof(unsigned long long) * p.n_tiles, cudaMemcpyHostToDevice));
  }
  CREATE_CUDA(dalloc(ctx, &p.perm, N));
  // per-(key, block) partition counts: blocks of phase A, at most one per tile
  // or the persistent grid
  const size_t max_blocks = p.n_tiles > 4096 ? p.n_tiles : 4096;
  CREATE_CUDA(dalloc(ctx, &p.block_counts, (size_t)kKeysFull * max_blocks));
  CREATE_CUDA(dalloc(ctx, &p.block_offsets, (size_t)kKeysFull * max_blocks));
  CREATE_CUDA(dalloc(ctx, &p.block_vacant, (size_t)kMaxLoopBlocks));
  CREATE_CUDA(dalloc(ctx, &p.block_quota, (size_t)kMaxLoopBlocks));
  CREATE_CUDA(dalloc(ctx, &p.block_prefix, (size_t)kMaxLoopBlocks));
  CREATE_CUDA(dalloc(ctx, &ctx->ring_state, (size_t)p.ring_capacity));
  double* d_zb = nullptr;
  int32_t* d_lmat = nullptr;
  CREATE_CUDA(dalloc(ctx, &d_zb, L + 1));
  CREATE_CUDA(dalloc(ctx, &d_lmat, L));
  CREATE_CUDA(cudaMemcpyAsync(d_zb, ctx->zb.data(), sizeof(double) * (L + 1), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int32_t> lm(ctx->layer_mat.begin(), ctx->layer_mat.end());
  CREATE_CUDA(cudaMemcpyAsync(d_lmat, lm.data(), sizeof(int32_t) * L, cudaMemcpyHostToDevice, ctx->stream));
  p.zb = d_zb;
  p.layer_mat = d_lmat;
  CREATE_CUDA(dalloc(ctx, &p.tally, (size_t)pb->max_events * n_bins));
  CREATE_CUDA(dalloc(ctx, &p.escaped, pb->max_events));
  CREATE_CUDA(dalloc(ctx, &p.event_live, pb->max_events));
  if (p.hist_cap > 0) {
    CREATE_CUDA(dalloc(ctx, &p.hist_steps, p.hist_cap));
    CREATE_CUDA(dalloc(ctx, &p.hist_secondaries, p.hist_cap));
    CREATE_CUDA(dalloc(ctx, &p.hist_escaped, p.hist_cap));
    CREATE_CUDA(dalloc(ctx, &p.hist_edep, p.hist_cap * n_bins));
  }
  CREATE_CUDA(dalloc(ctx, &p.trace, kTraceRows));

  // tables, built on the device
  double2* d_tables = nullptr;
  double* d_scratch = nullptr;
  MaterialData* d_mats = nullptr;
  CREATE_CUDA(dalloc(ctx, &d_tables, (size_t)pb->n_materials * kCols * kGrid));
  CREATE_CUDA(dalloc(ctx, &d_scratch, table_scratch_doubles(pb->n_materials)));
  CREATE_CUDA(dalloc(ctx, &d_mats, pb->n_materials));
  CREATE_CUDA(cudaMemcpyAsync(d_mats, mats.data(), sizeof(MaterialData) * mats.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
  TableBuild tb{};
  tb.n_mat = pb->n_materials;
  tb.mats = d_mats;
  tb.processes = pb->processes;
  tb.cut_moller = pb->cut_moller;
  tb.cut_brems = pb->cut_brems;
  tb.lnEmin = p.lnEmin;
  tb.dl = p.dl;
  CREATE_CUDA(build_tables(tb, d_tables, d_scratch, ctx->stream));
  p.tables = d_tables;
  double* d_mtab = nullptr;
  CREATE_CUDA(dalloc(ctx, &d_mtab, kMathTableSize));
  ctx->h_mtab.resize(kMathTableSize);
  build_math_table(ctx->h_mtab.data());
  CREATE_CUDA(cudaMemcpyAsync(d_mtab, ctx->h_mtab.data(), sizeof(double) * kMathTableSize, cudaMemcpyHostToDevice,
                              ctx->stream));
  p.mtab = d_mtab;

  // staging for primaries (bounded; larger batches go in chunks)
  ctx->stage_cap = C < (1ull << 20) ? C : (1ull << 20);
  CREATE_CUDA(dalloc(ctx, &ctx->d_stage, ctx->stage_cap));
  CREATE_CUDA(halloc(ctx, &ctx->h_stage, ctx->stage_cap));
  CREATE_CUDA(cudaEventCreateWithFlags(&ctx->stage_done, cudaEventDisableTiming));
  CREATE_CUDA(halloc(ctx, &ctx->h_ctl, 1));
  CREATE_CUDA(halloc(ctx, &ctx->h_cont, 2));
  for (auto& e : ctx->cont_ev) CREATE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  ctx->bounce_bytes = sizeof(double) * (size_t)(n_bins + 1) * 4096;
  CREATE_CUDA(halloc(ctx, &ctx->h_bounce, ctx->bounce_bytes / sizeof(double)));

  // control block
  Ctl init{};
  init.max_iterations = pb->max_iterations ? pb->max_iterations : 1000000ull;
  init.total_vacant = N;
  init.budget_end = ~0ull;
  init.cont = 0;
  CREATE_CUDA(cudaMemcpyAsync(p.ctl, &init, sizeof(Ctl), cudaMemcpyHostToDevice, ctx->stream));

  ctx->split_actions = pb->split_actions ? 1 : 0;
  const int block = pb->block_size ? pb->block_size : 256;
  CREATE_CUDA(configure_kernels(p, block, &ctx->shape));
  CREATE_CUDA(cudaStreamSynchronize(ctx->stream));
  CREATE_CUDA(cudaGetLastError());
#undef CREATE_CUDA
  *out = ctx;
  return CELER_OK;
}

celer_status celer_add_primaries(celer_ctx* ctx, uint32_t event, const celer_primary* prim, uint64_t n) {
  if (!ctx) return CELER_ERR_INVALID;
  if (n == 0) return CELER_OK;
  if (!prim) return fail(ctx, CELER_ERR_INVALID, "null primaries");
  const celer_problem& pb = ctx->prob;
  const double zmax = ctx->zb.back();
  for (uint64_t i = 0; i < n; ++i) {
    const celer_primary& q = prim[i];
    const double d2 = q.dir[0] * q.dir[0] + q.dir[1] * q.dir[1] + q.dir[2] * q.dir[2];
    const bool ok = std::isfinite(q.E) && q.E > 0.0 && q.E <= kGridEmax && std::isfinite(d2) &&
                    std::fabs(std::sqrt(d2) - 1.0) <= 1e-12 && std::fabs(q.pos[0]) <= pb.half_x &&
                    std::fabs(q.pos[1]) <= pb.half_y && q.pos[2] >= ctx->zb[0] && q.pos[2] <= zmax &&
                    (q.ptype == CELER_GAMMA || q.ptype == CELER_ELECTRON);
    if (!ok) return fail(ctx, CELER_ERR_INVALID, "primary " + std::to_string(i) + " is invalid");
  }
  if (ctx->p.hist_cap > 0 && ctx->next_history + n > ctx->p.hist_cap)
    return fail(ctx, CELER_ERR_CAPACITY, "history capacity exceeded");
  // The buffer's fill level: the host copy of the control block is current
  // if no kernel that moves the buffer's head or tail ran since it was read
  // (only this call's own pushes, which it accounts for), so a run of
  // admissions between two step runs synchronises the stream once.
  if (!ctx->ctl_fresh) {
    celer_status st = read_ctl(ctx);
    if (st != CELER_OK) return st;
  }
  const uint64_t queued = ctx->h_ctl->tail - ctx->h_ctl->head;
  if (queued + n > ctx->p.ring_capacity) return fail(ctx, CELER_ERR_CAPACITY, "initializer buffer full");

  uint64_t& tid = ctx->next_tid[event];
  for (uint64_t done = 0; done < n;) {
    const uint64_t m = (n - done) < ctx->stage_cap ? (n - done) : ctx->stage_cap;
    CELER_CUDA(ctx, cudaEventSynchronize(ctx->stage_done));
    for (uint64_t i = 0; i < m; ++i) {
      const celer_primary& q = prim[done + i];
      StagedPrimary& s = ctx->h_stage[i];
      s.E = q.E;
      s.x = q.pos[0];
      s.y = q.pos[1];
      s.z = q.pos[2];
      s.ux = q.dir[0];
      s.uy = q.dir[1];
      s.uz = q.dir[2];
      s.tid = tid++;
      s.event = event;
      s.primary = ctx->p.hist_cap > 0 ? (uint32_t)(ctx->next_history++) : 0xFFFFFFFFu;
      s.layer = layer_of(ctx->zb, q.pos[2], q.dir[2]);
      s.ptype = q.ptype;
    }
    CELER_CUDA(ctx, cudaMemcpyAsync(ctx->d_stage, ctx->h_stage, sizeof(StagedPrimary) * m, cudaMemcpyHostToDevice,
                                    ctx->stream));
    launch_push_primaries(ctx->p, ctx->d_stage, (uint32_t)m, ctx->stream);
    CELER_CUDA(ctx, cudaGetLastError());
    CELER_CUDA(ctx, cudaEventRecord(ctx->stage_done, ctx->stream));
    ctx->h_ctl->tail += m;  // the push appends exactly m entries
    done += m;
  }
  return CELER_OK;
}

celer_status celer_add_primaries_device(celer_ctx* ctx, uint32_t event, const celer_primary* dev, uint64_t n) {
  if (!ctx) return CELER_ERR_INVALID;
  ctx->ctl_fresh = false;  // the device decides whether the batch is taken
  if (n == 0) return CELER_OK;
  if (!dev) return fail(ctx, CELER_ERR_INVALID, "null primaries");
  if (n > 0xFFFFFFFFull) return fail(ctx, CELER_ERR_INVALID, "too many primaries in one call");
  if (ctx->p.hist_cap > 0 && ctx->next_history + n > ctx->p.hist_cap)
    return fail(ctx, CELER_ERR_CAPACITY, "history capacity exceeded");
  static_assert(sizeof(DevicePrimary) == sizeof(celer_primary), "primary layout");
  uint64_t& tid = ctx->next_tid[event];
  const uint32_t prim0 = ctx->p.hist_cap > 0 ? (uint32_t)ctx->next_history : 0xFFFFFFFFu;
  launch_push_device_primaries(ctx->p, reinterpret_cast<const DevicePrimary*>(dev), (uint32_t)n, event, tid, prim0,
                               ctx->stream);
  CELER_CUDA(ctx, cudaGetLastError());
  tid += n;
  if (ctx->p.hist_cap > 0) ctx->next_history += n;
  return CELER_OK;
}

celer_status celer_step(celer_ctx* ctx, celer_step_stats* stats) {
  if (!ctx) return CELER_ERR_INVALID;
  ctx->ctl_fresh = false;
  begin_policy_run(ctx);
  launch_iteration(ctx, ctx->stream, 0, 0);
  CELER_CUDA(ctx, cudaGetLastError());
  if (stats) {
    celer_status st = read_ctl(ctx);
    if (st != CELER_OK) return st;
    fill_stats(*ctx->h_ctl, stats);
    return status_from_error(ctx, ctx->h_ctl->error);
  }
  return CELER_OK;
}

celer_status celer_run_events(celer_ctx* ctx, int mode) { return celer_run_iterations(ctx, mode, 0, nullptr); }

celer_status celer_run_iterations(celer_ctx* ctx, int mode, uint64_t budget, uint64_t* done) {
  if (!ctx) return CELER_ERR_INVALID;
  ctx->ctl_fresh = false;
  if (mode < CELER_LOOP_HOST || mode > CELER_LOOP_ASYNC) return fail(ctx, CELER_ERR_INVALID, "unknown loop mode");
  if (mode == CELER_LOOP_ASYNC) {
    if (!fused_local(ctx))
      return fail(ctx, CELER_ERR_INVALID, "the asynchronous loop needs a block-pass policy (local, data) without split actions");
  }
  // iteration budget of this run; last-block tickets start from zero (an
  // aborted run could leave them set)
  launch_begin_run(ctx->p, budget, ctx->stream);
  begin_policy_run(ctx);
  CELER_CUDA(ctx, cudaGetLastError());
  if (mode == CELER_LOOP_GRAPH) {
    if (!ctx->graph_exec || ctx->graph_policy != ctx->p.policy || ctx->graph_split != ctx->split_actions) {
      celer_status st = build_graph(ctx);
      if (st != CELER_OK) return st;
    }
    CELER_CUDA(ctx, cudaGraphLaunch(ctx->graph_exec, ctx->stream));
  } else if (mode == CELER_LOOP_PERSISTENT) {
    CELER_CUDA(ctx, cudaMemsetAsync(ctx->p.barrier, 0, 4 * sizeof(unsigned int), ctx->stream));
    CELER_CUDA(ctx, launch_loop(ctx->p, ctx->shape, ctx->stream));
  } else if (mode == CELER_LOOP_ASYNC) {
    Params pa = ctx->p;
    pa.ring_state = ctx->ring_state;
    CELER_CUDA(ctx, cudaMemsetAsync(ctx->p.barrier, 0, 4 * sizeof(unsigned int), ctx->stream));
    launch_async_prepare(pa, ctx->stream);
    CELER_CUDA(ctx, cudaGetLastError());
    CELER_CUDA(ctx, launch_loop_async(pa, ctx->shape, ctx->stream));
  } else {
    // Host loop: launch batches of iterations; before each new batch, look at
    // the loop condition copied back after the batch before the previous one,
    // so that the GPU never waits for the host.
    const int batch = 8;
    int cur = 0;
    bool have_prev = false;
    const size_t hit_bytes = sizeof(double) * (size_t)ctx->p.max_events * (size_t)ctx->p.n_bins;
    for (;;) {
      for (int i = 0; i < batch; ++i) {
        launch_iteration(ctx, ctx->stream, 0, 0);
        if (ctx->hit_mode == 1) {
          CELER_CUDA(ctx, cudaMemcpyAsync(ctx->h_hits, ctx->p.tally, hit_bytes, cudaMemcpyDeviceToHost, ctx->stream));
        } else if (ctx->hit_mode == 2) {
          // a synchronous copy: the whole device waits (every stream), then the
          // host thread copies
          CELER_CUDA(ctx, cudaDeviceSynchronize());
          CELER_CUDA(ctx, cudaMemcpy(ctx->h_hits, ctx->p.tally, hit_bytes, cudaMemcpyDeviceToHost));
        }
      }
      CELER_CUDA(ctx, cudaGetLastError());
      CELER_CUDA(ctx, cudaMemcpyAsync(&ctx->h_cont[cur], &ctx->p.ctl->cont, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                      ctx->stream));
      CELER_CUDA(ctx, cudaEventRecord(ctx->cont_ev[cur], ctx->stream));
      if (have_prev) {
        const int prev = cur ^ 1;
        CELER_CUDA(ctx, cudaEventSynchronize(ctx->cont_ev[prev]));
        if (ctx->h_cont[prev] == 0u) break;
      }
      have_prev = true;
      cur ^= 1;
    }
  }
  celer_status st = read_ctl(ctx);
  if (st != CELER_OK) return st;
  if (done) *done = ctx->h_ctl->iteration - ctx->h_ctl->run_start;
  if (ctx->timing) timing_resolve(ctx);
  return status_from_error(ctx, ctx->h_ctl->error);
}

celer_status celer_read_tallies(celer_ctx* ctx, uint32_t event, double* out, uint64_t n, double* escaped) {
  if (!ctx || !out) return CELER_ERR_INVALID;
  const uint64_t nb = (uint64_t)ctx->p.n_bins;
  if (n != nb) return fail(ctx, CELER_ERR_INVALID, "n must equal the bin count");
  const uint32_t row = event % ctx->p.max_events;
  CELER_CUDA(ctx, cudaMemcpyAsync(ctx->h_bounce, ctx->p.tally + (size_t)row * nb, sizeof(double) * nb,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(ctx->h_bounce + nb, ctx->p.escaped + row, sizeof(double), cudaMemcpyDeviceToHost,
                                  ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::memcpy(out, ctx->h_bounce, sizeof(double) * nb);
  if (escaped) *escaped = ctx->h_bounce[nb];
  return CELER_OK;
}

celer_status celer_reset_event(celer_ctx* ctx, uint32_t event) {
  if (!ctx) return CELER_ERR_INVALID;
  const uint32_t row = event % ctx->p.max_events;
  const size_t nb = (size_t)ctx->p.n_bins;
  CELER_CUDA(ctx, cudaMemsetAsync(ctx->p.tally + row * nb, 0, sizeof(double) * nb, ctx->stream));
  CELER_CUDA(ctx, cudaMemsetAsync(ctx->p.escaped + row, 0, sizeof(double), ctx->stream));
  CELER_CUDA(ctx, cudaMemsetAsync(ctx->p.event_live + row, 0, sizeof(unsigned), ctx->stream));
  ctx->next_tid.erase(event);
  return CELER_OK;
}

celer_status celer_event_live(celer_ctx* ctx, uint32_t event, uint64_t* live) {
  if (!ctx || !live) return CELER_ERR_INVALID;
  const uint32_t row = event % ctx->p.max_events;
  unsigned* h = ctx->h_cont;
  CELER_CUDA(ctx, cudaMemcpyAsync(h, ctx->p.event_live + row, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *live = h[0];
  return CELER_OK;
}

celer_status celer_read_event_live(celer_ctx* ctx, uint32_t first_row, uint32_t count, uint32_t* host_out) {
  if (!ctx || !host_out) return CELER_ERR_INVALID;
  if ((uint64_t)first_row + count > ctx->p.max_events) return fail(ctx, CELER_ERR_INVALID, "row range out of bounds");
  if (count == 0) return CELER_OK;
  CELER_CUDA(ctx, cudaMemcpyAsync(host_out, ctx->p.event_live + first_row, sizeof(uint32_t) * count,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return CELER_OK;
}

celer_status celer_read_history(celer_ctx* ctx, uint64_t first, uint64_t count, celer_history* out, double* edep_out) {
  if (!ctx || (!out && !edep_out)) return CELER_ERR_INVALID;
  if (first + count > ctx->p.hist_cap) return fail(ctx, CELER_ERR_INVALID, "history range out of bounds");
  const size_t nb = (size_t)ctx->p.n_bins;
  const size_t chunk_rows = ctx->bounce_bytes / (sizeof(double) * (nb + 1)) - 1;
  std::vector<unsigned long long> steps(count), secs(count);
  std::vector<double> esc(count);
  CELER_CUDA(ctx, cudaMemcpyAsync(steps.data(), ctx->p.hist_steps + first, sizeof(unsigned long long) * count,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(secs.data(), ctx->p.hist_secondaries + first, sizeof(unsigned long long) * count,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(esc.data(), ctx->p.hist_escaped + first, sizeof(double) * count,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (uint64_t done = 0; done < count;) {
    const uint64_t m = (count - done) < chunk_rows ? (count - done) : chunk_rows;
    CELER_CUDA(ctx, cudaMemcpyAsync(ctx->h_bounce, ctx->p.hist_edep + (first + done) * nb, sizeof(double) * m * nb,
                                    cudaMemcpyDeviceToHost, ctx->stream));
    CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (uint64_t i = 0; i < m; ++i) {
      double sum = 0.0;
      for (size_t b = 0; b < nb; ++b) sum += ctx->h_bounce[i * nb + b];
      if (out) {
        celer_history& h = out[done + i];
        h.steps = steps[done + i];
        h.secondaries = secs[done + i];
        h.escaped = esc[done + i];
        h.edep = sum;
      }
      if (edep_out) std::memcpy(edep_out + (done + i) * nb, ctx->h_bounce + i * nb, sizeof(double) * nb);
    }
    done += m;
  }
  return CELER_OK;
}

celer_status celer_get_problem(const celer_ctx* ctx, celer_problem* out) {
  if (!ctx || !out) return CELER_ERR_INVALID;
  *out = ctx->prob;
  out->sort_policy = ctx->p.policy;
  return CELER_OK;
}

celer_status celer_get_stats(celer_ctx* ctx, celer_step_stats* out) {
  if (!ctx || !out) return CELER_ERR_INVALID;
  celer_status st = read_ctl(ctx);
  if (st != CELER_OK) return st;
  fill_stats(*ctx->h_ctl, out);
  return CELER_OK;
}

celer_status celer_read_loop_profile(celer_ctx* ctx, uint64_t* cycles_out, int n) {
  if (!ctx || !cycles_out || n < 1) return CELER_ERR_INVALID;
  celer_status st = read_ctl(ctx);
  if (st != CELER_OK) return st;
  const Ctl& c = *ctx->h_ctl;
  const unsigned long long all[10] = {c.phase_cycles[0], c.phase_cycles[1], c.phase_cycles[2], c.phase_cycles[3],
                                      c.max_total[0], c.max_total[1], c.max_total[2], c.max_total[3],
                                      c.book_total[0], c.book_total[1]};
  for (int k = 0; k < n; ++k) cycles_out[k] = k < 10 ? all[k] : 0;
  return CELER_OK;
}

celer_status celer_set_hit_readout(celer_ctx* ctx, int mode, double* host_hits, uint64_t n) {
  if (!ctx || mode < 0 || mode > 2) return CELER_ERR_INVALID;
  if (mode != 0 && (!host_hits || n < (uint64_t)ctx->p.max_events * (uint64_t)ctx->p.n_bins))
    return fail(ctx, CELER_ERR_INVALID, "hit buffer missing or smaller than max_events x bins");
  ctx->hit_mode = mode;
  ctx->h_hits = mode ? host_hits : nullptr;
  return CELER_OK;
}

celer_status celer_set_parent_reuse(celer_ctx* ctx, int on) {
  if (!ctx) return CELER_ERR_INVALID;
  ctx->p.reuse_parent = on ? 1 : 0;
  destroy_graph(ctx);  // captured with the old parameters
  return CELER_OK;
}

celer_status celer_set_async_warps(celer_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) return CELER_ERR_INVALID;
  ctx->p.async_warps = on;
  return CELER_OK;
}

celer_status celer_set_grid_blocks(celer_ctx* ctx, int blocks) {
  if (!ctx || blocks < 0) return CELER_ERR_INVALID;
  LaunchShape sh{};
  CELER_CUDA(ctx, configure_kernels(ctx->p, ctx->shape.block, &sh));
  if (blocks > 0) {
    sh.loop_grid = std::min(sh.loop_grid, blocks);
    sh.tile_grid = std::min(sh.tile_grid, blocks);
    sh.step_grid = std::min(sh.step_grid, blocks);
    sh.along_grid = std::min(sh.along_grid, blocks);
    sh.post_grid = std::min(sh.post_grid, blocks);
  }
  ctx->shape = sh;
  destroy_graph(ctx);  // captured with the old grids
  return CELER_OK;
}

celer_status celer_set_split_actions(celer_ctx* ctx, int split) {
  if (!ctx) return CELER_ERR_INVALID;
  ctx->split_actions = split ? 1 : 0;
  ctx->prob.split_actions = ctx->split_actions;
  return CELER_OK;
}

celer_status celer_set_sort_policy(celer_ctx* ctx, int policy) {
  if (!ctx || policy < 0 || policy >= kPolicyCount) return CELER_ERR_INVALID;
  ctx->p.policy = policy;
  ctx->p.n_keys = keys_of(policy);
  // stored keys belong to the previous policy: rewrite them all at the next step
  CELER_CUDA(ctx, cudaMemsetAsync(ctx->p.chunk_dirty, 1, ctx->p.n_chunks, ctx->stream));
  ctx->prob.sort_policy = policy;
  return CELER_OK;
}

celer_status celer_read_trace(celer_ctx* ctx, celer_trace_row* out, uint64_t n_max, uint64_t* n_out) {
  if (!ctx || !out || !n_out) return CELER_ERR_INVALID;
  celer_status st = read_ctl(ctx);
  if (st != CELER_OK) return st;
  const uint64_t total = ctx->h_ctl->trace_count;
  uint64_t n = total < (uint64_t)kTraceRows ? total : (uint64_t)kTraceRows;
  if (n > n_max) n = n_max;
  std::vector<TraceRow> rows(kTraceRows);
  CELER_CUDA(ctx, cudaMemcpyAsync(rows.data(), ctx->p.trace, sizeof(TraceRow) * kTraceRows, cudaMemcpyDeviceToHost,
                                  ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (uint64_t i = 0; i < n; ++i) {
    const TraceRow& r = rows[(total - n + i) % kTraceRows];
    out[i].iteration = r.iteration;
    out[i].alive = r.alive;
    out[i].queued = r.queued;
    out[i].steps = r.steps;
    for (int k = 0; k < 16; ++k) out[i].action_count[k] = r.action_count[k];
  }
  *n_out = n;
  return CELER_OK;
}

celer_status celer_enable_kernel_timing(celer_ctx* ctx, int enable) {
  if (!ctx) return CELER_ERR_INVALID;
  if (enable && ctx->t_start.empty()) {
    ctx->t_start.resize(kTimingPool);
    ctx->t_stop.resize(kTimingPool);
    ctx->t_kid.resize(kTimingPool);
    for (int i = 0; i < kTimingPool; ++i) {
      CELER_CUDA(ctx, cudaEventCreate(&ctx->t_start[i]));
      CELER_CUDA(ctx, cudaEventCreate(&ctx->t_stop[i]));
    }
  }
  timing_resolve(ctx);
  for (int k = 0; k < KID_COUNT; ++k) {
    ctx->t_total_ms[k] = 0.0;
    ctx->t_launches[k] = 0;
  }
  ctx->timing = enable != 0;
  return CELER_OK;
}

celer_status celer_kernel_timing(celer_ctx* ctx, const char** names, double* total_ms, uint64_t* launches, int n_max,
                                 int* n_out) {
  if (!ctx || !n_out) return CELER_ERR_INVALID;
  timing_resolve(ctx);
  int n = 0;
  for (int k = 0; k < KID_COUNT && n < n_max; ++k, ++n) {
    if (names) names[n] = kernel_name(k);
    if (total_ms) total_ms[n] = ctx->t_total_ms[k];
    if (launches) launches[n] = ctx->t_launches[k];
  }
  *n_out = n;
  return CELER_OK;
}

celer_status celer_debug_partition(celer_ctx* ctx, uint8_t* keys_out, uint32_t* perm_out, uint32_t* offsets_out,
                                   int* n_keys, int* n_blocks) {
  if (!ctx || !keys_out || !perm_out || !offsets_out || !n_keys || !n_blocks) return CELER_ERR_INVALID;
  if (!policy_sorted(ctx->p.policy)) return fail(ctx, CELER_ERR_STATE, "no grid-wide partition under this policy");
  celer_status st = read_ctl(ctx);
  if (st != CELER_OK) return st;
  const uint32_t N = ctx->p.n_slots;
  CELER_CUDA(ctx, cudaMemcpyAsync(keys_out, ctx->p.trk.key, N, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(perm_out, ctx->p.perm, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *n_keys = ctx->p.n_keys;
  *n_blocks = (int)ctx->h_ctl->part_blocks;
  for (int k = 0; k <= ctx->p.n_keys; ++k) offsets_out[k] = ctx->h_ctl->offsets[k];
  return CELER_OK;
}

celer_status celer_debug_lane_counts(uint64_t* host_out, int n_max, int* n_out) {
  if (!host_out || !n_out || n_max < 0) return CELER_ERR_INVALID;
  *n_out = 0;
  const int n = n_max < celer::kLaneSites ? n_max : celer::kLaneSites;
  std::vector<unsigned long long> v((size_t)celer::kLaneValues * celer::kLaneSites, 0ull);
  const cudaError_t e = celer::read_lane_counts(v.data(), celer::kLaneSites);
  if (e == cudaErrorNotSupported) return CELER_ERR_STATE;
  if (e != cudaSuccess) return CELER_ERR_CUDA;
  for (int k = 0; k < celer::kLaneValues * n; ++k) host_out[k] = v[k];
  *n_out = n;
  return CELER_OK;
}

celer_status celer_debug_slots(celer_ctx* ctx, uint8_t* status_out, uint8_t* ptype_out, int* n_blocks) {
  if (!ctx || !status_out || !ptype_out || !n_blocks) return CELER_ERR_INVALID;
  const uint32_t N = ctx->p.n_slots;
  CELER_CUDA(ctx, cudaMemcpyAsync(status_out, ctx->p.trk.status, N, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(ptype_out, ctx->p.trk.ptype, N, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *n_blocks = ctx->shape.loop_grid;
  return CELER_OK;
}

celer_status celer_debug_tracks(celer_ctx* ctx, uint64_t* tid_out, uint32_t* event_out, int32_t* layer_out,
                                double* state_out) {
  if (!ctx || !tid_out || !event_out || !layer_out || !state_out) return CELER_ERR_INVALID;
  const size_t N = ctx->p.n_slots;
  const Tracks& t = ctx->p.trk;
  CELER_CUDA(ctx, cudaMemcpyAsync(tid_out, t.tid, sizeof(uint64_t) * N, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(event_out, t.event, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaMemcpyAsync(layer_out, t.layer, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, ctx->stream));
  const double* cols[7] = {t.x, t.y, t.z, t.ux, t.uy, t.uz, t.E};
  for (int k = 0; k < 7; ++k)
    CELER_CUDA(ctx, cudaMemcpyAsync(state_out + (size_t)k * N, cols[k], sizeof(double) * N, cudaMemcpyDeviceToHost,
                                    ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return CELER_OK;
}

celer_status celer_debug_barrier_timeout(int blocks, int absent_block, uint64_t timeout_cycles, uint32_t* error_bits,
                                         uint32_t* abort_word) {
  if (blocks < 2 || blocks > 8 || absent_block < -1 || absent_block >= blocks || timeout_cycles == 0 ||
      timeout_cycles > 4000000000ull || !error_bits || !abort_word)
    return CELER_ERR_INVALID;
  Ctl* d_ctl = nullptr;
  unsigned* d_bar = nullptr;
  if (cudaMalloc(&d_ctl, sizeof(Ctl)) != cudaSuccess) return CELER_ERR_CUDA;
  if (cudaMalloc(&d_bar, 4 * sizeof(unsigned)) != cudaSuccess) {
    cudaFree(d_ctl);
    return CELER_ERR_CUDA;
  }
  celer_status st = CELER_OK;
  if (cudaMemset(d_ctl, 0, sizeof(Ctl)) != cudaSuccess || cudaMemset(d_bar, 0, 4 * sizeof(unsigned)) != cudaSuccess)
    st = CELER_ERR_CUDA;
  Params p{};
  p.ctl = d_ctl;
  p.barrier = d_bar;
  if (st == CELER_OK && (launch_barrier_probe(p, blocks, absent_block, (long long)timeout_cycles, 0) != cudaSuccess ||
                         cudaDeviceSynchronize() != cudaSuccess))
    st = CELER_ERR_CUDA;
  Ctl h{};
  unsigned bar[4] = {0, 0, 0, 0};
  if (st == CELER_OK && (cudaMemcpy(&h, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess ||
                         cudaMemcpy(bar, d_bar, sizeof(bar), cudaMemcpyDeviceToHost) != cudaSuccess))
    st = CELER_ERR_CUDA;
  cudaFree(d_ctl);
  cudaFree(d_bar);
  if (st != CELER_OK) return st;
  *error_bits = h.error;
  *abort_word = bar[2];
  return (h.error & ERR_BARRIER_TIMEOUT) ? CELER_ERR_TIMEOUT : CELER_OK;
}

celer_status celer_debug_queue_wait(int which, uint64_t timeout_cycles, uint32_t* error_bits, uint32_t* abort_word) {
  if (which < 0 || which > 3 || timeout_cycles == 0 || timeout_cycles > 4000000000ull || !error_bits || !abort_word)
    return CELER_ERR_INVALID;
  Ctl* d_ctl = nullptr;
  unsigned* d_bar = nullptr;
  uint32_t* d_state = nullptr;
  celer_status st = CELER_OK;
  if (cudaMalloc(&d_ctl, sizeof(Ctl)) != cudaSuccess || cudaMalloc(&d_bar, 4 * sizeof(unsigned)) != cudaSuccess ||
      cudaMalloc(&d_state, sizeof(uint32_t)) != cudaSuccess)
    st = CELER_ERR_CUDA;
  if (st == CELER_OK && (cudaMemset(d_ctl, 0, sizeof(Ctl)) != cudaSuccess ||
                         cudaMemset(d_bar, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
                         cudaMemset(d_state, 0, sizeof(uint32_t)) != cudaSuccess))
    st = CELER_ERR_CUDA;
  Params p{};
  p.ctl = d_ctl;
  p.barrier = d_bar;
  p.ring_state = d_state;  // a one-entry buffer: entry 0, lap 0
  p.ring_capacity = 1;
  p.ring_mask = 0;
  if (st == CELER_OK && (launch_queue_wait_probe(p, which, (long long)timeout_cycles, 0) != cudaSuccess ||
                         cudaDeviceSynchronize() != cudaSuccess))
    st = CELER_ERR_CUDA;
  Ctl h{};
  unsigned bar[4] = {0, 0, 0, 0};
  if (st == CELER_OK && (cudaMemcpy(&h, d_ctl, sizeof(Ctl), cudaMemcpyDeviceToHost) != cudaSuccess ||
                         cudaMemcpy(bar, d_bar, sizeof(bar), cudaMemcpyDeviceToHost) != cudaSuccess))
    st = CELER_ERR_CUDA;
  if (d_ctl) cudaFree(d_ctl);
  if (d_bar) cudaFree(d_bar);
  if (d_state) cudaFree(d_state);
  if (st != CELER_OK) return st;
  *error_bits = h.error;
  *abort_word = bar[2];
  return (h.error & ERR_BARRIER_TIMEOUT) ? CELER_ERR_TIMEOUT : CELER_OK;
}

celer_status celer_debug_table(celer_ctx* ctx, int mat, int col, double* out) {
  if (!ctx || !out || mat < 0 || mat >= ctx->p.n_materials || col < 0 || col >= kCols) return CELER_ERR_INVALID;
  std::vector<double2> v(kGrid);
  CELER_CUDA(ctx, cudaMemcpyAsync(v.data(), ctx->p.tables + ((size_t)mat * kCols + col) * kGrid,
                                  sizeof(double2) * kGrid, cudaMemcpyDeviceToHost, ctx->stream));
  CELER_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < kGrid; ++i) out[i] = v[i].x;
  return CELER_OK;
}

}  // extern "C"
