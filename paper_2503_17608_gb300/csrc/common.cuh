// Device-side data layout and launch parameters of the step-based transport
// loop (Sec. 2 of the paper: struct-of-arrays track state, a separate buffer
// of track initializers, one kernel per action).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace celer {

constexpr int kGrid = 200;          // log-spaced energy grid points
constexpr double kGridEmin = 1e-3;  // MeV
constexpr double kGridEmax = 1e4;   // MeV
constexpr int kCols = 6;            // device table columns per material
constexpr int kMaxMaterials = 8;
constexpr int kMaxLayers = 1024;
constexpr int kMaxKeys = 16;
constexpr int kTile = 256;          // slots per tile: partition, initializer and step-limit work unit
constexpr int kTraceRows = 1 << 16;
constexpr int kMaxLoopBlocks = 4096;  // grid of the persistent loop and the block-local launches

// device table columns
enum Col : int { COL_COMPTON = 0, COL_PE, COL_PAIR, COL_MOLLER, COL_BREMS, COL_RANGE };

enum ProcBits : int {
  PROC_COMPTON = 1, PROC_PE = 2, PROC_PAIR = 4, PROC_MOLLER = 8, PROC_BREMS = 16, PROC_ELOSS = 32
};

enum PType : uint8_t { GAMMA = 0, ELECTRON = 1, POSITRON = 2 };
enum Status : uint8_t { VACANT = 0, ALIVE = 1, DEFERRED = 2 };

// Next action of a track, chosen by the step-limit kernel: the
// geometric/range limits handled by the along-step kernels, then the
// discrete interactions handled by one kernel each.
enum Action : uint8_t {
  A_NONE = 0,
  A_ZUP,      // crosses the upper z-plane of its layer
  A_ZDOWN,    // crosses the lower z-plane of its layer
  A_SIDE,     // leaves through a side plane
  A_RANGE,    // range-limited step
  A_TRAPPED,  // no finite step limit: ends in place
  A_COMPTON,
  A_PE,
  A_PAIR,
  A_MOLLER,
  A_BREMS,
  A_FIELD,    // a field step cut at the substep cap: no crossing, no interaction
  A_COUNT
};

// Partition keys of the ACTION_TYPE policy: (particle type, next action).
// Geometric and range-limited steps first, interactions after them, vacant
// last, so that the along-step range (all live keys) and the interaction
// range are each one contiguous interval of the partition.
enum Key : uint8_t {
  K_G_GEOM = 0, K_E_GEOM, K_E_RANGE,
  K_G_COMPTON, K_G_PE, K_G_PAIR, K_E_MOLLER, K_E_BREMS,
  K_VACANT_FULL = 8
};
constexpr int kFirstInteractionKey = K_G_COMPTON;
constexpr int kKeysFull = 9;
// Keys of the ACTION policy (along-step action only).
enum KeyAlong : uint8_t { KA_NEUTRAL = 0, KA_CHARGED = 1, KA_VACANT = 2 };
constexpr int kKeysAlong = 3;

// NONE: slot order. ACTION / ACTION_TYPE: a grid-wide partition of the live
// slots by key before the step phase. LOCAL: no grid-wide partition; each
// block groups its own live tracks by action and particle type in shared
// memory during the step phase. DATA: no reindexing; each block places its
// neutral initializers at the low end of its slots and its charged ones at
// the high end (Sec. 3.2) and steps its chunks in slot order.
enum Policy : int { POLICY_NONE = 0, POLICY_ACTION = 1, POLICY_ACTION_TYPE = 2, POLICY_LOCAL = 3, POLICY_DATA = 4 };
constexpr int kPolicyCount = 5;
// LOCAL and DATA run one pass per block and iteration (block-owned chunks).
__host__ __device__ __forceinline__ bool block_pass(int policy) {
  return policy == POLICY_LOCAL || policy == POLICY_DATA;
}
__host__ __device__ __forceinline__ bool global_partition(int policy) {
  return policy == POLICY_ACTION || policy == POLICY_ACTION_TYPE;
}

enum ErrorBits : uint32_t { ERR_RING_OVERFLOW = 1u, ERR_NO_PROGRESS = 2u, ERR_ITERATIONS = 4u, ERR_SAMPLING = 8u,
                            ERR_PRIMARIES_REJECTED = 16u, ERR_BARRIER_TIMEOUT = 32u,
                            ERR_VACANCY = 64u };

struct Tracks {
  double *x, *y, *z, *ux, *uy, *uz, *E, *nmfp, *step, *rpost;
  double* gfrac;   // a photon's grid position in ln E (bin, fraction), kept
  int32_t* gbin;   // from the step that sampled its n_mfp (same energy since)
  unsigned long long* tid;
  uint32_t *ctr, *event, *primary;
  int32_t* layer;
  uint8_t *ptype, *status, *action, *key;
};

struct Ring {
  double *x, *y, *z, *ux, *uy, *uz, *E;
  unsigned long long* tid;
  uint32_t *event, *primary;
  int32_t* layer;
  uint8_t* ptype;
};

// Device-resident loop control. Ring indices are monotonic counters; the
// entry of index i lives at i & ring_mask.
struct Ctl {
  unsigned long long head, tail;
  unsigned long long alive;          // slots holding a live or deferred track
  unsigned long long steps_total;
  unsigned long long steps_iter;
  unsigned long long iteration;
  unsigned long long max_iterations;
  unsigned long long budget_end;     // the current run stops when iteration reaches this
  unsigned long long run_start;      // iteration count when the current run began
  unsigned int action_count[kMaxKeys];
  unsigned int key_total[kMaxKeys];
  unsigned int offsets[kMaxKeys + 1];
  unsigned int defer;                // 1: secondary-producing kernels postpone this iteration
  unsigned int n_deferred;
  unsigned int error;
  unsigned int cont;                 // 1 while alive + queued > 0
  unsigned int stall;                // consecutive iterations without progress
  unsigned int done_a, done_c;       // last-block tickets of the fill/step-limit and step phases
  unsigned long long total_vacant;   // vacant slots (scanned at the end of an iteration)
  unsigned long long filled_total;   // slots filled in the current iteration
  unsigned int part_blocks;          // blocks that counted the last partition (chunk g: block g mod it)
  unsigned long long trace_count;
  unsigned long long last_steps_iter;          // copies of the last finished iteration's counters
  unsigned int last_n_deferred;
  unsigned int last_action_count[kMaxKeys];
  // persistent loop profile (SM cycles): per phase as seen by block 0 (work +
  // barrier), sum over iterations of the slowest block's work, and the
  // last-block bookkeeping of the fill/step-limit and step phases
  unsigned long long phase_cycles[4];
  unsigned long long iter_max[2][4];
  unsigned long long max_total[4];
  unsigned long long book_total[2];
  // block-local policy (one pass per block and iteration): initializers the
  // next iteration takes, its secondary-buffer verdict, the last-block ticket
  // of the per-block vacancy scan, and the grid that scan was made for
  unsigned long long fill_take;
  unsigned int defer_local;
  unsigned int done_p;
  unsigned int local_blocks;
  // asynchronous block loop: tracks ended since the buffer's first entry
  // (head - alive at the start of the run; the run is over when it reaches
  // tail), the most block passes any block ran, and the exit ticket
  unsigned long long finished;
  unsigned long long avail;          // written entries not yet claimed by a reader (may dip below 0 briefly)
  unsigned long long async_passes;
  unsigned int done_x;
};

struct TraceRow {
  unsigned long long iteration, alive, queued, steps;
  unsigned int action_count[kMaxKeys];
};

struct Params {
  // state
  Tracks trk;
  Ring ring;
  Ctl* ctl;
  uint32_t n_slots;
  uint32_t n_tiles;        // ceil(n_slots / kTile)
  unsigned long long ring_mask;
  unsigned long long ring_capacity;
  uint32_t n_chunks;       // ceil(n_slots / 32): warp-tiles of the fill / step-limit phase
  uint32_t* vacant;        // vacant slots per chunk, n_chunks (kept current by every release)
  uint32_t* filled;        // slots filled per chunk in the current iteration, n_chunks
  uint32_t* tile_vacant;   // vacant slots per 256-slot tile, n_tiles
  unsigned long long* tile_prefix;  // vacant slots before each tile, n_tiles (scanned once per iteration)
  uint8_t* chunk_dirty;    // 1 if the chunk's stored keys may name live keys (n_chunks); after
                           // phase A: 1 exactly for the chunks holding live keys
  unsigned int* barrier;   // grid barrier state of the persistent loop: count, generation, abort
  uint32_t* block_vacant;  // block-local policy: vacant slots of each block's chunks (grid of the loop)
  uint32_t* block_quota;   // initializers each block takes in the next iteration (level filling)
  unsigned long long* block_prefix;  // exclusive scan of the quotas: each block's first initializer
  uint32_t* ring_state;    // asynchronous block loop only (null otherwise): per buffer entry, 2 lap + 1
                           // once written and 2 lap + 2 once read, lap = index / capacity
  // partition
  int policy;
  int n_keys;
  uint32_t* perm;          // n_slots
  uint32_t* block_counts;  // live-key counts per counting block, (n_keys - 1) x blocks, key major
  uint32_t* block_offsets; // their exclusive scan: each block's first position per key
  // geometry
  int n_layers;
  int n_materials;
  const double* zb;        // n_layers + 1
  const int32_t* layer_mat;
  double hx, hy, Bz;
  // physics
  double cut_track, cut_moller, cut_brems;
  int processes;
  int reuse_parent;        // 1: a pair's first photon starts in the parent's slot (Sec. 3.2)
  int field_cap;           // 0: exact helix; > 0: Runge-Kutta substeps, at most this many per step
  int async_warps;         // asynchronous loop, block-local policy: 1 per-warp scheduling, 0 block passes
  const double2* tables;   // [mat][col][kGrid] (value, next - value)
  const double* mtab;      // log/exp reduction tables (fastmath.cuh)
  double lnEmin, inv_dl, dl;
  uint32_t seed;
  // tallies
  int tally_mode;
  int n_bins;
  double z0, zscale;
  uint32_t max_events;
  double* tally;           // max_events * n_bins
  double* escaped;         // max_events
  unsigned int* event_live;  // max_events
  // per-primary history
  unsigned long long hist_cap;
  unsigned long long* hist_steps;
  unsigned long long* hist_secondaries;
  double* hist_escaped;
  double* hist_edep;       // hist_cap * n_bins
  TraceRow* trace;
};

// ---- active-lane counters (diagnostic build only)
// Built with -DCELER_LANE_COUNTERS, every site below counts its warp-level
// visits and the lanes active at each visit (for the per-warp piece sites,
// the tracks the piece holds), so that the mean active lanes per site show
// how much each sort policy cuts divergence. The counters are spread over 16
// copies by block to keep the atomics apart. The product build compiles every
// site to nothing.
enum LaneSite : int {
  LS_PIECE = 0,        // + K_* key: per-warp pieces of the asynchronous loop (tracks claimed)
  LS_FILL = 8,         // per-warp fills of the asynchronous loop (initializers taken)
  LS_STEP_LIMIT = 9,   // step limit of a live track
  LS_ALONG = 10,       // along-step
  LS_COMPTON = 11, LS_PE = 12, LS_PAIR = 13, LS_MOLLER = 14, LS_BREMS = 15,
  LS_COMPTON_TRY = 16, // one rejection attempt of the Compton sampler
  LS_MOLLER_TRY = 17,  // one rejection attempt of the Moller sampler
  LS_HELIX_SIDE = 18,  // side-plane distance along the helix
  LS_IDLE = 19,        // per-warp loop rounds of the asynchronous loop that found nothing to do
  LS_T_PHOTON = 20,    // photon crossing pieces timed in three parts: choice and claim, the
                       // step, the next step limit and requeue (20, 21, 22)
  LS_T_ELECTRON = 23,  // the same for electron crossing pieces (23, 24, 25)
  LS_T_LIMIT = 26,     // the step limit of a photon timed in five parts: the state loads, the
                       // grid position (logarithm), the cross sections, the distances to the
                       // planes, the rest with the stores (26-30)
  LS_T_PUSH = 31,      // queueing a track by its next kind (per-warp loop)
  LS_T_COMPTON = 32,   // Compton pieces timed in three parts as the crossings (32, 33, 34)
  kLaneSites = 35
};
constexpr int kLaneCopies = 16;
constexpr int kLaneValues = 3;  // per site: visits, lanes, SM cycles (where timed)
#ifdef CELER_LANE_COUNTERS
static __device__ unsigned long long g_lane_counts[kLaneCopies][kLaneSites][kLaneValues];
__device__ __forceinline__ void lane_site(int site) {
  const unsigned m = __activemask();
  if ((int)(threadIdx.x & 31u) == __ffs(m) - 1) {
    unsigned long long* c = g_lane_counts[blockIdx.x % kLaneCopies][site];
    atomicAdd(c, 1ull);
    atomicAdd(c + 1, (unsigned long long)__popc(m));
  }
}
__device__ __forceinline__ void lane_site_n(int site, unsigned n) {  // one thread, n lanes of work
  unsigned long long* c = g_lane_counts[blockIdx.x % kLaneCopies][site];
  atomicAdd(c, 1ull);
  atomicAdd(c + 1, (unsigned long long)n);
}
__device__ __forceinline__ void lane_cycles(int site, long long cycles) {  // one thread
  atomicAdd(&g_lane_counts[blockIdx.x % kLaneCopies][site][2], (unsigned long long)cycles);
}
#define CELER_LANES(site) ::celer::lane_site(site)
#define CELER_LANES_N(site, n) ::celer::lane_site_n((site), (n))
#define CELER_LANE_CLOCK() clock64()
#define CELER_LANE_CYCLES(site, c) ::celer::lane_cycles((site), (c))
// the lanes here gathered, the time since mark t recorded at site, t reset
#define CELER_LANE_MARK(site, t)                                     \
  do {                                                               \
    const unsigned m_ = __activemask();                              \
    __syncwarp(m_);                                                  \
    const long long n_ = clock64();                                  \
    if ((int)(threadIdx.x & 31u) == __ffs(m_) - 1) {                 \
      ::celer::lane_site_n((site), (unsigned)__popc(m_));            \
      ::celer::lane_cycles((site), n_ - (t));                        \
    }                                                                \
    (t) = n_;                                                        \
  } while (0)
#else
#define CELER_LANES(site) ((void)0)
#define CELER_LANES_N(site, n) ((void)0)
#define CELER_LANE_CLOCK() 0ll
#define CELER_LANE_CYCLES(site, c) ((void)0)
#define CELER_LANE_MARK(site, t) ((void)0)
#endif

}  // namespace celer
