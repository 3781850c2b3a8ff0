// Kernels of one step iteration (Sec. 2 of the paper): fill vacant slots from
// the track-initializer buffer, compute each track's step limit and next
// action, reorder slot indices by action (Sec. 3.1), propagate, and apply the
// discrete interactions, pushing secondaries back into the buffer.
//
// Every action kernel is persistent: a grid sized to the GPU (a multiple of
// the SM count) strides over its work range, which is either all slots with
// masking (policy NONE) or one contiguous range of the partition read from
// device memory (sorted policies), so that no host round trip is needed to
// size a launch.
#include <cooperative_groups.h>
#include <cooperative_groups/scan.h>

#include "launch.h"
#include "physics.cuh"

namespace cg = cooperative_groups;

namespace celer {

namespace {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint32_t row_of(const Params& p, uint32_t ev) { return ev % p.max_events; }

__device__ __forceinline__ int tally_bin(const Params& p, int layer, double z) {
  if (p.tally_mode == 1) return layer;
  int b = __double2int_rd((z - p.z0) * p.zscale);  // (int)floor, one conversion
  return b < 0 ? 0 : (b > p.n_bins - 1 ? p.n_bins - 1 : b);
}

__device__ __forceinline__ void deposit(const Params& p, uint32_t ev, uint32_t prim, int layer, double z, double e) {
  if (((unsigned long long)__double_as_longlong(e) << 1) == 0ull) return;  // e == +-0 on the bits
  const int b = tally_bin(p, layer, z);
  atomicAdd(&p.tally[(size_t)row_of(p, ev) * p.n_bins + b], e);
  if (prim < p.hist_cap) atomicAdd(&p.hist_edep[(size_t)prim * p.n_bins + b], e);
}

__device__ __forceinline__ void escape(const Params& p, uint32_t ev, uint32_t prim, double e) {
  atomicAdd(&p.escaped[row_of(p, ev)], e);
  if (prim < p.hist_cap) atomicAdd(&p.hist_escaped[prim], e);
}

__device__ __forceinline__ void release(const Params& p, uint32_t slot, uint32_t ev) {
  p.trk.status[slot] = VACANT;
  p.trk.action[slot] = A_NONE;
  atomicSub(&p.event_live[row_of(p, ev)], 1u);
  atomicAdd(&p.vacant[slot >> 5], 1u);
  atomicAdd(&p.tile_vacant[slot >> 8], 1u);
}

// Warp-sum a per-thread counter and add it to a device counter (negated if
// asked). Called by whole warps at kernel end.
__device__ __forceinline__ void flush_counter(unsigned long long* dst, unsigned long long v, bool negate) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v != 0) atomicAdd(dst, negate ? (0ull - v) : v);
}

// ---- the initializer buffer as a concurrent queue (asynchronous block loop)
//
// Entry i of the buffer (stored at i & ring_mask) carries a state word: with
// lap = i / capacity, 2 lap means free for the writer of i, 2 lap + 1 written
// and not yet read, 2 lap + 2 read (free for the writer of i + capacity).
// A writer reserves i on the tail only while i < head + capacity, with the
// head read just before: by compare-and-swap, or by one atomic add while the
// room exceeds what every thread of the grid could reserve at once (should
// the buffer still fill within that window, the writer's wait below for the
// entry's reader is bounded like every other). So the reader of
// i - capacity has claimed its entry already, and every wait is for a claim
// or reservation that the other side completes without waiting on the
// waiter: reads and writes follow their claims and reservations directly.
// Readers claim written entries on an availability count (avail) before
// taking their indices from the head, so the head never passes the tail.
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* a) {
  unsigned v;
  asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* a) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(a) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* a, unsigned v) {
  asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ring_lap_code(const Params& p, unsigned long long index) {
  return (unsigned)(index >> __popcll(p.ring_mask)) * 2u;
}
// Bounded wait of one thread for entry `index` to reach state `code`. After
// `timeout` cycles (~1 s by default), or if another wait gave up first (abort
// word), it sets the abort word and ERR_BARRIER_TIMEOUT and returns false.
__device__ __noinline__ bool ring_wait(const Params& p, unsigned long long index, unsigned code,
                                       long long timeout = kBarrierTimeoutCycles) {
  const unsigned* st = p.ring_state + (index & p.ring_mask);
  if (ld_acquire_u32(st) == code) return true;
  unsigned* abort_word = p.barrier + 2;
  const long long t0 = clock64();
  for (;;) {
    __nanosleep(32);
    if (ld_acquire_u32(st) == code) return true;
    if (*reinterpret_cast<volatile unsigned*>(abort_word) != 0u) return false;
    if (clock64() - t0 > timeout) {
      atomicExch(abort_word, 1u);
      atomicOr(&p.ctl->error, ERR_BARRIER_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void write_initializer(const Params& p, unsigned long long index, double x, double y,
                                                  double z, double ux, double uy, double uz, double E,
                                                  unsigned long long tid, uint32_t ev, uint32_t prim, int32_t layer,
                                                  uint8_t ptype) {
  const unsigned long long i = index & p.ring_mask;
  unsigned code = 0;
  if (p.ring_state) {  // asynchronous loop: wait until the entry's last reader is done
    code = ring_lap_code(p, index);
    if (!ring_wait(p, index, code)) return;
  }
  p.ring.x[i] = x;
  p.ring.y[i] = y;
  p.ring.z[i] = z;
  p.ring.ux[i] = ux;
  p.ring.uy[i] = uy;
  p.ring.uz[i] = uz;
  p.ring.E[i] = E;
  p.ring.tid[i] = tid;
  p.ring.event[i] = ev;
  p.ring.primary[i] = prim;
  p.ring.layer[i] = layer;
  p.ring.ptype[i] = ptype;
  if (p.ring_state) {
    st_release_u32(p.ring_state + i, code + 1u);
    atomicAdd(&p.ctl->avail, 1ull);  // one more entry readers may claim
  }
}

struct Span {
  uint32_t lo, hi;
  const uint32_t* perm;
};

// Order in which the block-local policy deals its groups to the warps: the
// interactions (costliest first), then the charged along-steps, then the
// photon along-steps (unused keys last).
__constant__ uint8_t kPieceOrder[kMaxKeys] = {K_G_COMPTON, K_E_MOLLER, K_G_PAIR, K_E_BREMS, K_E_RANGE, K_E_GEOM,
                                              K_G_GEOM, K_G_PE, 8, 9, 10, 11, 12, 13, 14, 15};

__device__ __forceinline__ uint8_t key_of(int policy, uint8_t ptype, uint8_t act) {
  if (policy == POLICY_ACTION) return ptype == GAMMA ? KA_NEUTRAL : KA_CHARGED;
  if (ptype == GAMMA) {
    switch (act) {
      case A_COMPTON: return K_G_COMPTON;
      case A_PE: return K_G_PE;
      case A_PAIR: return K_G_PAIR;
      default: return K_G_GEOM;
    }
  }
  switch (act) {
    case A_RANGE: return K_E_RANGE;
    case A_MOLLER: return K_E_MOLLER;
    case A_BREMS: return K_E_BREMS;
    default: return K_E_GEOM;
  }
}

// --------------------------------------------------------------- step limit
// Step limit of one live track: fresh number of mean free paths if unset,
// cross-sections from the shared-memory tables, range limit, distance to
// the layer's planes (straight line, or the exact helix for charged tracks in
// the field), the shortest of them with ties resolved boundary > range >
// interaction, and for an interaction the process, chosen now with the
// pre-step cross-sections. Writes the step length, the residual range after
// the step, n_mfp and the draw counter; returns the next action.
__device__ __forceinline__ uint8_t step_limit(const Params& p, uint32_t slot, const double2* tab, const double* zb,
                                              const int32_t* lmat) {
  const Tracks& t = p.trk;
  [[maybe_unused]] long long t_mark = CELER_LANE_CLOCK();  // diagnostic build only
  const double E = t.E[slot];
  CELER_LANES(LS_STEP_LIMIT);
  const uint8_t pt = t.ptype[slot];
  const int layer = t.layer[slot];
  double nmfp = t.nmfp[slot];
  TrackRng rng(p.seed, t.event[slot], t.tid[slot], t.ctr[slot]);
  // every field of the state in one round of loads, before the calls below
  // (the compiler keeps loads behind a call it cannot see into): +1-2 %
  const double x = t.x[slot], y = t.y[slot], z = t.z[slot];
  const double ux = t.ux[slot], uy = t.uy[slot], uz = t.uz[slot];
  const double gfrac = t.gfrac[slot];
  const int gbin = t.gbin[slot];
  // nmfp < 0 on the bits: -1 marks it unset; otherwise it is >= +0 (a
  // zero difference rounds to +0)
  const bool fresh = dbits(nmfp) < 0;
  if (fresh) nmfp = -fast_log(rng.uniform(), p.mtab);

  const double2* mt = tab + lmat[layer] * (kCols * kGrid);
  const bool charged = pt != GAMMA;
  if (!charged) CELER_LANE_MARK(LS_T_LIMIT, t_mark);
  // A photon's energy changes only where its n_mfp is reset (creation, an
  // interaction), so the grid position computed at the step that samples
  // n_mfp holds until the next such step: later steps reload it.
  GridPos g;
  if (charged || fresh) {
    g = grid_pos(E, p.lnEmin, p.inv_dl, p.mtab);
    if (!charged) {
      t.gbin[slot] = g.bin;
      t.gfrac[slot] = g.frac;
    }
  } else {
    g = GridPos{gbin, gfrac};
  }
  if (!charged) CELER_LANE_MARK(LS_T_LIMIT + 1, t_mark);
  double mu0, mu1, mu2 = 0.0;
  if (!charged) {
    mu0 = interp(mt + COL_COMPTON * kGrid, g);
    mu1 = interp(mt + COL_PE * kGrid, g);
    // E > threshold on the bits (E >= +0; a NaN E makes mu NaN either way)
    mu2 = dbits(E) > dbits(kPairThreshold) ? interp(mt + COL_PAIR * kGrid, g) : 0.0;
  } else {
    mu0 = interp(mt + COL_MOLLER * kGrid, g);
    mu1 = interp(mt + COL_BREMS * kGrid, g);
  }
  const double mu = (mu0 + mu1) + mu2;
  const bool eloss = charged && (p.processes & PROC_ELOSS);
  const double R = eloss ? interp(mt + COL_RANGE * kGrid, g) : 0.0;
  if (!charged) CELER_LANE_MARK(LS_T_LIMIT + 2, t_mark);

  // The limits are compared in the order z-planes, side planes, range,
  // interaction, each candidate replacing the current one only if strictly
  // shorter. A candidate that is a quotient d / u (or bounded below by an
  // expression) is evaluated only if it can be shorter than the current
  // limit s, i.e. unless |d| > s |u| (1 + 2^-50): beyond that margin the
  // rounded quotient is >= s too, so skipping its division changes no choice
  // (the divisions dominate the FP64 cost of the step limit).
  double s_geo = kInf;
  uint8_t act = A_NONE;
  const long long uzb = __double_as_longlong(uz);
  const unsigned long long uza = (unsigned long long)uzb & 0x7FFFFFFFFFFFFFFFull;
  if (uza != 0ull && uza <= 0x7FF0000000000000ull) {  // uz nonzero, not NaN: one division whatever the sign
    const bool up = uzb >= 0;
    s_geo = (zb[up ? layer + 1 : layer] - z) / uz;
    act = up ? A_ZUP : A_ZDOWN;
  }
  double s_side = kInf;
  const bool helix = charged && ((unsigned long long)dbits(p.Bz) << 1) != 0ull;  // Bz != 0 on the bits
  if (helix) {
    // Over a path s the transverse position moves by at most s, so a side
    // plane farther than s_geo + 1e-3 cm lies beyond the z-plane limit: its
    // helix distance (rounded within ~2e-5 cm even at grazing incidence)
    // cannot be the shorter one, and is not computed (+4 % on the 4 T
    // calorimeter, whose high-energy circles all cross the side planes).
    const double reach = s_geo + 1e-3;
    if (!(p.hx - fabs(x) > reach && p.hy - fabs(y) > reach))
      s_side = helix_side_distance(curvature(pt, E, p.Bz), x, y, ux, uy, p.hx, p.hy);
  } else {
    const double reach = s_geo * kLimitMargin;
    // both planes beyond reach along their axis (|u| <= 1 + 2^-52, hence
    // the second margin): both tests below would fail, and most steps skip
    // them (+4 % on the 4 T calorimeter, +8 % on the 1 GeV one)
    const double reach2 = reach * kLimitMargin;
    if (!(p.hx - fabs(x) > reach2 && p.hy - fabs(y) > reach2)) {
      // the signs of ux, uy on their bits: nonzero (NaN included) and
      // positive; for a positive NaN the distance test fails either way
      const long long bx = dbits(ux), by = dbits(uy);
      if (((unsigned long long)bx << 1) != 0ull) {
        const double d = bx > 0 ? p.hx - x : -p.hx - x;
        if ((bx > 0 ? d : -d) <= reach * fabs(ux)) s_side = d / ux;
      }
      if (((unsigned long long)by << 1) != 0ull) {
        const double d = by > 0 ? p.hy - y : -p.hy - y;
        if ((by > 0 ? d : -d) <= reach * fabs(uy)) s_side = fmin(s_side, d / uy);
      }
    }
  }
  // most steps reach no side plane (s_side = inf): those skip the FP64
  // comparison; s_geo < 0 on the bits (negative, not -0, which stays)
  if (dbits(s_side) != dbits(kInf) && s_side < s_geo) {
    s_geo = s_side;
    act = A_SIDE;
  }
  if (dbits(s_geo) < 0 && dbits(s_geo) != dbits(-0.0)) s_geo = 0.0;
  if (!charged) CELER_LANE_MARK(LS_T_LIMIT + 3, t_mark);

  double s = s_geo;
  if (eloss) {
    // s_rng = R (R <= f) or a R + f (1 - a)(2 - f / R) >= a R + f (1 - a)
    double s_rng = kInf;
    // R, s and the bound are >= +0 (a NaN fails both tests, as in FP64)
    if (dbits(R) <= dbits(kFinalR)) {
      s_rng = R;
    } else if (dbits(kAlphaR * R + kFinalR * (1.0 - kAlphaR)) <= dbits(s * kRangeMargin)) {
      s_rng = kAlphaR * R + kFinalR * (1.0 - kAlphaR) * (2.0 - kFinalR / R);
    }
    if (dbits(s_rng) < dbits(s)) {  // s_rng >= +0; s >= +0 or -0 (then false either way)
      s = s_rng;
      act = A_RANGE;
    }
  }
  bool interact = false;
  // mu > 0 on the bits (mu >= +0: a sum of interpolated non-negative
  // tables; for a NaN mu the second test fails either way)
  if (dbits(mu) > 0 && nmfp <= s * mu * kLimitMargin) {
    const double s_int = nmfp / mu;
    if (dbits(s_int) < dbits(s)) {  // s_int >= +0; s >= +0 or -0 (then false either way)
      s = s_int;
      interact = true;
    }
  }
  if (dbits(s) == dbits(kInf)) {
    act = A_TRAPPED;
    s = 0.0;
  } else {
    // Runge-Kutta field propagation with a substep cap (Sec. 3.3): a step
    // needing more than `cap` substeps of 0.1 rad of turn is cut there and
    // ends without a crossing or an interaction, to go on next iteration
    if (helix && p.field_cap > 0) {
      const double kappa = curvature(pt, E, p.Bz).kappa;
      if (s * fabs(kappa) > kRkTurn * p.field_cap) {
        s = kRkTurn * p.field_cap / fabs(kappa);
        act = A_FIELD;
        interact = false;
      }
    }
    nmfp -= s * mu;
  }
  if (interact) {
    // an interaction means a finite mu, so every operand below is finite
    // and >= +0: the comparisons on the bits are exact
    const double target = rng.uniform() * mu;
    int last = -1;
    if (dbits(mu0) > 0) last = 0;
    if (dbits(mu1) > 0) last = 1;
    if (dbits(mu2) > 0) last = 2;
    int sel;
    double acc = mu0;
    if (dbits(target) < dbits(acc)) {
      sel = 0;
    } else {
      acc += mu1;
      if (dbits(target) < dbits(acc)) {
        sel = 1;
      } else {
        acc += mu2;
        sel = (!charged && dbits(target) < dbits(acc)) ? 2 : last;
      }
    }
    act = charged ? (sel == 0 ? A_MOLLER : A_BREMS) : (uint8_t)(A_COMPTON + sel);
  }
  t.nmfp[slot] = nmfp;
  t.ctr[slot] = rng.ctr;
  t.step[slot] = s;
  if (eloss) t.rpost[slot] = R - s;
  t.action[slot] = act;
  if (!charged) CELER_LANE_MARK(LS_T_LIMIT + 4, t_mark);
  return act;
}

// ------------------------------------------------------------------ phases
// Each phase is executed by every thread of a block; bid / nb are the block's
// index and the number of blocks sharing the phase. The same functions run as
// stand-alone kernels (host loop or CUDA graph) and inside the persistent
// loop kernel. One iteration is three phases:
//   A  fill vacant slots from the initializer buffer and compute the step
//      limit (next action) of every live track, tile by tile; the last block
//      to finish does the bookkeeping (buffer head, vacancy counts, partition
//      offsets, whether secondaries are sure to fit);
//   B  scatter slot indices into the partition (sorted policies only);
//   C  along-step and, for tracks whose step ends in an interaction, the
//      interaction, in partition order; the last block to finish ends the
//      iteration (counters, trace, loop condition).

// Static data every step kernel needs in shared memory: cross-section and
// range tables, layer planes and layer materials.
struct SharedStatic {
  double2* tab;
  double* zb;
  int32_t* lmat;
};

__device__ __forceinline__ SharedStatic carve_static(const Params& p, unsigned char* raw) {
  SharedStatic s;
  s.tab = reinterpret_cast<double2*>(raw);
  s.zb = reinterpret_cast<double*>(s.tab + p.n_materials * kCols * kGrid);
  s.lmat = reinterpret_cast<int32_t*>(s.zb + p.n_layers + 1);
  return s;
}

__device__ __forceinline__ void stage_static(const Params& p, const SharedStatic& s) {
  const int ntab = p.n_materials * kCols * kGrid;
  for (int i = threadIdx.x; i < ntab; i += blockDim.x) s.tab[i] = p.tables[i];
  for (int i = threadIdx.x; i <= p.n_layers; i += blockDim.x) s.zb[i] = p.zb[i];
  for (int i = threadIdx.x; i < p.n_layers; i += blockDim.x) s.lmat[i] = p.layer_mat[i];
  __syncthreads();
}


// Clear the per-iteration counters (one thread).
__device__ __forceinline__ void clear_iteration_counters(Ctl* c) {
  for (int k = 0; k < kMaxKeys; ++k) {
    c->action_count[k] = 0;
    c->key_total[k] = 0;
  }
  c->steps_iter = 0;
  c->n_deferred = 0;
}

// True in exactly one block: the last one to reach this point in the current
// phase (the counter is reset for the next phase instance). The block that
// returns true sees every other block's writes of the phase.
__device__ __forceinline__ bool last_block_done(unsigned* counter, unsigned nb) {
  __shared__ unsigned s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned ticket = atomicAdd(counter, 1u);
    s_last = (ticket == nb - 1) ? 1u : 0u;
    if (s_last) *reinterpret_cast<volatile unsigned*>(counter) = 0u;
  }
  __syncthreads();
  const bool last = s_last != 0u;
  if (last) __threadfence();
  return last;
}

// Warp-interleaved walk over [lo, hi): chunk g of `width` elements (8, 16
// or 32; lanes at and above the width idle) goes to block g % nb, so
// consecutive chunks land on different SMs. With few live tracks this
// spreads the FP64 work over all SMs instead of stacking warps on the few
// SMs that own the first chunks (an FP64 warp instruction occupies its
// sub-partition's pipe for the same time whatever its active lanes).
struct ChunkWalk {
  uint32_t lo, hi, step, g, width;
  __device__ ChunkWalk(uint32_t lo_, uint32_t hi_, int bid, int nb, uint32_t width_ = 32u)
      : lo(lo_), hi(hi_), step((uint32_t)nb * (blockDim.x >> 5)), g((uint32_t)bid + (threadIdx.x >> 5) * (uint32_t)nb),
        width(width_) {}
  __device__ __forceinline__ bool more() const { return (unsigned long long)lo + (unsigned long long)width * g < hi; }
  __device__ __forceinline__ uint32_t index() const {
    const uint32_t lane = threadIdx.x & 31;
    return lane < width ? lo + width * g + lane : hi;
  }
  __device__ __forceinline__ void next() { g += step; }
};

// Width of the step-phase chunks for a partition range of n live tracks: as
// few tracks per warp as keep one warp per SM sub-partition (nb blocks of
// four), since a warp's time is set by its instruction count and the
// slowest of its lanes (rejection loops), not by how many lanes it runs.
__device__ __forceinline__ uint32_t spread_width(uint32_t n, int nb) {
  const uint32_t subs = (uint32_t)nb * 4u;
  return n <= subs * 8u ? 8u : (n <= subs * 16u ? 16u : 32u);
}

// ---- phase A: initializer fill + step limit, on 32-slot warp-tiles
// A warp owns a 32-slot chunk: it fills the chunk's vacant slots from the
// initializer buffer (the r-th vacant slot in ascending slot order over the
// whole store takes initializer head + r, for r < queued: deterministic
// filling; vprefix[g] = vacant slots before chunk g, scanned at the end of
// the previous iteration), then computes the step limit of every live slot
// of the chunk and adds the chunk's key counts to its 256-slot tile. Chunks
// are dealt to warps interleaved over the blocks, so a handful of live
// chunks is spread over as many SMs.
__device__ __forceinline__ void fill_and_limit_chunk(const Params& p, uint32_t g, const SharedStatic& ss, bool fill,
                                                     bool do_step, unsigned long long head,
                                                     unsigned long long queued, unsigned* s_acts,
                                                     unsigned* s_keys, unsigned long long& my_steps) {
  const int lane = threadIdx.x & 31;
  const uint32_t slot = g * 32u + lane;
  const bool real = slot < p.n_slots;
  unsigned nfill = 0;
  if (fill) {
    // vacant slots before this chunk: those before its tile, plus the ones in
    // the tile's earlier chunks (at most 7, read in parallel by the lanes)
    const uint32_t first = (g >> 3) << 3;
    unsigned part = (first + lane < g) ? __ldcg(&p.vacant[first + lane]) : 0u;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    const unsigned long long before = __ldcg(&p.tile_prefix[g >> 3]) + __shfl_sync(0xffffffffu, part, 0);
    if (before < queued) {
      const bool vac = real && p.trk.status[slot] == VACANT;
      const unsigned bal = __ballot_sync(0xffffffffu, vac);
      const unsigned long long r = before + __popc(bal & ((1u << lane) - 1u));
      if (vac && r < queued) {
        const unsigned long long i = (head + r) & p.ring_mask;
        const Tracks& t = p.trk;
        t.x[slot] = p.ring.x[i];
        t.y[slot] = p.ring.y[i];
        t.z[slot] = p.ring.z[i];
        t.ux[slot] = p.ring.ux[i];
        t.uy[slot] = p.ring.uy[i];
        t.uz[slot] = p.ring.uz[i];
        t.E[slot] = p.ring.E[i];
        t.tid[slot] = p.ring.tid[i];
        t.event[slot] = p.ring.event[i];
        t.primary[slot] = p.ring.primary[i];
        t.layer[slot] = p.ring.layer[i];
        t.ptype[slot] = p.ring.ptype[i];
        t.ctr[slot] = 0u;
        t.nmfp[slot] = -1.0;
        t.action[slot] = A_NONE;
        t.status[slot] = ALIVE;
      }
      const unsigned long long left = queued - before;
      nfill = (unsigned)((unsigned long long)__popc(bal) < left ? __popc(bal) : left);
    }
    if (lane == 0) {
      p.filled[g] = nfill;
      if (nfill) atomicAdd(&p.ctl->filled_total, (unsigned long long)nfill);
    }
  } else if (do_step) {
    nfill = __ldcg(&p.filled[g]);  // set by a separate fill launch
  }
  if (!do_step) return;
  const bool sorted = global_partition(p.policy);
  const uint8_t vacant_key = p.policy == POLICY_ACTION ? KA_VACANT : K_VACANT_FULL;
  const unsigned csize = (p.n_slots - g * 32u) < 32u ? (p.n_slots - g * 32u) : 32u;
  const bool live = __ldcg(&p.vacant[g]) < csize || nfill > 0;  // warp-uniform
  uint8_t key = vacant_key;
  if (live) {
    if (real) {
      const uint8_t st = p.trk.status[slot];
      uint8_t act = A_NONE;
      if (st == ALIVE) {
        act = step_limit(p, slot, ss.tab, ss.zb, ss.lmat);
        ++my_steps;
      } else if (st == DEFERRED) {
        act = p.trk.action[slot];
      }
      if (st != VACANT) {
        atomicAdd(&s_acts[act], 1u);
        if (sorted) key = key_of(p.policy, p.trk.ptype[slot], act);
      }
    }
  }
  if (sorted) {
    if (real) p.trk.key[slot] = key;
    if (lane == 0) p.chunk_dirty[g] = live ? 1 : 0;
    // only live keys are counted (per block, for the scatter): the vacant
    // key is the last one, so its slots need no position
    const unsigned k = (real && key != vacant_key) ? (unsigned)key : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, k);
    if (k != 0xFFFFFFFFu && lane == __ffs(peers) - 1) atomicAdd(&s_keys[k], (unsigned)__popc(peers));
  }
}

// Block-wide exclusive scan of n 32-bit counts: each thread takes a
// contiguous segment (a multiple of 32 entries), loads it eight 16-byte
// vectors at a time with all loads in flight, the segment sums are scanned
// across the block, and write(i, prefix) receives the exclusive prefix of
// entry i (written to a different array than `in`). Returns the total. One
// block; every thread must call it.
template <class Write>
__device__ unsigned long long block_scan_counts(const uint32_t* __restrict__ in, uint32_t n, Write write) {
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_total;
  const uint32_t per = ((n + blockDim.x - 1) / blockDim.x + 31u) & ~31u;
  const uint32_t beg = min(threadIdx.x * per, n);
  const uint32_t end = min(beg + per, n);
  const uint4* v = reinterpret_cast<const uint4*>(in);
  unsigned long long local = 0;
  uint32_t i = beg;
  // the first 32 values stay in registers for the second pass (all of them
  // when the segment is a single round, the common case)
  uint4 q0[8];
  const bool first = i + 32 <= end;
  if (first) {
#pragma unroll
    for (int k = 0; k < 8; ++k) q0[k] = __ldcg(v + (i >> 2) + k);
#pragma unroll
    for (int k = 0; k < 8; ++k) local += (unsigned long long)q0[k].x + q0[k].y + q0[k].z + q0[k].w;
    i += 32;
  }
  for (; i + 32 <= end; i += 32) {
    uint4 q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = __ldcg(v + (i >> 2) + k);
#pragma unroll
    for (int k = 0; k < 8; ++k) local += (unsigned long long)q[k].x + q[k].y + q[k].z + q[k].w;
  }
  for (; i < end; ++i) local += __ldcg(in + i);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  __syncthreads();
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned long long w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0ull;
    unsigned long long wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_total = wi;
  }
  __syncthreads();
  unsigned long long run = s_warp[warp] + incl - local;
  i = beg;
  if (first) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      write(i + 4 * k, run);
      run += q0[k].x;
      write(i + 4 * k + 1, run);
      run += q0[k].y;
      write(i + 4 * k + 2, run);
      run += q0[k].z;
      write(i + 4 * k + 3, run);
      run += q0[k].w;
    }
    i += 32;
  }
  for (; i + 32 <= end; i += 32) {
    uint4 q[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) q[k] = __ldcg(v + (i >> 2) + k);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      write(i + 4 * k, run);
      run += q[k].x;
      write(i + 4 * k + 1, run);
      run += q[k].y;
      write(i + 4 * k + 2, run);
      run += q[k].z;
      write(i + 4 * k + 3, run);
      run += q[k].w;
    }
  }
  for (; i < end; ++i) {
    const unsigned t = __ldcg(in + i);
    write(i, run);
    run += t;
  }
  const unsigned long long total = s_total;
  __syncthreads();
  return total;
}

// Exclusive scan of the per-tile vacancy counts into tile_prefix and their
// total, by one block (end of an iteration, when every release is counted).
__device__ void scan_vacancy(const Params& p) {
  unsigned long long* out = p.tile_prefix;
  const unsigned long long total =
      block_scan_counts(p.tile_vacant, p.n_tiles, [out](uint32_t i, unsigned long long v) { out[i] = v; });
  if (threadIdx.x == 0) p.ctl->total_vacant = total;
}

// Bookkeeping at the end of phase A, by one block: commit the initializers
// taken, scan the per-(key, block) counts of the live keys (nb blocks counted
// them) in key-major order into each block's first output position per key
// and the key offsets, and decide whether this iteration's secondaries are
// sure to fit.
__device__ void bookkeeping_after_fill_step(const Params& p, bool did_fill, int nb) {
  Ctl* c = p.ctl;
  if (did_fill && threadIdx.x == 0) {
    const unsigned long long queued = c->tail - c->head;
    const unsigned long long tv = c->total_vacant;
    const unsigned long long take = tv < queued ? tv : queued;
    if (take != c->filled_total) c->error |= ERR_VACANCY;
    c->filled_total = 0;
    c->head += take;
    c->alive += take;
    c->total_vacant = tv - take;
  }
  if (global_partition(p.policy)) {
    uint32_t* offs = p.block_offsets;
    const int live_keys = p.n_keys - 1;  // the last key is the vacant one
    const unsigned long long total = block_scan_counts(
        p.block_counts, (uint32_t)(live_keys * nb), [offs](uint32_t i, unsigned long long v) { offs[i] = (uint32_t)v; });
    __syncthreads();
    if ((int)threadIdx.x < live_keys) c->offsets[threadIdx.x] = offs[threadIdx.x * nb];
    if (threadIdx.x == 0) c->part_blocks = (unsigned)nb;
    if ((int)threadIdx.x == live_keys) {
      c->offsets[live_keys] = (unsigned)total;
      c->offsets[p.n_keys] = p.n_slots;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const unsigned long long queued = c->tail - c->head;
    const unsigned long long max_new =
        2ull * c->action_count[A_PAIR] + c->action_count[A_MOLLER] + c->action_count[A_BREMS];
    c->defer = (queued + max_new > p.ring_capacity) ? 1u : 0u;
  }
}

// Move the fills of this iteration into the vacancy counts (all blocks, any
// phase after the fill has finished everywhere).
__device__ __forceinline__ void apply_fills(const Params& p, int bid, int nb) {
  for (uint32_t g = bid * blockDim.x + threadIdx.x; g < p.n_chunks; g += nb * blockDim.x) {
    const unsigned f = __ldcg(&p.filled[g]);
    if (f) {
      atomicSub(&p.vacant[g], f);
      atomicSub(&p.tile_vacant[g >> 3], f);
      p.filled[g] = 0u;
    }
  }
}

// Phase A (or its two halves in the per-action launch mode).
__device__ void phase_fill_step(const Params& p, int bid, int nb, const SharedStatic& ss, bool do_fill, bool do_step,
                                bool bookkeeping) {
  __shared__ unsigned s_acts[A_COUNT];
  __shared__ unsigned s_keys[kMaxKeys];
  Ctl* c = p.ctl;
  const unsigned long long head = c->head;
  const unsigned long long queued = c->tail - head;
  const bool fill = do_fill && queued > 0;
  if (threadIdx.x < A_COUNT) s_acts[threadIdx.x] = 0;
  if (threadIdx.x < kMaxKeys) s_keys[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long my_steps = 0;
  if (fill || do_step) {
    // This warp's chunks are g0, g0 + step, ...: 32 at a time, each lane reads
    // one chunk's vacancy (and its tile's prefix) so the warp visits only the
    // chunks that hold live tracks or may receive initializers.
    const int lane = threadIdx.x & 31;
    const uint32_t step = (uint32_t)nb * (blockDim.x >> 5);
    const uint32_t g0 = (uint32_t)bid + (threadIdx.x >> 5) * (uint32_t)nb;
    for (uint32_t base = g0; base < p.n_chunks; base += 32u * step) {
      const uint32_t g = base + lane * step;
      bool cand = false;
      if (g < p.n_chunks) {
        const unsigned csize = (p.n_slots - g * 32u) < 32u ? (p.n_slots - g * 32u) : 32u;
        const unsigned vac = __ldcg(&p.vacant[g]);
        cand = vac < csize;
        if (!cand && fill && vac > 0) cand = __ldcg(&p.tile_prefix[g >> 3]) < queued;
        if (!cand && !do_fill) cand = __ldcg(&p.filled[g]) > 0;  // filled by a separate fill launch
        if (!cand && do_step && global_partition(p.policy)) cand = p.chunk_dirty[g] != 0;  // keys to reset
      }
      unsigned mask = __ballot_sync(0xffffffffu, cand);
      while (mask) {
        const int j = __ffs(mask) - 1;
        mask &= mask - 1;
        fill_and_limit_chunk(p, base + (uint32_t)j * step, ss, fill, do_step, head, queued, s_acts, s_keys, my_steps);
      }
    }
  }
  __syncthreads();
  if (do_step) {
    if (threadIdx.x < A_COUNT && s_acts[threadIdx.x] != 0)
      atomicAdd(&c->action_count[threadIdx.x], s_acts[threadIdx.x]);
    if (global_partition(p.policy) && (int)threadIdx.x < p.n_keys - 1)
      p.block_counts[threadIdx.x * nb + bid] = s_keys[threadIdx.x];
    flush_counter(&c->steps_iter, my_steps, false);
  }
  if (bookkeeping && last_block_done(&c->done_a, nb)) {
    const long long t0 = clock64();
    bookkeeping_after_fill_step(p, true, nb);
    if (threadIdx.x == 0) c->book_total[0] += (unsigned long long)(clock64() - t0);
  }
}

// Scatter slot indices into the partition. Block b owns chunks b, b + nb,
// b + 2 nb, ... (the chunks it counted in phase A). It walks those that hold
// live keys in that order, one per warp, and places each live slot at: the
// block's first position for the key (from the scan) + the block's same-key
// slots placed so far (a running cursor) + same-key slots of earlier warps in
// this pass of the loop + same-key lanes below. The order within a key is thus by owning
// block, then chunk, then lane: deterministic, and no scan over all tiles.
__device__ void phase_scatter(const Params& p, int bid, int nb) {
  __shared__ unsigned s_cnt[kTile / 32][kMaxKeys];
  __shared__ unsigned s_cursor[kMaxKeys];
  __shared__ unsigned s_wlive[kTile / 32];
  __shared__ uint32_t s_live[kTile];
  const int live_keys = p.n_keys - 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const unsigned lt = (1u << lane) - 1u;
  if ((int)threadIdx.x < live_keys) s_cursor[threadIdx.x] = p.block_offsets[threadIdx.x * nb + bid];
  const uint32_t n_own = (uint32_t)bid < p.n_chunks ? (p.n_chunks - (uint32_t)bid + nb - 1) / nb : 0u;
  for (uint32_t m0 = 0; m0 < n_own; m0 += blockDim.x) {
    // this pass's live chunks of the block, compacted in order
    const uint32_t m = m0 + threadIdx.x;
    const uint32_t gm = (uint32_t)bid + (uint32_t)nb * m;
    const bool live = m < n_own && p.chunk_dirty[gm] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, live);
    __syncthreads();  // the previous round is done with s_wlive and s_live
    if (lane == 0) s_wlive[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, nlive = 0;
    for (int w = 0; w < nwarps; ++w) {
      const unsigned cw = s_wlive[w];
      before += w < warp ? cw : 0u;
      nlive += cw;
    }
    if (live) s_live[before + __popc(bal & lt)] = gm;
    __syncthreads();
    for (unsigned j0 = 0; j0 < nlive; j0 += (unsigned)nwarps) {
      const unsigned j = j0 + (unsigned)warp;
      unsigned key = 0xFFFFFFFFu;
      uint32_t slot = 0;
      if (j < nlive) {
        slot = s_live[j] * 32u + lane;
        if (slot < p.n_slots && p.trk.status[slot] != VACANT) key = p.trk.key[slot];
        if (key >= (unsigned)live_keys) key = 0xFFFFFFFFu;
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (lane < live_keys) s_cnt[warp][lane] = 0u;
      __syncwarp();
      if (key != 0xFFFFFFFFu && lane == __ffs(peers) - 1) s_cnt[warp][key] = __popc(peers);
      __syncthreads();
      if (key != 0xFFFFFFFFu) {
        unsigned pos = s_cursor[key] + __popc(peers & lt);
        for (int w = 0; w < warp; ++w) pos += s_cnt[w][key];
        p.perm[pos] = slot;
      }
      __syncthreads();
      if ((int)threadIdx.x < live_keys) {
        unsigned add = 0;
        for (int w = 0; w < nwarps; ++w) add += s_cnt[w][threadIdx.x];
        s_cursor[threadIdx.x] += add;
      }
      __syncthreads();
    }
  }
}

// Along-step of one live track: move by the step length (straight line, or
// the exact helix for charged tracks in the field), continuous energy loss
// through the inverse range table, then the geometric post-step: next layer
// or escape through a z-plane, escape through a side plane, tracking cut.
// Returns true if the track ended.
__device__ __forceinline__ bool along_one(const Params& p, uint32_t slot, uint8_t pt, const SharedStatic& ss) {
  CELER_LANES(LS_ALONG);
  const Tracks& t = p.trk;
  const bool charged = pt != GAMMA;
  const uint8_t act = t.action[slot];
  const uint32_t ev = t.event[slot], prim = t.primary[slot];
  int layer = t.layer[slot];
  double E = t.E[slot];
  double z = t.z[slot];
  // the rest of the state in the same round of loads, ahead of the atomic
  const double s = t.step[slot];
  double x = t.x[slot], y = t.y[slot];
  double ux = t.ux[slot], uy = t.uy[slot];
  const double uz = t.uz[slot];
  if (prim < p.hist_cap) atomicAdd(&p.hist_steps[prim], 1ull);
  if (act == A_TRAPPED) {
    deposit(p, ev, prim, layer, z, E);
    release(p, slot, ev);
    return true;
  }
  const bool eloss = charged && (p.processes & PROC_ELOSS);
  const bool helix = charged && ((unsigned long long)dbits(p.Bz) << 1) != 0ull;  // Bz != 0 on the bits
  if (helix) {
    const Curvature cv = curvature(pt, E, p.Bz);
    if (p.field_cap > 0)
      rk_move(cv.kappa, s, act == A_FIELD ? p.field_cap : rk_substeps(cv.kappa, s), x, y, z, ux, uy, uz);
    else
      helix_move(cv, s, x, y, z, ux, uy, uz, p.mtab);
  } else {
    x += s * ux;
    y += s * uy;
    z += s * uz;
  }
  if (eloss) {
    const double2* R = ss.tab + (ss.lmat[layer] * kCols + COL_RANGE) * kGrid;
    const double Ep = inverse_range(R, t.rpost[slot], p.lnEmin, p.dl, p.mtab);
    deposit(p, ev, prim, layer, z, E - Ep);
    E = Ep;
  }
  bool out = false;
  if (act == A_ZUP) {
    layer += 1;
    if (layer >= p.n_layers) {
      out = true;
    } else {
      z = ss.zb[layer];
    }
  } else if (act == A_ZDOWN) {
    z = ss.zb[layer];
    layer -= 1;
    if (layer < 0) out = true;
  } else if (act == A_SIDE) {
    out = true;
  }
  if (out) {
    escape(p, ev, prim, E);
    release(p, slot, ev);
    return true;
  }
  // E < cut on the bits (E >= +0; a NaN E fails it, as in FP64)
  if (dbits(E) < dbits(p.cut_track)) {
    deposit(p, ev, prim, layer, z, E);
    release(p, slot, ev);
    return true;
  }
  t.x[slot] = x;
  t.y[slot] = y;
  t.z[slot] = z;
  if (helix) {
    t.ux[slot] = ux;
    t.uy[slot] = uy;
  }
  if (eloss) t.E[slot] = E;
  if (act == A_ZUP || act == A_ZDOWN) t.layer[slot] = layer;
  return false;
}

// ---- discrete interactions (one track each; return true if the track ended)

// Compton scattering: Klein-Nishina sampling, the recoil energy deposited
// locally, the photon rotated; below the tracking cut it is absorbed.
__device__ __forceinline__ bool compton_one(const Params& p, uint32_t slot) {
  CELER_LANES(LS_COMPTON);
  const Tracks& t = p.trk;
  const double E = t.E[slot];
  const uint32_t ev = t.event[slot], prim = t.primary[slot];
  const int layer = t.layer[slot];
  const double z = t.z[slot];
  TrackRng rng(p.seed, ev, t.tid[slot], t.ctr[slot]);
  double cost;
  bool ok;
  const double eps = sample_compton(E, rng, cost, ok, p.mtab);
  if (!ok) {  // non-finite input: end the track, flag the run
    atomicOr(&p.ctl->error, ERR_SAMPLING);
    deposit(p, ev, prim, layer, z, E);
    release(p, slot, ev);
    return true;
  }
  const double u_phi = rng.uniform();
  const double E1 = eps * E;
  deposit(p, ev, prim, layer, z, E - E1);
  if (dbits(E1) < dbits(p.cut_track)) {  // on the bits: a negative E1 passes, a positive NaN fails, as in FP64
    deposit(p, ev, prim, layer, z, E1);
    release(p, slot, ev);
    return true;
  }
  double ux = t.ux[slot], uy = t.uy[slot], uz = t.uz[slot];
  rotate_dir(ux, uy, uz, cost, u_phi, p.mtab);
  t.ux[slot] = ux;
  t.uy[slot] = uy;
  t.uz[slot] = uz;
  t.E[slot] = E1;
  t.nmfp[slot] = -1.0;
  t.ctr[slot] = rng.ctr;
  return false;
}

// Photoelectric absorption: all energy deposited locally.
__device__ __forceinline__ bool photoelectric_one(const Params& p, uint32_t slot) {
  CELER_LANES(LS_PE);
  const Tracks& t = p.trk;
  const uint32_t ev = t.event[slot];
  deposit(p, ev, t.primary[slot], t.layer[slot], t.z[slot], t.E[slot]);
  release(p, slot, ev);
  return true;
}

// Secondary-producing interactions reserve their initializer entries before
// any side effect. When the iteration's worst case fits in the free part of
// the buffer ("tight" is false) a group of lanes takes its entries with one
// atomic add on the tail. Otherwise the group claims, by compare-and-swap,
// the longest prefix of its lanes that still fits; the other lanes defer:
// the track keeps its state and draw counter, so the interaction replays
// identically in a later iteration.
__device__ __forceinline__ bool reserve_entries(const Params& p, unsigned n, bool tight, unsigned long long& base) {
  Ctl* c = p.ctl;
  cg::coalesced_group g = cg::coalesced_threads();
  const unsigned prefix = cg::exclusive_scan(g, n);
  const unsigned end = prefix + n;
  const unsigned total = g.shfl(end, g.num_threads() - 1);
  if (total == 0) {
    base = 0;
    return true;
  }
  // The asynchronous loop checks the room against the current head. With
  // room for the largest reservation every thread of the grid could make
  // (two entries each), one atomic add; otherwise compare-and-swap. (A
  // reservation past the room would only make its writer wait, bounded, for
  // the entry's previous reader.)
  const bool async = p.ring_state != nullptr;
  if (async) {
    unsigned long long h = 0, cur = 0;
    if (g.thread_rank() == 0) {
      h = ld_acquire_u64(&c->head);  // before the tail: h <= tail
      cur = *reinterpret_cast<volatile unsigned long long*>(&c->tail);
    }
    h = g.shfl(h, 0);
    cur = g.shfl(cur, 0);
    const unsigned long long in_flight = 2ull * blockDim.x * gridDim.x;
    tight = cur - h + in_flight > p.ring_capacity;
  }
  if (!tight) {
    unsigned long long old = 0;
    if (g.thread_rank() == 0) old = atomicAdd(&c->tail, (unsigned long long)total);
    base = g.shfl(old, 0) + prefix;
    return true;
  }
  unsigned long long head = c->head;
  for (int attempt = 0; attempt < kMaxCasAttempts; ++attempt) {
    unsigned long long cur = 0;
    if (g.thread_rank() == 0) {
      if (async) head = ld_acquire_u64(&c->head);  // read before the tail: head <= tail
      cur = *reinterpret_cast<volatile unsigned long long*>(&c->tail);
    }
    cur = g.shfl(cur, 0);
    if (async) head = g.shfl(head, 0);
    const unsigned long long used = cur - head;
    const unsigned long long room = used < p.ring_capacity ? p.ring_capacity - used : 0ull;
    const unsigned fits_mask = g.ballot((unsigned long long)end <= room);
    const int last = fits_mask ? 31 - __clz(fits_mask) : -1;
    unsigned take = g.shfl(end, last >= 0 ? last : 0);
    if (last < 0) take = 0;
    if (take == 0) break;
    unsigned long long got = 0;
    if (g.thread_rank() == 0) got = atomicCAS(&c->tail, cur, cur + take);
    got = g.shfl(got, 0);
    if (got == cur) {
      base = cur + prefix;
      return n == 0 || end <= take;
    }
  }
  base = 0;
  return n == 0;
}

__device__ __forceinline__ void defer_track(const Params& p, uint32_t slot, uint8_t st, unsigned long long& n_def) {
  if (st == ALIVE) {
    p.trk.status[slot] = DEFERRED;
    ++n_def;
  }
}

// Pair production: the pair's kinetic energy E - 2 m_e c^2 deposited locally,
// two photons of m_e c^2 back to back in an isotropic direction.
__device__ __forceinline__ bool pair_one(const Params& p, uint32_t slot, uint8_t st, bool tight,
                                         unsigned long long& n_def) {
  CELER_LANES(LS_PAIR);
  const Tracks& t = p.trk;
  const bool keep = kMe >= p.cut_track;
  const bool reuse = keep && p.reuse_parent != 0;  // the first photon takes the parent's slot
  unsigned long long base;
  if (!reserve_entries(p, keep ? (reuse ? 1u : 2u) : 0u, tight, base)) {
    defer_track(p, slot, st, n_def);
    return false;
  }
  const double E = t.E[slot];
  const uint32_t ev = t.event[slot], prim = t.primary[slot];
  const int layer = t.layer[slot];
  const double x = t.x[slot], y = t.y[slot], z = t.z[slot];
  TrackRng rng(p.seed, ev, t.tid[slot], t.ctr[slot]);
  deposit(p, ev, prim, layer, z, E - 2.0 * kMe);
  const double cost = 2.0 * rng.uniform() - 1.0;
  const double u_phi = rng.uniform();
  const double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
  double sp_, cp_;
  fast_sincos_2pi(u_phi, p.mtab, &sp_, &cp_);
  const double dx = sint * cp_, dy = sint * sp_, dz = cost;
  if (keep) {
    const unsigned long long tid1 = rng.raw();
    const unsigned long long tid2 = rng.raw();
    if (prim < p.hist_cap) atomicAdd(&p.hist_secondaries[prim], 2ull);
    if (reuse) {
      // parent-slot reuse (Sec. 3.2): the first photon starts in the slot the
      // pair ended (position, layer, event and primary are the parent's), as
      // a fresh track; the second goes to the initializer buffer
      write_initializer(p, base, x, y, z, -dx, -dy, -dz, kMe, tid2, ev, prim, layer, GAMMA);
      atomicAdd(&p.event_live[row_of(p, ev)], 1u);
      t.ux[slot] = dx;
      t.uy[slot] = dy;
      t.uz[slot] = dz;
      t.E[slot] = kMe;
      t.tid[slot] = tid1;
      t.ctr[slot] = 0u;
      t.nmfp[slot] = -1.0;
      t.action[slot] = A_NONE;
      t.status[slot] = ALIVE;
      return false;
    }
    write_initializer(p, base, x, y, z, dx, dy, dz, kMe, tid1, ev, prim, layer, GAMMA);
    write_initializer(p, base + 1, x, y, z, -dx, -dy, -dz, kMe, tid2, ev, prim, layer, GAMMA);
    atomicAdd(&p.event_live[row_of(p, ev)], 2u);
  } else {
    deposit(p, ev, prim, layer, z, kMe);
    deposit(p, ev, prim, layer, z, kMe);
  }
  release(p, slot, ev);
  return true;
}

// Moller scattering: delta ray above the production cut from the Moller
// cross-section, directions from two-body kinematics (delta polar angle from
// energy-momentum conservation, primary from momentum conservation).
__device__ __forceinline__ bool moller_one(const Params& p, uint32_t slot, uint8_t st, bool tight,
                                           unsigned long long& n_def) {
  CELER_LANES(LS_MOLLER);
  const Tracks& t = p.trk;
  const double T = t.E[slot];
  if (T <= 2.0 * p.cut_moller) {  // kinematically closed at the post-step energy: null collision
    t.nmfp[slot] = -1.0;
    t.status[slot] = ALIVE;
    return false;
  }
  const uint32_t ev = t.event[slot], prim = t.primary[slot];
  TrackRng rng(p.seed, ev, t.tid[slot], t.ctr[slot]);
  bool ok;
  const double eps = sample_moller(T, p.cut_moller, rng, ok);
  const double Td = eps * T;
  const bool keep = ok && Td >= p.cut_track;
  unsigned long long base;
  if (!reserve_entries(p, keep ? 1u : 0u, tight, base)) {
    defer_track(p, slot, st, n_def);
    return false;
  }
  const int layer = t.layer[slot];
  const double x = t.x[slot], y = t.y[slot], z = t.z[slot];
  if (!ok) {  // non-finite input: end the track, flag the run
    atomicOr(&p.ctl->error, ERR_SAMPLING);
    deposit(p, ev, prim, layer, z, T);
    release(p, slot, ev);
    return true;
  }
  // momenta p^2 = T (T + 2 m) and the delta's polar cosine
  // sqrt(Td (T + 2m) / (T (Td + 2m))) = Td (T + 2m) / (p p_delta), from two
  // reciprocal square roots
  const double pp2 = T * (T + 2.0 * kMe), pd2 = Td * (Td + 2.0 * kMe);
  const double rpp = rsqrt(pp2), rpd = rsqrt(pd2);
  const double cost = fmin(1.0, Td * (T + 2.0 * kMe) * rpp * rpd);
  const double u_phi = rng.uniform();
  const double ux = t.ux[slot], uy = t.uy[slot], uz = t.uz[slot];
  double dx = ux, dy = uy, dz = uz;
  rotate_dir(dx, dy, dz, cost, u_phi, p.mtab);
  const double pp = pp2 * rpp;
  const double pd = pd2 * rpd;
  const double vx = pp * ux - pd * dx, vy = pp * uy - pd * dy, vz = pp * uz - pd * dz;
  const double inv = rsqrt(vx * vx + vy * vy + vz * vz);
  const double E1 = T - Td;
  if (keep) {
    const unsigned long long tid = rng.raw();
    write_initializer(p, base, x, y, z, dx, dy, dz, Td, tid, ev, prim, layer, ELECTRON);
    atomicAdd(&p.event_live[row_of(p, ev)], 1u);
    if (prim < p.hist_cap) atomicAdd(&p.hist_secondaries[prim], 1ull);
  } else {
    deposit(p, ev, prim, layer, z, Td);
  }
  if (dbits(E1) < dbits(p.cut_track)) {  // on the bits: a negative E1 passes, a positive NaN fails, as in FP64
    deposit(p, ev, prim, layer, z, E1);
    release(p, slot, ev);
    return true;
  }
  t.ux[slot] = vx * inv;
  t.uy[slot] = vy * inv;
  t.uz[slot] = vz * inv;
  t.E[slot] = E1;
  t.nmfp[slot] = -1.0;
  t.ctr[slot] = rng.ctr;
  t.status[slot] = ALIVE;
  return false;
}

// Bremsstrahlung: photon energy from the 1/k spectrum on (k_cut, T], emitted
// along the parent direction; the parent keeps its direction.
__device__ __forceinline__ bool brems_one(const Params& p, uint32_t slot, uint8_t st, bool tight,
                                          unsigned long long& n_def) {
  CELER_LANES(LS_BREMS);
  const Tracks& t = p.trk;
  const double T = t.E[slot];
  if (T <= p.cut_brems) {  // null collision
    t.nmfp[slot] = -1.0;
    t.status[slot] = ALIVE;
    return false;
  }
  const uint32_t ev = t.event[slot], prim = t.primary[slot];
  TrackRng rng(p.seed, ev, t.tid[slot], t.ctr[slot]);
  double k = p.cut_brems * fast_exp(rng.uniform() * fast_log(T / p.cut_brems, p.mtab), p.mtab);
  if (k > T) k = T;
  const bool keep = k >= p.cut_track;
  unsigned long long base;
  if (!reserve_entries(p, keep ? 1u : 0u, tight, base)) {
    defer_track(p, slot, st, n_def);
    return false;
  }
  const int layer = t.layer[slot];
  const double x = t.x[slot], y = t.y[slot], z = t.z[slot];
  const double E1 = T - k;
  if (keep) {
    const unsigned long long tid = rng.raw();
    write_initializer(p, base, x, y, z, t.ux[slot], t.uy[slot], t.uz[slot], k, tid, ev, prim, layer, GAMMA);
    atomicAdd(&p.event_live[row_of(p, ev)], 1u);
    if (prim < p.hist_cap) atomicAdd(&p.hist_secondaries[prim], 1ull);
  } else {
    deposit(p, ev, prim, layer, z, k);
  }
  if (dbits(E1) < dbits(p.cut_track)) {  // on the bits: a negative E1 passes, a positive NaN fails, as in FP64
    deposit(p, ev, prim, layer, z, E1);
    release(p, slot, ev);
    return true;
  }
  t.E[slot] = E1;
  t.nmfp[slot] = -1.0;
  t.ctr[slot] = rng.ctr;
  t.status[slot] = ALIVE;
  return false;
}

// Interaction of one track whose step ended in one (or whose interaction is
// waiting for buffer space). Returns true if the track ended.
__device__ __forceinline__ bool post_one(const Params& p, uint32_t slot, uint8_t st, uint8_t act, bool tight,
                                         unsigned long long& n_def) {
  switch (act) {
    case A_COMPTON: return compton_one(p, slot);
    case A_PE: return photoelectric_one(p, slot);
    case A_PAIR: return pair_one(p, slot, st, tight, n_def);
    case A_MOLLER: return moller_one(p, slot, st, tight, n_def);
    case A_BREMS: return brems_one(p, slot, st, tight, n_def);
    default: return false;
  }
}

__device__ __forceinline__ bool is_interaction(uint8_t act) { return act >= A_COMPTON && act <= A_BREMS; }


// Work range of the step phase for the policy: all slots (masking), or the
// partition range of the live keys.
__device__ __forceinline__ Span live_span(const Params& p) {
  if (!global_partition(p.policy)) return Span{0u, p.n_slots, nullptr};
  const int hi = p.policy == POLICY_ACTION ? KA_VACANT : K_VACANT_FULL;
  return Span{p.ctl->offsets[0], p.ctl->offsets[hi], p.perm};
}

// Plan of the block-local policy's next fill (one thread, between
// iterations): the initializers it takes, min(vacant slots, queued), and
// whether the secondary buffer could overflow during that iteration: every
// track steps at most once and creates at most two secondaries, and the
// taken entries stay counted until the iteration ends, so the buffer is
// sure to suffice if queued + 2 (live + taken) fits its capacity.
__device__ __forceinline__ unsigned long long plan_local_fill(const Params& p, unsigned long long head,
                                                              unsigned long long tail, unsigned long long alive,
                                                              unsigned long long total_vacant) {
  Ctl* c = p.ctl;
  const unsigned long long queued = tail - head;
  const unsigned long long take = total_vacant < queued ? total_vacant : queued;
  c->fill_take = take;
  c->defer_local = (queued + 2ull * (alive + take) > p.ring_capacity) ? 1u : 0u;
  return take;
}

// End of an iteration: counters, the per-iteration trace row, stall and
// iteration-limit checks, the loop condition, and the per-iteration counters
// cleared for the next one. One warp: every counter is read in one batch of
// loads, the per-action counts one per lane.
__device__ void loop_ctl_warp(const Params& p, unsigned long long* take_out = nullptr) {
  Ctl* c = p.ctl;
  const int lane = threadIdx.x & 31;
  const unsigned long long head = c->head, tail = c->tail, alive = c->alive, total_vacant = c->total_vacant;
  const unsigned long long steps_iter = c->steps_iter, steps_total = c->steps_total;
  const unsigned long long iteration = c->iteration, trace_count = c->trace_count;
  const unsigned long long max_iterations = c->max_iterations, budget_end = c->budget_end;
  const unsigned n_def = c->n_deferred, stall = c->stall, error = c->error;
  const unsigned ac = lane < kMaxKeys ? c->action_count[lane] : 0u;
  const unsigned long long queued = tail - head;
  const bool worked = steps_iter > 0 || n_def > 0;
  TraceRow& r = p.trace[trace_count % kTraceRows];
  if (lane < kMaxKeys) {
    c->last_action_count[lane] = ac;
    if (worked) r.action_count[lane] = ac;
    c->action_count[lane] = 0u;
    c->key_total[lane] = 0u;
  }
  if (lane == 0) {
    c->last_steps_iter = steps_iter;
    c->last_n_deferred = n_def;
    unsigned long long it = iteration;
    if (worked) {
      c->steps_total = steps_total + steps_iter;
      r.iteration = iteration;
      r.alive = alive;
      r.queued = queued;
      r.steps = steps_iter;
      c->trace_count = trace_count + 1;
      it = iteration + 1;
      c->iteration = it;
    }
    const bool pending = alive + queued > 0;
    // No track stepped although work is pending: every live track waits for
    // buffer space. One such iteration can still place deferred secondaries;
    // three in a row cannot make progress any more.
    unsigned err = error;
    if (steps_iter == 0 && pending) {
      if (stall + 1 >= 3) err |= ERR_NO_PROGRESS;
      c->stall = stall + 1;
    } else {
      c->stall = 0u;
    }
    if (pending && it >= max_iterations) err |= ERR_ITERATIONS;
    if (err != error) c->error = err;
    c->cont = (pending && err == 0u && it < budget_end) ? 1u : 0u;
    c->steps_iter = 0;
    c->n_deferred = 0;
    const unsigned long long take = plan_local_fill(p, head, tail, alive, total_vacant);
    if (take_out) *take_out = take;
  }
}

// Along-step and, if the step ends in one, the interaction of the track in
// `slot` (phase C's body). Returns true if the track ended.
__device__ __forceinline__ bool step_one(const Params& p, uint32_t slot, uint8_t st, const SharedStatic& ss, bool tight,
                                         unsigned long long& n_def) {
  const uint8_t act = p.trk.action[slot];
  if (st == ALIVE && along_one(p, slot, p.trk.ptype[slot], ss)) return true;
  return is_interaction(act) && post_one(p, slot, st, act, tight, n_def);
}

#include "block_pass.cuh"

// Per-block vacancy counts and the plan of the first fill (fill_take and the
// block quotas) for the block-local policy, at the start of a run (its
// iterations keep them current; a run of another policy, or primaries pushed
// since, leave them to be recomputed). Same grid as the loop.
__global__ void __launch_bounds__(kTile) k_local_prepare(Params p) {
  count_block_vacancies(p, blockIdx.x, gridDim.x);
  Ctl* c = p.ctl;
  if (last_block_done(&c->done_p, gridDim.x)) {
    __shared__ uint32_t s_v[kMaxLoopBlocks];
    __shared__ unsigned long long s_sum, s_take;
    __shared__ unsigned s_vmin, s_vmax;
    load_block_vacancies(p, s_v, (int)gridDim.x, &s_sum, &s_vmin, &s_vmax);
    if (threadIdx.x == 0) {
      if (s_sum != c->total_vacant) c->error |= ERR_VACANCY;
      c->local_blocks = gridDim.x;
      s_take = plan_local_fill(p, c->head, c->tail, c->alive, s_sum);
    }
    __syncthreads();
    const unsigned long long planned =
        plan_block_quotas(p, s_v, (int)gridDim.x, s_vmin, s_vmax, s_take, block_quota_cap(p.policy));
    if (threadIdx.x == 0 && planned != s_take) c->fill_take = planned;
  }
}

// Per-tile vacancy prefix and total, recomputed at the start of a run of a
// policy that fills in slot order after block-local iterations (which keep
// the per-tile counts but not their scan). One block.
__global__ void __launch_bounds__(kTile) k_scan_tiles(Params p) { scan_vacancy(p); }

// Phase C: along-step of every live track and, where the step ends in an
// interaction, that interaction, in partition order; deferred interactions
// are retried. The last block ends the iteration.
__device__ void phase_step(const Params& p, int bid, int nb, const SharedStatic& ss, bool bookkeeping,
                           cudaGraphConditionalHandle handle, int use_handle) {
  const Span sp = live_span(p);
  const bool tight = p.ctl->defer != 0u;
  const Tracks& t = p.trk;
  unsigned long long killed = 0, n_def = 0;
  const uint32_t width = sp.perm ? spread_width(sp.hi - sp.lo, nb) : 32u;
  for (ChunkWalk w(sp.lo, sp.hi, bid, nb, width); w.more(); w.next()) {
    const uint32_t i = w.index();
    if (i >= sp.hi) continue;
    const uint32_t slot = sp.perm ? sp.perm[i] : i;
    const uint8_t st = t.status[slot];
    if (st == VACANT) continue;
    const uint8_t act = t.action[slot];
    if (st == ALIVE) {
      if (along_one(p, slot, t.ptype[slot], ss)) {
        ++killed;
        continue;
      }
    }
    if (is_interaction(act) && post_one(p, slot, st, act, tight, n_def)) ++killed;
  }
  flush_counter(&p.ctl->alive, killed, true);
  if (n_def) atomicAdd(&p.ctl->n_deferred, (unsigned)n_def);
  apply_fills(p, bid, nb);
  if (bookkeeping && last_block_done(&p.ctl->done_c, nb)) {
    const long long t0 = clock64();
    scan_vacancy(p);
    if (threadIdx.x < 32) loop_ctl_warp(p);
    if (threadIdx.x == 0) {
      if (use_handle) cudaGraphSetConditional(handle, p.ctl->cont);
      p.ctl->book_total[1] += (unsigned long long)(clock64() - t0);
    }
  }
}

// Along-step only, for one particle kind (per-action launch mode).
__device__ void phase_along_only(const Params& p, bool charged, int bid, int nb, const SharedStatic& ss) {
  Span sp = live_span(p);
  if (p.policy == POLICY_ACTION) {
    sp.lo = p.ctl->offsets[charged ? KA_CHARGED : KA_NEUTRAL];
    sp.hi = p.ctl->offsets[charged ? KA_VACANT : KA_CHARGED];
  }
  unsigned long long killed = 0;
  for (ChunkWalk w(sp.lo, sp.hi, bid, nb); w.more(); w.next()) {
    const uint32_t i = w.index();
    if (i >= sp.hi) continue;
    const uint32_t slot = sp.perm ? sp.perm[i] : i;
    if (p.trk.status[slot] != ALIVE) continue;
    const uint8_t pt = p.trk.ptype[slot];
    if ((pt != GAMMA) != charged) continue;
    if (along_one(p, slot, pt, ss)) ++killed;
  }
  flush_counter(&p.ctl->alive, killed, true);
}

// One interaction process only (per-action launch mode).
__device__ void phase_post_only(const Params& p, uint8_t which, int bid, int nb) {
  Span sp = live_span(p);
  if (p.policy == POLICY_ACTION) {
    const bool charged = which == A_MOLLER || which == A_BREMS;
    sp.lo = p.ctl->offsets[charged ? KA_CHARGED : KA_NEUTRAL];
    sp.hi = p.ctl->offsets[charged ? KA_VACANT : KA_CHARGED];
  } else if (p.policy == POLICY_ACTION_TYPE) {
    int k = K_G_COMPTON;
    switch (which) {
      case A_PE: k = K_G_PE; break;
      case A_PAIR: k = K_G_PAIR; break;
      case A_MOLLER: k = K_E_MOLLER; break;
      case A_BREMS: k = K_E_BREMS; break;
      default: break;
    }
    sp.lo = p.ctl->offsets[k];
    sp.hi = p.ctl->offsets[k + 1];
  }
  const bool tight = p.ctl->defer != 0u;
  unsigned long long killed = 0, n_def = 0;
  for (ChunkWalk w(sp.lo, sp.hi, bid, nb); w.more(); w.next()) {
    const uint32_t i = w.index();
    if (i >= sp.hi) continue;
    const uint32_t slot = sp.perm ? sp.perm[i] : i;
    const uint8_t st = p.trk.status[slot];
    if (st == VACANT || p.trk.action[slot] != which) continue;
    if (post_one(p, slot, st, which, tight, n_def)) ++killed;
  }
  flush_counter(&p.ctl->alive, killed, true);
  if (n_def) atomicAdd(&p.ctl->n_deferred, (unsigned)n_def);
}

// ------------------------------------------------------------------ kernels
// Phase-merged launches (host loop / graph): A, B, C.
__global__ void __launch_bounds__(kTile) k_fill_step(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  phase_fill_step(p, blockIdx.x, gridDim.x, ss, true, true, true);
}

__global__ void __launch_bounds__(kTile) k_scatter(Params p) { phase_scatter(p, blockIdx.x, gridDim.x); }

__global__ void k_step(Params p, cudaGraphConditionalHandle handle, int use_handle) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  phase_step(p, blockIdx.x, gridDim.x, ss, true, handle, use_handle);
}

// The block-pass policies (LOCAL, DATA): one launch per iteration (same grid
// as the loop).
__global__ void __launch_bounds__(kTile) k_local(Params p, cudaGraphConditionalHandle handle, int use_handle) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  const BlockIter it = load_block_iter(p, blockIdx.x, gridDim.x);
  block_iteration(p, blockIdx.x, gridDim.x, ss, handle, use_handle, false, it);
}

// Per-action launches: fill, step limit (+ bookkeeping), scatter, one
// along-step kernel per particle kind, one kernel per interaction, end.
__global__ void __launch_bounds__(kTile) k_fill(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  phase_fill_step(p, blockIdx.x, gridDim.x, ss, true, false, false);
}

__global__ void __launch_bounds__(kTile) k_pre_step(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  phase_fill_step(p, blockIdx.x, gridDim.x, ss, false, true, false);
  if (last_block_done(&p.ctl->done_a, gridDim.x)) bookkeeping_after_fill_step(p, true, gridDim.x);
}

__global__ void k_along(Params p, int charged) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  phase_along_only(p, charged != 0, blockIdx.x, gridDim.x, ss);
}

__global__ void k_post(Params p, int which) { phase_post_only(p, (uint8_t)which, blockIdx.x, gridDim.x); }

__global__ void __launch_bounds__(kTile) k_loop_ctl(Params p, cudaGraphConditionalHandle handle, int use_handle) {
  apply_fills(p, 0, 1);
  __syncthreads();
  scan_vacancy(p);
  if (threadIdx.x < 32) loop_ctl_warp(p);
  if (threadIdx.x == 0 && use_handle) cudaGraphSetConditional(handle, p.ctl->cont);
}

// Start a run: the loop stops after `budget` more iterations (0: no limit).
__global__ void k_begin_run(Ctl* c, unsigned long long budget) {
  c->run_start = c->iteration;
  c->budget_end = budget ? c->iteration + budget : ~0ull;
  c->done_a = 0u;
  c->done_c = 0u;
  c->done_p = 0u;
}

// Grid-wide barrier of the persistent loop (generation counter). Every wait
// is bounded: after ~1 s a block gives up, sets the abort word and the error
// bit, and every block then leaves the loop at its next barrier.
__device__ __forceinline__ bool grid_barrier(const Params& p, unsigned nblocks,
                                             long long timeout = kBarrierTimeoutCycles) {
  __shared__ int s_ok;
  unsigned int* count = p.barrier;
  unsigned int* gen = p.barrier + 1;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = *reinterpret_cast<volatile unsigned*>(gen);
    int ok = 1;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      *reinterpret_cast<volatile unsigned*>(count) = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
      if (*reinterpret_cast<volatile unsigned*>(p.barrier + 2) != 0u) ok = 0;
    } else {
      ok = wait_generation(p, g, timeout) ? 1 : 0;
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The whole step loop in one persistent cooperative launch: one block per
// SM slot, the static tables staged into shared memory once, three grid
// barriers per iteration (two without sorting).
__global__ void __launch_bounds__(kTile, 1) k_loop(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  const unsigned nb = gridDim.x;
  const int bid = blockIdx.x;
  const bool sorted = global_partition(p.policy);
  if (bid == 0 && threadIdx.x == 0) {
    clear_iteration_counters(p.ctl);
    p.ctl->cont = 1u;
  }
  if (!grid_barrier(p, nb)) return;
  Ctl* c = p.ctl;
  long long t_prev = clock64();
  unsigned parity = 0;
  // phase k took (now - t_prev) for block 0 including the barrier wait; every
  // block also records its own work time so the slowest one can be told apart
  auto mark = [&](int k, long long work) {
    if (threadIdx.x == 0) {
      atomicMax(&c->iter_max[parity][k], (unsigned long long)work);
      if (bid == 0) {
        const long long now = clock64();
        c->phase_cycles[k] += (unsigned long long)(now - t_prev);
        t_prev = now;
      }
    }
  };
  for (;;) {
    if (*reinterpret_cast<volatile unsigned*>(&c->cont) == 0u) break;
    if (bid == 0 && threadIdx.x == 0) {
      for (int k = 0; k < 4; ++k) {
        c->max_total[k] += c->iter_max[parity ^ 1][k];
        c->iter_max[parity ^ 1][k] = 0;
      }
    }
    long long t0 = clock64();
    phase_fill_step(p, bid, nb, ss, true, true, true);
    const long long wa = clock64() - t0;
    if (!grid_barrier(p, nb)) break;
    mark(0, wa);
    if (sorted) {
      t0 = clock64();
      phase_scatter(p, bid, nb);
      const long long wb = clock64() - t0;
      if (!grid_barrier(p, nb)) break;
      mark(1, wb);
    }
    t0 = clock64();
    phase_step(p, bid, nb, ss, true, 0, 0);
    const long long wc = clock64() - t0;
    if (!grid_barrier(p, nb)) break;
    mark(2, wc);
    parity ^= 1u;
  }
  if (bid == 0 && threadIdx.x == 0) {
    for (int k = 0; k < 4; ++k) {
      c->max_total[k] += c->iter_max[0][k] + c->iter_max[1][k];
      c->iter_max[0][k] = c->iter_max[1][k] = 0;
    }
  }
}

// The persistent loop of the block-pass policies: one pass per block and
// iteration (block_iteration), one grid barrier per iteration.
__global__ void __launch_bounds__(kTile, 1) k_loop_local(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  const unsigned nb = gridDim.x;
  const int bid = blockIdx.x;
  Ctl* c = p.ctl;
  if (bid == 0 && threadIdx.x == 0) {
    clear_iteration_counters(c);
    c->cont = 1u;
  }
  if (!grid_barrier(p, nb)) return;
  long long t_prev = clock64();
  for (;;) {
    const BlockIter it = load_block_iter(p, bid, (int)nb);  // one batch of loads per iteration
    if (!it.cont) break;
    const unsigned parity = (unsigned)(it.iteration & 1);
    if (bid == 0 && threadIdx.x == 0) {  // the slowest block's work of the previous iteration
      c->max_total[2] += c->iter_max[parity ^ 1u][2];
      c->iter_max[parity ^ 1u][2] = 0;
    }
    const bool ok = block_iteration(p, bid, (int)nb, ss, 0, 0, true, it);
    if (!ok) break;
    if (bid == 0 && threadIdx.x == 0) {
      const long long now = clock64();
      c->phase_cycles[2] += (unsigned long long)(now - t_prev);
      t_prev = now;
    }
  }
  if (bid == 0 && threadIdx.x == 0) {
    c->max_total[2] += c->iter_max[0][2] + c->iter_max[1][2];
    c->iter_max[0][2] = c->iter_max[1][2] = 0;
  }
}

#include "async_loop.cuh"

// Check of the bounded waits: every block but `absent` meets at a grid
// barrier that `absent` never reaches, so the waiters must give up after
// `timeout` cycles, set the abort word and the error bit, and return.
__global__ void k_barrier_probe(Params p, int absent, long long timeout) {
  if ((int)blockIdx.x == absent) return;
  grid_barrier(p, gridDim.x, timeout);
}

// Queue staged primaries at the tail of the initializer buffer.
__global__ void __launch_bounds__(1024) k_push_primaries(Params p, const StagedPrimary* src, uint32_t n) {
  __shared__ unsigned long long s_base;
  if (threadIdx.x == 0) s_base = p.ctl->tail;
  __syncthreads();
  const unsigned long long base = s_base;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const StagedPrimary& q = src[i];
    write_initializer(p, base + i, q.x, q.y, q.z, q.ux, q.uy, q.uz, q.E, q.tid, q.event, q.primary, q.layer,
                      (uint8_t)q.ptype);
    atomicAdd(&p.event_live[row_of(p, q.event)], 1u);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    p.ctl->tail = base + n;
    plan_local_fill(p, p.ctl->head, base + n, p.ctl->alive, p.ctl->total_vacant);
  }
}

// Validate and queue primaries that are already in device memory: one block;
// pass 1 checks every record (and the buffer fill level), pass 2 queues all
// of them only if every check passed.
__global__ void __launch_bounds__(1024) k_push_device_primaries(Params p, const DevicePrimary* src, uint32_t n,
                                                                 uint32_t event, unsigned long long tid0,
                                                                 uint32_t prim0) {
  __shared__ unsigned s_bad;
  __shared__ unsigned long long s_base;
  if (threadIdx.x == 0) {
    s_bad = 0;
    s_base = p.ctl->tail;
    const unsigned long long queued = p.ctl->tail - p.ctl->head;
    if (queued + n > p.ring_capacity) s_bad = 1;
  }
  __syncthreads();
  const double zmax = p.zb[p.n_layers];
  unsigned bad = 0;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const DevicePrimary& q = src[i];
    const double d2 = q.dir[0] * q.dir[0] + q.dir[1] * q.dir[1] + q.dir[2] * q.dir[2];
    const bool ok = isfinite(q.E) && q.E > 0.0 && q.E <= kGridEmax && isfinite(d2) &&
                    fabs(sqrt(d2) - 1.0) <= 1e-12 && fabs(q.pos[0]) <= p.hx && fabs(q.pos[1]) <= p.hy &&
                    q.pos[2] >= p.zb[0] && q.pos[2] <= zmax && (q.ptype == GAMMA || q.ptype == ELECTRON);
    if (!ok) bad = 1;
  }
  if (bad) atomicOr(&s_bad, 1u);
  __syncthreads();
  if (s_bad) {
    if (threadIdx.x == 0) atomicOr(&p.ctl->error, ERR_PRIMARIES_REJECTED);
    return;
  }
  const unsigned long long base = s_base;
  const int L = p.n_layers;
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
    const DevicePrimary& q = src[i];
    const double z = q.pos[2], uz = q.dir[2];
    // layer: the largest l <= L-1 with z_l <= z; on an inner plane moving
    // backwards, the layer behind it
    int lo = 0;
    if (z >= zmax) {
      lo = L - 1;
    } else {
      int hi = L - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (p.zb[mid] <= z)
          lo = mid;
        else
          hi = mid - 1;
      }
      if (z == p.zb[lo] && uz < 0.0 && lo > 0) --lo;
    }
    const uint32_t prim = p.hist_cap > 0 ? prim0 + i : 0xFFFFFFFFu;
    write_initializer(p, base + i, q.pos[0], q.pos[1], z, q.dir[0], q.dir[1], uz, q.E, tid0 + i, event, prim, lo,
                      (uint8_t)q.ptype);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    p.ctl->tail = base + n;
    atomicAdd(&p.event_live[row_of(p, event)], n);
    plan_local_fill(p, p.ctl->head, base + n, p.ctl->alive, p.ctl->total_vacant);
  }
}

int occupancy_grid(const void* fn, int block, size_t smem, int sms, int cap) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, block, smem) != cudaSuccess || nb < 1) nb = 1;
  long g = (long)nb * sms;
  if (cap > 0 && g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

cudaError_t configure_kernels(const Params& p, int block, LaunchShape* sh) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t stat = (size_t)p.n_materials * kCols * kGrid * sizeof(double2) +
                      (size_t)(p.n_layers + 1) * sizeof(double) + (size_t)p.n_layers * sizeof(int32_t);
  sh->static_smem = stat;
  sh->block = block;
  const void* with_smem[] = {(const void*)k_fill_step, (const void*)k_step, (const void*)k_fill,
                             (const void*)k_pre_step, (const void*)k_along, (const void*)k_loop,
                             (const void*)k_local, (const void*)k_loop_local, (const void*)k_loop_async};
  for (const void* fn : with_smem) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)stat);
    if (e != cudaSuccess) return e;
  }
  sh->tile_grid = occupancy_grid((const void*)k_fill_step, kTile, stat, sms, (int)p.n_tiles);
  const int cap_action = (int)((p.n_slots + block - 1) / block);
  sh->step_grid = occupancy_grid((const void*)k_step, block, stat, sms, cap_action);
  sh->along_grid = occupancy_grid((const void*)k_along, block, stat, sms, cap_action);
  sh->post_grid = occupancy_grid((const void*)k_post, block, 0, sms, cap_action);
  int nb = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, (const void*)k_loop, kTile, stat);
  if (e != cudaSuccess) return e;
  int nb_local = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_local, (const void*)k_loop_local, kTile, stat);
  if (e != cudaSuccess) return e;
  if (nb_local < nb) nb = nb_local;  // one grid for every loop (and the block-local launches)
  int nb_async = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_async, (const void*)k_loop_async, kTile, stat);
  if (e != cudaSuccess) return e;
  if (nb_async < nb) nb = nb_async;
  sh->loop_grid = (nb < 1 ? 1 : nb) * sms;
  if (sh->loop_grid > kMaxLoopBlocks) sh->loop_grid = kMaxLoopBlocks;  // size of the per-block arrays
  return cudaGetLastError();
}

void launch_fill_step(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  k_fill_step<<<sh.tile_grid, kTile, sh.static_smem, s>>>(p);
}
void launch_scatter(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  k_scatter<<<sh.tile_grid, kTile, 0, s>>>(p);
}
void launch_step(const Params& p, const LaunchShape& sh, unsigned long long handle, int use_handle, cudaStream_t s) {
  k_step<<<sh.step_grid, sh.block, sh.static_smem, s>>>(p, (cudaGraphConditionalHandle)handle, use_handle);
}
void launch_local(const Params& p, const LaunchShape& sh, unsigned long long handle, int use_handle, cudaStream_t s) {
  k_local<<<sh.loop_grid, kTile, sh.static_smem, s>>>(p, (cudaGraphConditionalHandle)handle, use_handle);
}
void launch_local_prepare(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  k_local_prepare<<<sh.loop_grid, kTile, 0, s>>>(p);
}
void launch_scan_tiles(const Params& p, cudaStream_t s) { k_scan_tiles<<<1, kTile, 0, s>>>(p); }
cudaError_t launch_queue_wait_probe(const Params& p, int which, long long timeout, cudaStream_t s) {
  k_queue_wait_probe<<<1, 32, 0, s>>>(p, which, timeout);
  return cudaGetLastError();
}
cudaError_t launch_barrier_probe(const Params& p, int blocks, int absent, long long timeout, cudaStream_t s) {
  void* args[] = {const_cast<Params*>(&p), &absent, &timeout};
  return cudaLaunchCooperativeKernel((const void*)k_barrier_probe, dim3(blocks), dim3(32), args, 0, s);
}
void launch_fill(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  k_fill<<<sh.tile_grid, kTile, sh.static_smem, s>>>(p);
}
void launch_pre_step(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  k_pre_step<<<sh.tile_grid, kTile, sh.static_smem, s>>>(p);
}
void launch_along(const Params& p, int charged, const LaunchShape& sh, cudaStream_t s) {
  k_along<<<sh.along_grid, sh.block, sh.static_smem, s>>>(p, charged);
}
void launch_post(const Params& p, int which, const LaunchShape& sh, cudaStream_t s) {
  k_post<<<sh.post_grid, sh.block, 0, s>>>(p, which);
}
void launch_loop_ctl(const Params& p, unsigned long long handle, int use_handle, cudaStream_t s) {
  k_loop_ctl<<<1, kTile, 0, s>>>(p, (cudaGraphConditionalHandle)handle, use_handle);
}
void launch_begin_run(const Params& p, unsigned long long budget, cudaStream_t s) {
  k_begin_run<<<1, 1, 0, s>>>(p.ctl, budget);
}
void launch_async_prepare(const Params& p, cudaStream_t s) { k_async_prepare<<<256, 256, 0, s>>>(p); }
cudaError_t launch_loop_async(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  void* args[] = {const_cast<Params*>(&p)};
  return cudaLaunchCooperativeKernel((const void*)k_loop_async, dim3(sh.loop_grid), dim3(kTile), args, sh.static_smem,
                                     s);
}
cudaError_t launch_loop(const Params& p, const LaunchShape& sh, cudaStream_t s) {
  void* args[] = {const_cast<Params*>(&p)};
  const void* fn = block_pass(p.policy) ? (const void*)k_loop_local : (const void*)k_loop;
  return cudaLaunchCooperativeKernel(fn, dim3(sh.loop_grid), dim3(kTile), args, sh.static_smem, s);
}
void launch_push_primaries(const Params& p, const StagedPrimary* d_prim, uint32_t n, cudaStream_t s) {
  k_push_primaries<<<1, 1024, 0, s>>>(p, d_prim, n);
}
void launch_push_device_primaries(const Params& p, const DevicePrimary* src, uint32_t n, uint32_t event,
                                  unsigned long long tid0, uint32_t prim0, cudaStream_t s) {
  k_push_device_primaries<<<1, 1024, 0, s>>>(p, src, n, event, tid0, prim0);
}

const char* kernel_name(int id) {
  static const char* names[KID_COUNT] = {"fill_step", "scatter", "step", "fill", "pre_step", "along_neutral",
                                         "along_charged", "compton", "photoelectric", "pair", "moller", "brems",
                                         "loop_ctl", "loop", "local"};
  return (id >= 0 && id < KID_COUNT) ? names[id] : "?";
}

// Active-lane counters of the instrumented build: per site, visits and lanes
// summed over the copies, then cleared. Without the instrumentation there
// is nothing to read.
cudaError_t read_lane_counts(unsigned long long* host_out, int n_sites) {
#ifdef CELER_LANE_COUNTERS
  unsigned long long all[kLaneCopies][kLaneSites][kLaneValues];
  cudaError_t e = cudaMemcpyFromSymbol(all, g_lane_counts, sizeof(all));
  if (e != cudaSuccess) return e;
  for (int k = 0; k < n_sites && k < kLaneSites; ++k) {
    for (int j = 0; j < kLaneValues; ++j) {
      unsigned long long v = 0;
      for (int c = 0; c < kLaneCopies; ++c) v += all[c][k][j];
      host_out[kLaneValues * k + j] = v;
    }
  }
  static const unsigned long long zeros[kLaneCopies][kLaneSites][kLaneValues] = {};
  return cudaMemcpyToSymbol(g_lane_counts, zeros, sizeof(zeros));
#else
  (void)host_out;
  (void)n_sites;
  return cudaErrorNotSupported;
#endif
}

}  // namespace celer
