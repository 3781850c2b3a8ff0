// The asynchronous step loop (CELER_LOOP_ASYNC) of the block-pass policies:
// the persistent kernel in which every block runs its own passes with no
// grid barrier (k_loop_async), the per-warp schedule of the block-local
// policy (warp_queue_loop and its shared-memory queues), the start-of-run
// kernel that sets the buffer entries' states (k_async_prepare), and the
// check of the bounded queue waits (k_queue_wait_probe). Included by step.cu
// inside its anonymous namespace, after the block passes (local_pass,
// data_pass) and the buffer protocol (ring_wait, take_initializer) it uses.
#pragma once

// Block-wide sums of a pass's counts (every thread gets them).
__device__ PassCounts block_total(const PassCounts& n) {
  __shared__ unsigned long long s_n[4];
  if (threadIdx.x < 4) s_n[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long v[4] = {n.killed, n.n_def, n.steps, n.fill};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    if ((threadIdx.x & 31) == 0 && v[k] != 0) atomicAdd(&s_n[k], v[k]);
  }
  __syncthreads();
  const PassCounts out{s_n[0], s_n[1], s_n[2], s_n[3]};
  __syncthreads();  // s_n is reused by the next call
  return out;
}

// Start of an asynchronous run: the buffer entries' states from head and
// tail (entries in [head, tail) written and unread, the others free for
// their next writer) and the count of ended tracks, head - alive (every
// track came from a buffer entry; a pair photon that reuses its parent's
// slot continues the parent's count).
__global__ void k_async_prepare(Params p) {
  const unsigned long long head = p.ctl->head, tail = p.ctl->tail;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long j = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; j < p.ring_capacity;
       j += stride) {
    const unsigned long long index = head + ((j - head) & p.ring_mask);  // the index in [head, head + capacity) at j
    p.ring_state[j] = ring_lap_code(p, index) + (index < tail ? 1u : 0u);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.ctl->finished = head - p.ctl->alive;
    p.ctl->avail = tail - head;
    p.ctl->async_passes = 0;
    p.ctl->done_x = 0u;
  }
}

// Live tracks a block of the asynchronous loop fills itself up to when
// entries are queued (it takes at least ceil(queued / blocks) in any case):
// a few per warp keeps every sub-partition busy without lengthening the pass.
constexpr unsigned kAsyncFill = 32;

// ---- the asynchronous loop with per-warp scheduling (block-local policy)
//
// Every warp of a block runs its own loop: it takes up to 32 tracks waiting
// for the same kind of step (particle type and next action) from the block's
// queues in shared memory, runs their along-step and interaction, computes
// the survivors' next step limits and queues them again by their new kind. A
// track thus moves on as soon as its own step is done instead of waiting for
// the block's slowest piece, and each piece still holds one kind of step. A
// warp with nothing waiting, or a block holding fewer than kAsyncFill live
// tracks, fills vacant slots from the initializer buffer (one warp at a
// time). The block holds at most kWarpLive live tracks; a block that starts
// with more runs block passes instead.
constexpr unsigned kWarpLive = 1024;  // live tracks per block in this mode: capacity of each queue
constexpr int kLiveKeys = 8;          // the (particle type, action) keys of live tracks, K_G_GEOM..K_E_BREMS
// Warps of a block that take pieces of any size; the others take full pieces
// only (2 measured fastest on the 4 T calorimeter; 3 is 1 % slower there and
// 2 % faster on the 1 GeV one; 4 is 7 % slower there).
constexpr int kAnyPieceWarps = 2;

// Shared-memory queues: entry t of a queue (at t mod kWarpLive) holds a
// 16-bit state in its high half (2 lap: free for its writer; 2 lap + 1:
// written; lap = t / kWarpLive, modulo 2^15) and the value in its low half:
// the slot's index among the block's own slots. Writers reserve on the tail
// counter and readers claim on the head counter; each side waits (bounded)
// only for the other side's access of the same entry, which follows that
// side's claim or reservation directly.
struct WarpQueues {
  unsigned* q;     // kLiveKeys queues of kWarpLive entries, then the free-slot queue
  unsigned* head;  // kLiveKeys + 1 counters
  unsigned* tail;
};
constexpr int kFreeQueue = kLiveKeys;

// Bounded wait of one thread for a shared-memory queue entry to reach
// `state` (as ring_wait).
__device__ __forceinline__ bool wq_wait(const Params& p, volatile unsigned* e, unsigned state,
                                        long long timeout = kBarrierTimeoutCycles) {
  if ((*e >> 16) == state) return true;
  const long long t0 = clock64();
  for (;;) {
    __nanosleep(20);
    if ((*e >> 16) == state) return true;
    if (clock64() - t0 > timeout) {
      atomicExch(p.barrier + 2, 1u);
      atomicOr(&p.ctl->error, ERR_BARRIER_TIMEOUT);
      return false;
    }
  }
}

// Block-scope release store and acquire load of a shared-memory word.
__device__ __forceinline__ void st_release_cta(volatile unsigned* a, unsigned v) {
  const unsigned s = (unsigned)__cvta_generic_to_shared((const void*)a);
  asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(s), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_cta(volatile unsigned* a) {
  const unsigned s = (unsigned)__cvta_generic_to_shared((const void*)a);
  unsigned v;
  asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(s) : "memory");
  return v;
}

// Append v to queue k (one thread). The entry is written with a release
// store, so the caller's global-memory writes of the track are visible to
// the warp that reads it (block scope: a warp of the same block).
__device__ __forceinline__ void wq_push(const Params& p, const WarpQueues& w, int k, unsigned v) {
  const unsigned t = atomicAdd(&w.tail[k], 1u);
  volatile unsigned* e = w.q + (size_t)k * kWarpLive + (t % kWarpLive);
  const unsigned lap2 = (2u * (t / kWarpLive)) & 0xFFFFu;
  if (!wq_wait(p, e, lap2)) return;
  st_release_cta(e, (((lap2 + 1u) & 0xFFFFu) << 16) | (v & 0xFFFFu));
}

// Read entry t of queue k (one thread; t claimed by its warp) with an
// acquire load (the pusher's writes of the track come before the reader's
// reads of it) and free it for the next lap. Returns 0xFFFFFFFF if the wait
// gave up.
__device__ __forceinline__ unsigned wq_read(const Params& p, const WarpQueues& w, int k, unsigned t) {
  volatile unsigned* e = w.q + (size_t)k * kWarpLive + (t % kWarpLive);
  const unsigned lap2 = (2u * (t / kWarpLive)) & 0xFFFFu;
  if (!wq_wait(p, e, (lap2 + 1u) & 0xFFFFu)) return 0xFFFFFFFFu;
  const unsigned v = ld_acquire_cta(e) & 0xFFFFu;
  *e = ((lap2 + 2u) & 0xFFFFu) << 16;
  return v;
}

// The block's slot of local index li (li = m * 32 + lane for its m-th chunk).
__device__ __forceinline__ uint32_t local_slot(unsigned li, int bid, int nb) {
  return ((uint32_t)bid + (uint32_t)nb * (li >> 5)) * 32u + (li & 31u);
}

// Next step of a live track in `slot` (one thread): a fresh step limit if it
// is alive (counted as a step), or its pending interaction if it is deferred;
// then it is queued by its kind.
__device__ __forceinline__ void wq_requeue(const Params& p, const WarpQueues& w, const SharedStatic& ss, uint32_t slot,
                                           unsigned li, unsigned& steps) {
  const Tracks& t = p.trk;
  uint8_t act;
  if (t.status[slot] == ALIVE) {
    act = step_limit(p, slot, ss.tab, ss.zb, ss.lmat);
    ++steps;
  } else {
    act = t.action[slot];
  }
#ifdef CELER_LANE_COUNTERS
  long long t_push = clock64();
#endif
  wq_push(p, w, key_of(POLICY_ACTION_TYPE, t.ptype[slot], act), li);
  CELER_LANE_MARK(LS_T_PUSH, t_push);
}

// Warp sums of the per-lane counts since the last flush (at most 16 pieces
// or fills, a few per lane each, so 32-bit sums), added to the device
// counters by lane 0. Ended tracks are counted after a fence, behind the
// tail reservations of their interactions (the run's end condition).
__device__ __forceinline__ void wq_flush_counts(const Params& p, unsigned steps, unsigned killed, unsigned fill) {
  Ctl* c = p.ctl;
  steps = __reduce_add_sync(0xffffffffu, steps);
  killed = __reduce_add_sync(0xffffffffu, killed);
  fill = __reduce_add_sync(0xffffffffu, fill);
  if ((threadIdx.x & 31) == 0) {
    if (steps) atomicAdd(&c->steps_total, (unsigned long long)steps);
    const long long dalive = (long long)fill - (long long)killed;
    if (dalive != 0) atomicAdd(&c->alive, (unsigned long long)dalive);
    if (killed) {
      __threadfence();
      atomicAdd(&c->finished, (unsigned long long)killed);
    }
  }
}

// The per-warp loop of one block. live0: the block's live tracks at the
// start (at most kWarpLive). A run with an iteration budget ends by draining:
// once a warp has run `budget` pieces the block stops filling, its warps step
// the queued tracks without computing new step limits (the survivors stay
// alive in their slots, between two steps, as a synchronous iteration leaves
// them), and every warp leaves when no track waits. Returns the most pieces
// any of its warps ran.
__device__ unsigned long long warp_queue_loop(const Params& p, int bid, int nb, const SharedStatic& ss, unsigned owned,
                                              unsigned live0, unsigned long long budget) {
  __shared__ unsigned s_q[(kLiveKeys + 1) * kWarpLive];
  __shared__ unsigned s_head[kLiveKeys + 1], s_tail[kLiveKeys + 1];
  __shared__ unsigned s_live, s_filling, s_budget, s_exit, s_drain;
  __shared__ unsigned long long s_pieces;
  Ctl* c = p.ctl;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (int)(blockDim.x >> 5);
  const WarpQueues w{s_q, s_head, s_tail};
  for (unsigned i = threadIdx.x; i < (kLiveKeys + 1) * kWarpLive; i += blockDim.x) s_q[i] = 0u;
  if (threadIdx.x <= kLiveKeys) s_head[threadIdx.x] = s_tail[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    s_live = live0;
    s_filling = 0u;
    s_budget = kWarpLive - live0;  // free slots the block may hold
    s_exit = 0u;
    s_drain = budget == 0ull ? 1u : 0u;
    s_pieces = 0ull;
  }
  __syncthreads();
  // the block's live tracks to their queues, vacant slots to the free queue
  unsigned steps = 0, killed = 0, fill = 0, events = 0;
  unsigned long long pieces = 0;
  const unsigned n_own = (owned + 31u) / 32u;
  for (unsigned m = (unsigned)warp; m < n_own; m += (unsigned)nwarps) {
    const unsigned li = m * 32u + (unsigned)lane;
    const uint32_t slot = local_slot(li, bid, nb);
    if (li < owned) {
      if (p.trk.status[slot] != VACANT) {
        wq_requeue(p, w, ss, slot, li, steps);
      } else if (atomicSub(&s_budget, 1u) - 1u < kWarpLive) {  // a budget left: the slot joins the free queue
        wq_push(p, w, kFreeQueue, li);
      } else {
        atomicAdd(&s_budget, 1u);
      }
    }
  }
  wq_flush_counts(p, steps, 0, 0);
  steps = 0;
  __syncthreads();
  const unsigned long long max_pieces = __ldcg(&c->max_iterations);  // per run
  unsigned long long seen = ~0ull;
  long long t_seen = clock64();
  unsigned last_k = 0xFFu;  // the kind of the warp's last piece
  // Whole-job runs concentrate a block's work in full pieces (throughput);
  // budgeted runs (a serving loop's chunks, interactive stepping) let every
  // warp take any piece, so that no track waits for a free warp (latency:
  // served at 2,000 events/s, p50 5.8 ms against 6.5 ms with the rule).
  const int any_warps = budget == ~0ull ? kAnyPieceWarps : nwarps;
  for (;;) {
    // the loop's flags, read by lane 0 and broadcast: every decision below
    // must be the same for the whole warp (its lanes may arrive here
    // diverged, and a lane leaving alone would strand the others' shuffles)
    unsigned flags = 0;
    if (lane == 0)
      flags = (*reinterpret_cast<volatile unsigned*>(&s_exit) != 0u ? 1u : 0u) |
              (*reinterpret_cast<volatile unsigned*>(&s_drain) != 0u ? 2u : 0u);
    flags = __shfl_sync(0xffffffffu, flags, 0);
    if (flags & 1u) break;
    const bool drain = (flags & 2u) != 0u;
    const long long t_round = CELER_LANE_CLOCK();  // diagnostic build only
    (void)t_round;
    // the kind with the most tracks waiting (lanes 0..7 look at one each)
    unsigned waiting = 0;
    if (lane < kLiveKeys) {
      const unsigned hd = *reinterpret_cast<volatile unsigned*>(&s_head[lane]);  // before the tail: hd <= tail
      waiting = *reinterpret_cast<volatile unsigned*>(&s_tail[lane]) - hd;
    }
    // (one warp-wide maximum of waiting << 8 | (255 - lane): the most
    // waiting, the lowest kind among equals)
    const unsigned kb = __reduce_max_sync(0xffffffffu, (waiting << 8) | (255u - (unsigned)lane));
    unsigned best = kb >> 8;
    const unsigned best_k = 255u - (kb & 0xFFu);
    // Charged tracks first: their steps carry a shower's longest chains of
    // dependent steps (the primary crossing layer after layer and radiating),
    // so the job ends sooner when they wait least; the photons' chains are
    // shorter. In whole-job runs the first kAnyPieceWarps warps take a piece
    // of any size, the others only full ones, so that with few tracks alive a
    // block's work is concentrated in full warps instead of spread over many
    // part-filled ones. A warp keeps the kind it ran last while at least half
    // as many of it wait, so that its code is still in the instruction cache.
    const unsigned ew = (lane == K_E_GEOM || lane == K_E_RANGE || lane == K_E_MOLLER || lane == K_E_BREMS) ? waiting : 0u;
    const unsigned ke = __reduce_max_sync(0xffffffffu, (ew << 8) | (255u - (unsigned)lane));
    const unsigned eb = ke >> 8, ek = 255u - (ke & 0xFFu);
    const unsigned w_last = __shfl_sync(0xffffffffu, waiting, last_k & 31u);
    const bool keep_last = last_k < (unsigned)kLiveKeys && w_last > 0 && 2u * w_last >= best;
    // (while draining any warp takes any piece: a warp that leaves the loop
    // may have been the last one allowed to take a small piece)
    const unsigned min_piece = (drain || warp < any_warps) ? 1u : 32u;
    unsigned pick_k = 0xFFu;
    if (eb >= min_piece) {
      pick_k = ek;
    } else if (best >= min_piece) {
      pick_k = (keep_last && w_last >= min_piece) ? last_k : best_k;
    }
    if (eb > 0) best = eb;  // fills count the charged tracks waiting first
    // fill (one warp at a time) when nothing waits, or when no full piece
    // waits and the block holds fewer than half its share of the tracks,
    // alive and queued, over all blocks (at least kAsyncFill): few tracks
    // spread over all SMs, many keep every block's pieces full (half the
    // share measured fastest: the full share, or kAsyncFill alone, lose
    // 6 % and 33 % on the 4 T calorimeter)
    const unsigned live = *reinterpret_cast<volatile unsigned*>(&s_live);
    unsigned take = 0, f0 = 0;
    unsigned long long first = 0;
    if (drain && best == 0) break;  // budget spent and nothing queued: the block's tracks sit between steps
    if (!drain && best < 32u && lane == 0 && atomicCAS(&s_filling, 0u, 1u) == 0u) {
      const unsigned free_now = *reinterpret_cast<volatile unsigned*>(&s_tail[kFreeQueue]) -
                                *reinterpret_cast<volatile unsigned*>(&s_head[kFreeQueue]);
      const long long a = (long long)*reinterpret_cast<volatile unsigned long long*>(&c->avail);
      const unsigned long long alive = *reinterpret_cast<volatile unsigned long long*>(&c->alive);
      unsigned long long target = (alive + (a > 0 ? (unsigned long long)a : 0ull) + (unsigned long long)nb - 1ull) /
                                  (unsigned long long)nb;
      target = (target + 1ull) / 2ull;
      if (target < kAsyncFill) target = kAsyncFill;
      if (free_now > 0 && a > 0 && (best == 0 || live < target)) {
        unsigned long long want = ((unsigned long long)a + (unsigned long long)nb - 1ull) / (unsigned long long)nb;
        const unsigned long long fill_up = live < target ? target - live : 0ull;
        if (want < fill_up) want = fill_up < (unsigned long long)a ? fill_up : (unsigned long long)a;
        if (want > 32ull) want = 32ull;
        if (want > free_now) want = free_now;
        const long long old = (long long)atomicAdd(&c->avail, 0ull - want);
        if (old >= (long long)want) {
          take = (unsigned)want;
          CELER_LANES_N(LS_FILL, take);
          first = atomicAdd(&c->head, want);
          f0 = atomicAdd(&s_head[kFreeQueue], take);  // only the filler claims free slots
          atomicAdd(&s_live, take);
        } else {
          atomicAdd(&c->avail, want);
        }
      }
      atomicExch(&s_filling, 0u);
    }
    take = __shfl_sync(0xffffffffu, take, 0);
    // this lane's track: a freshly filled one (step limit only) or one of a
    // claimed piece (its step, then the step limit), both through one code
    // path so that the step functions exist once in the loop
    unsigned my_li = 0xFFFFFFFFu;
    bool fresh = false;
    unsigned n = 0;
    if (take > 0) {
      first = __shfl_sync(0xffffffffu, first, 0);
      f0 = __shfl_sync(0xffffffffu, f0, 0);
      if ((unsigned)lane < take) {
        my_li = wq_read(p, w, kFreeQueue, f0 + (unsigned)lane);
        if (my_li != 0xFFFFFFFFu) {
          const uint32_t slot = local_slot(my_li, bid, nb);
          take_initializer<true>(p, first + (unsigned)lane, slot);
          atomicSub(&p.vacant[slot >> 5], 1u);
          atomicSub(&p.tile_vacant[slot >> 8], 1u);
          ++fill;
          fresh = true;
        }
      }
    } else if (pick_k != 0xFFu) {
      // claim up to 32 tracks of kind pick_k
      unsigned h = 0;
      if (lane == 0) {
        for (int a = 0; a < 8; ++a) {
          h = *reinterpret_cast<volatile unsigned*>(&s_head[pick_k]);
          const unsigned q = *reinterpret_cast<volatile unsigned*>(&s_tail[pick_k]) - h;
          if (q == 0) break;
          const unsigned want = q < 32u ? q : 32u;
          if (atomicCAS(&s_head[pick_k], h, h + want) == h) {
            n = want;
            CELER_LANES_N(LS_PIECE + (int)pick_k, n);
            break;
          }
        }
      }
      n = __shfl_sync(0xffffffffu, n, 0);
      if (n == 0) continue;
      last_k = pick_k;
      h = __shfl_sync(0xffffffffu, h, 0);
      if ((unsigned)lane < n) my_li = wq_read(p, w, (int)pick_k, h + (unsigned)lane);
    }
    if (take > 0 || n > 0) {
      unsigned long long n_def = 0;
#ifndef CELER_LANE_COUNTERS
      if (my_li != 0xFFFFFFFFu) {
        const uint32_t slot = local_slot(my_li, bid, nb);
        if (!fresh && step_one(p, slot, p.trk.status[slot], ss, true, n_def)) {
          ++killed;
          atomicSub(&s_live, 1u);
          wq_push(p, w, kFreeQueue, my_li);
        } else if (fresh || !drain) {
          wq_requeue(p, w, ss, slot, my_li, steps);
        }
      }
#else
      // the same work in two phases with the warp gathered between them, so
      // that the diagnostic build can time the claim, the step and the next
      // step limit of the photon and electron crossing pieces apart
      __syncwarp();
      const long long t_read = clock64();
      bool ended = false;
      if (my_li != 0xFFFFFFFFu && !fresh) {
        const uint32_t slot = local_slot(my_li, bid, nb);
        ended = step_one(p, slot, p.trk.status[slot], ss, true, n_def);
      }
      __syncwarp();
      const long long t_step = clock64();
      if (my_li != 0xFFFFFFFFu) {
        const uint32_t slot = local_slot(my_li, bid, nb);
        if (ended) {
          ++killed;
          atomicSub(&s_live, 1u);
          wq_push(p, w, kFreeQueue, my_li);
        } else if (fresh || !drain) {
          wq_requeue(p, w, ss, slot, my_li, steps);
        }
      }
      __syncwarp();
      if (lane == 0 && take == 0 && (pick_k == K_G_GEOM || pick_k == K_E_GEOM || pick_k == K_G_COMPTON)) {
        const int base = pick_k == K_G_GEOM ? LS_T_PHOTON : (pick_k == K_E_GEOM ? LS_T_ELECTRON : LS_T_COMPTON);
        CELER_LANES_N(base, n);
        CELER_LANE_CYCLES(base, t_read - t_round);
        CELER_LANES_N(base + 1, n);
        CELER_LANE_CYCLES(base + 1, t_step - t_read);
        CELER_LANES_N(base + 2, n);
        CELER_LANE_CYCLES(base + 2, clock64() - t_step);
      }
#endif
      if (lane == 0) CELER_LANE_CYCLES(take > 0 ? LS_FILL : LS_PIECE + (int)pick_k, CELER_LANE_CLOCK() - t_round);
      if ((++events & 15u) == 0) {  // the device counters every 16 pieces or fills, and whenever the warp idles
        wq_flush_counts(p, steps, killed, fill);
        steps = killed = fill = 0;
      }
      if (take > 0) continue;
      ++pieces;
      if (pieces >= budget && lane == 0) atomicExch(&s_drain, 1u);
      if (pieces >= max_pieces && lane == 0) {
        atomicOr(&c->error, ERR_ITERATIONS);
        atomicExch(p.barrier + 2, 1u);
        atomicExch(&s_exit, 1u);
      }
      // a piece without deferrals made progress; one with deferrals (the
      // buffer is full) goes on to the idle path: watchdog and a pause
      if (!__any_sync(0xffffffffu, n_def != 0)) continue;
    }
    // nothing done: leave if every track has ended, else poll (bounded)
    wq_flush_counts(p, steps, killed, fill);
    steps = killed = fill = 0;
    if (lane == 0) {
      if (*reinterpret_cast<volatile unsigned*>(p.barrier + 2) != 0u) {
        atomicExch(&s_exit, 1u);
      } else if (budget != ~0ull && *reinterpret_cast<volatile unsigned*>(&s_live) == 0u) {
        atomicExch(&s_drain, 1u);  // a budgeted run and no track here: the rest is left to the next run
      } else if (*reinterpret_cast<volatile unsigned*>(&s_live) == 0u) {
        const unsigned long long f = ld_acquire_u64(&c->finished);
        if (f == *reinterpret_cast<volatile unsigned long long*>(&c->tail)) atomicExch(&s_exit, 1u);
      }
      const unsigned long long now_steps = *reinterpret_cast<volatile unsigned long long*>(&c->steps_total);
      const long long now = clock64();
      if (now_steps != seen) {
        seen = now_steps;
        t_seen = now;
      } else if (now - t_seen > kBarrierTimeoutCycles) {
        atomicOr(&c->error, ERR_NO_PROGRESS);
        atomicExch(p.barrier + 2, 1u);
        atomicExch(&s_exit, 1u);
      }
      __nanosleep(500);
      CELER_LANES_N(LS_IDLE, 0u);
      CELER_LANE_CYCLES(LS_IDLE, CELER_LANE_CLOCK() - t_round);
    }
    __syncwarp();
  }
  wq_flush_counts(p, steps, killed, fill);
  if (lane == 0) atomicMax(&s_pieces, pieces);
  __syncthreads();
  if (threadIdx.x == 0) p.block_vacant[bid] = owned - s_live;
  return s_pieces;
}

// The asynchronous block loop of the block-pass policies (LOCAL, DATA): one
// cooperative launch in which every block runs its own passes over its own
// chunks with no grid barrier. At the start of a pass a block claims
// written entries on an availability count (atomic, undone if short) and
// takes their indices from the head: ceil(queued / blocks) or enough to hold
// kAsyncFill live tracks, at most its vacant slots. Secondaries are reserved
// at the tail against the current head, and each entry's state word orders
// its writer and its reader. A track's steps and draws do not depend
// on where or when it runs (its random stream is keyed by its own id), so
// histories are those of the synchronous loops; only the tally summation
// order differs. The run ends when every track taken from the buffer has
// ended (finished reaches tail), or, with an iteration budget, when every
// block has run that many passes or holds no track (warp_queue_loop: has
// drained). Every wait is bounded: a block with nothing to do polls, and if
// no track anywhere steps for ~1 s it sets ERR_NO_PROGRESS and the abort
// word; all blocks leave at their next pass. The last block to leave adds
// the most passes (pieces) any block ran to the iteration count.
__global__ void __launch_bounds__(kTile, 1) k_loop_async(Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SharedStatic ss = carve_static(p, smem_raw);
  stage_static(p, ss);
  const int nb = (int)gridDim.x, bid = (int)blockIdx.x;
  Ctl* c = p.ctl;
  unsigned* abort_word = p.barrier + 2;
  __shared__ unsigned long long s_first;
  __shared__ unsigned s_take, s_vtot;
  __shared__ int s_go;  // 0 leave, 1 nothing to do yet, 2 run a pass
  const uint32_t n_own = (uint32_t)bid < p.n_chunks ? (p.n_chunks - (uint32_t)bid + nb - 1) / nb : 0u;
  const bool owns_last = n_own > 0 && (uint32_t)bid + (uint32_t)nb * (n_own - 1u) == p.n_chunks - 1u;
  const unsigned owned = n_own * 32u - (owns_last ? p.n_chunks * 32u - p.n_slots : 0u);
  const unsigned quota_cap = block_quota_cap(p.policy);
  unsigned long long passes = 0, seen = ~0ull;
  const unsigned long long max_passes = __ldcg(&c->max_iterations);  // per run
  const unsigned long long budget_end = __ldcg(&c->budget_end);
  const unsigned long long budget = budget_end == ~0ull ? ~0ull : budget_end - __ldcg(&c->iteration);
  long long t_seen = clock64();
  if (threadIdx.x == 0) {
    s_vtot = __ldcg(&p.block_vacant[bid]);
    if (__ldcg(&c->local_blocks) != (unsigned)nb) {  // vacancy counts made for another grid
      atomicOr(&c->error, ERR_VACANCY);
      atomicExch(abort_word, 1u);
    }
  }
  __syncthreads();
  // block-local policy with per-warp scheduling: the block's warps run their
  // own loops, if the block's live tracks fit the queues (kWarpLive) and its
  // slot indices their 16 bits
  if (p.policy == POLICY_LOCAL && p.async_warps && owned - s_vtot <= kWarpLive && owned <= 0xFFFFu &&
      *reinterpret_cast<volatile unsigned*>(abort_word) == 0u) {
    passes = warp_queue_loop(p, bid, nb, ss, owned, owned - s_vtot, budget);
    if (threadIdx.x == 0) s_vtot = p.block_vacant[bid];
  } else {
  // thread 0: no track anywhere stepped for ~1 s
  auto watchdog = [&]() {
    const unsigned long long now_steps = *reinterpret_cast<volatile unsigned long long*>(&c->steps_total);
    const long long now = clock64();
    if (now_steps != seen) {
      seen = now_steps;
      t_seen = now;
    } else if (now - t_seen > kBarrierTimeoutCycles) {
      atomicOr(&c->error, ERR_NO_PROGRESS);
      atomicExch(abort_word, 1u);
    }
  };
  for (;;) {
    __syncthreads();  // every thread has read the previous decision
    if (threadIdx.x == 0) {
      int go = 1;
      unsigned take = 0;
      unsigned long long first = 0;
      const unsigned vtot = s_vtot;
      if (*reinterpret_cast<volatile unsigned*>(abort_word) != 0u || passes >= budget) {
        go = 0;  // aborted, or the run's budget of passes is spent
      } else {
        // claim `want` written entries on the availability count (undone if
        // there were fewer), then their indices on the head: at least
        // ceil(avail / blocks), and up to kAsyncFill live tracks in the block
        const unsigned room = vtot < quota_cap ? vtot : quota_cap;
        const long long a = (long long)*reinterpret_cast<volatile unsigned long long*>(&c->avail);
        if (room > 0 && a > 0) {
          const unsigned live = owned - vtot;
          unsigned long long want = ((unsigned long long)a + (unsigned long long)nb - 1ull) / (unsigned long long)nb;
          const unsigned long long fill_up = live < kAsyncFill ? (unsigned long long)(kAsyncFill - live) : 0ull;
          if (want < fill_up) want = fill_up < (unsigned long long)a ? fill_up : (unsigned long long)a;
          if (want > room) want = room;
          const long long old = (long long)atomicAdd(&c->avail, 0ull - want);
          if (old >= (long long)want) {
            take = (unsigned)want;
            first = atomicAdd(&c->head, want);
          } else {
            atomicAdd(&c->avail, want);
          }
        }
        if (take > 0 || vtot < owned) {
          go = 2;
        } else if (budget != ~0ull) {
          go = 0;  // a budgeted run: nothing here now, the rest is left to the next run
        } else {
          const unsigned long long f = ld_acquire_u64(&c->finished);
          if (f == *reinterpret_cast<volatile unsigned long long*>(&c->tail)) go = 0;  // every track has ended
        }
      }
      s_go = go;
      s_take = take;
      s_first = first;
    }
    __syncthreads();
    const int go = s_go;
    if (go == 0) break;
    if (go == 1) {
      if (threadIdx.x == 0) {
        watchdog();
        __nanosleep(1000);  // about a microsecond between polls of the shared counters
      }
      continue;
    }
    const PassPlan pl{s_first, s_take, s_vtot, true, false, 0u};
    PassCounts n{0, 0, 0, 0};
    if (p.policy == POLICY_DATA)
      data_pass<true>(p, bid, nb, ss, pl, n);
    else
      local_pass<true>(p, bid, nb, ss, pl, n);
    const PassCounts tot = block_total(n);
    if (threadIdx.x == 0) {
      if (tot.fill != pl.quota) atomicOr(&c->error, ERR_VACANCY);
      s_vtot = (unsigned)((long long)pl.vtot + (long long)tot.killed - (long long)tot.fill);
      if (tot.steps) atomicAdd(&c->steps_total, tot.steps);
      const long long dalive = (long long)tot.fill - (long long)tot.killed;
      if (dalive != 0) atomicAdd(&c->alive, (unsigned long long)dalive);
      if (tot.killed) {
        __threadfence();  // the block's reservations on the tail precede its count of ended tracks
        atomicAdd(&c->finished, tot.killed);
      }
      ++passes;
      if (passes >= max_passes) {
        atomicOr(&c->error, ERR_ITERATIONS);
        atomicExch(abort_word, 1u);
      }
      if (tot.steps == 0) watchdog();
    }
  }
  }
  if (threadIdx.x == 0) {
    p.block_vacant[bid] = s_vtot;
    atomicMax(&c->async_passes, passes);
    __threadfence();
    if (atomicAdd(&c->done_x, 1u) == (unsigned)nb - 1u) {
      __threadfence();
      c->iteration = __ldcg(&c->iteration) + __ldcg(&c->async_passes);
      const unsigned long long queued = __ldcg(&c->tail) - __ldcg(&c->head), alive = __ldcg(&c->alive);
      c->total_vacant = (unsigned long long)p.n_slots - alive;
      c->cont = (alive + queued > 0 && __ldcg(&c->error) == 0u) ? 1u : 0u;
      c->done_x = 0u;
    }
  }
}

// Check of the queue waits of the asynchronous loop: one thread waits for
// an entry to be written, either buffer entry 0 (which = 0, 2) or an entry
// of a shared-memory queue (which = 1, 3). For which = 0, 1 nothing writes
// it, so the wait must give up after `timeout` cycles, set the abort word
// and ERR_BARRIER_TIMEOUT; for which = 2, 3 it was written first and the
// wait must pass.
__global__ void k_queue_wait_probe(Params p, int which, long long timeout) {
  __shared__ unsigned s_e;
  if (threadIdx.x == 0) {
    s_e = (which & 2) ? (1u << 16) : 0u;  // lap 0: 0 free, 1 written
    if (which & 2) p.ring_state[0] = 1u;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (which & 1)
      wq_wait(p, &s_e, 1u, timeout);
    else
      ring_wait(p, 0ull, 1u, timeout);
  }
}

