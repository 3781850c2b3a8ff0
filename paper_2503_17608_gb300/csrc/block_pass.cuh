// The block pass of the block-pass policies (LOCAL, DATA): one pass per
// block over its own chunks b, b + nb, ... that fills its vacancies, steps
// its live tracks and (synchronous loops) ends with the last block's
// bookkeeping and the grid barrier. Holds the per-block vacancy counts and
// the level-filling plan of the fill, the iteration inputs read after each
// barrier, the passes themselves (local_pass, data_pass: shared by the
// synchronous and asynchronous loops) and the synchronous iteration
// (block_iteration). Included by step.cu inside its anonymous namespace.
#pragma once

// Block-wide exclusive scan of one count per thread (blockDim.x a multiple
// of 32, at most 32 warps); returns the thread's exclusive prefix and sets
// total to the block's sum. Every thread must call it.
__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned& total) {
  __shared__ unsigned s_w[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = (int)(blockDim.x >> 5);
  unsigned incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  __syncthreads();
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  unsigned before = 0, all = 0;
  for (int w = 0; w < nwarps; ++w) {
    const unsigned cw = s_w[w];
    before += w < warp ? cw : 0u;
    all += cw;
  }
  total = all;
  return before + incl - v;
}

// Vacant slots of this block's chunks b, b + nb, ... (block-local policy),
// summed by the whole block into block_vacant[b].
__device__ __forceinline__ void count_block_vacancies(const Params& p, int bid, int nb) {
  __shared__ unsigned long long s_r[32];
  const uint32_t n_own = (uint32_t)bid < p.n_chunks ? (p.n_chunks - (uint32_t)bid + nb - 1) / nb : 0u;
  unsigned long long own = 0;
  for (uint32_t m = threadIdx.x; m < n_own; m += blockDim.x) own += __ldcg(&p.vacant[(uint32_t)bid + (uint32_t)nb * m]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) own += __shfl_xor_sync(0xffffffffu, own, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) s_r[threadIdx.x >> 5] = own;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long sum = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s_r[w];
    p.block_vacant[bid] = (uint32_t)sum;
  }
}

// Level filling of the block-local policy's next fill, by one whole block:
// the `take` initializers are dealt to the nb blocks as evenly as their
// vacancies allow. With v_b the vacant slots of block b, the level L is the
// largest with sum_b min(v_b, L) <= take; block b takes min(v_b, L), plus one
// for the first (take - that sum) blocks, in block order, with v_b > L. The
// quotas' exclusive scan gives each block's first initializer. Fresh tracks
// thus spread over all SMs (a block fills its lowest vacancies, in its chunk
// order), and the fill stays deterministic. s_v holds v_b; vmin and vmax
// are their extremes. When every block has room for take/nb + 1 the level
// is take/nb; otherwise one warp finds it by bisection. A block takes at most
// `cap` (its counts and the take are clamped); returns the take planned,
// which the caller stores as the next fill_take.
__device__ unsigned long long plan_block_quotas(const Params& p, uint32_t* s_v, int nb, unsigned vmin, unsigned vmax,
                                                unsigned long long take, unsigned cap) {
  __shared__ unsigned s_level, s_extra;
  __shared__ unsigned long long s_room;
  const int lane = threadIdx.x & 31;
  if (vmax > cap) {  // a block takes at most `cap`: clamp the counts, and the take to their sum
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s_v[b] = min(s_v[b], cap);
    __syncthreads();
    if (threadIdx.x < 32) {
      unsigned long long sm = 0;
      for (int b = lane; b < nb; b += 32) sm += s_v[b];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
      if (lane == 0) s_room = sm;
    }
    __syncthreads();
    if (take > s_room) take = s_room;
    vmin = min(vmin, cap);
    vmax = cap;
  }
  const unsigned long long l0 = take / (unsigned)nb;
  if (l0 + 1 <= vmin) {
    if (threadIdx.x == 0) {
      s_level = (unsigned)l0;
      s_extra = (unsigned)(take - l0 * (unsigned)nb);
    }
  } else if (threadIdx.x < 32) {
    unsigned lo = 0, hi = vmax;  // S(0) = 0 <= take <= S(vmax) = sum v_b
    unsigned long long s_lo = 0;
    while (lo < hi) {
      const unsigned mid = lo + (hi - lo + 1) / 2;
      unsigned long long sm = 0;
      for (int b = lane; b < nb; b += 32) sm += min(s_v[b], mid);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sm += __shfl_xor_sync(0xffffffffu, sm, o);
      if (sm <= take) {
        lo = mid;
        s_lo = sm;
      } else {
        hi = mid - 1;
      }
    }
    if (lane == 0) {
      s_level = lo;
      s_extra = (unsigned)(take > s_lo ? take - s_lo : 0ull);
    }
  }
  __syncthreads();
  const unsigned L = s_level, extra = s_extra;
  unsigned above_before = 0;
  unsigned long long quota_before = 0;
  for (int b0 = 0; b0 < nb; b0 += (int)blockDim.x) {
    const int b = b0 + (int)threadIdx.x;
    const unsigned v = b < nb ? s_v[b] : 0u;
    const unsigned above = v > L ? 1u : 0u;
    unsigned round_above = 0, round_quota = 0;
    const unsigned rank = above_before + block_exclusive_scan(above, round_above);
    const unsigned q = b < nb ? min(v, L) + ((above && rank < extra) ? 1u : 0u) : 0u;
    const unsigned qpre = block_exclusive_scan(q, round_quota);
    if (b < nb) {
      p.block_quota[b] = q;
      p.block_prefix[b] = quota_before + qpre;
    }
    above_before += round_above;
    quota_before += round_quota;
  }
  return take;
}

// Per-block vacancy counts into shared memory (whole block) with their sum
// and extremes (one warp); block_vacant holds them (count_block_vacancies).
__device__ __forceinline__ void load_block_vacancies(const Params& p, uint32_t* s_v, int nb, unsigned long long* sum,
                                                     unsigned* vmin, unsigned* vmax) {
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s_v[b] = __ldcg(&p.block_vacant[b]);
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    unsigned lo = 0xFFFFFFFFu, hi = 0;
    unsigned long long sm = 0;
    for (int b = lane; b < nb; b += 32) {
      lo = min(lo, s_v[b]);
      hi = max(hi, s_v[b]);
      sm += s_v[b];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      sm += __shfl_xor_sync(0xffffffffu, sm, o);
    }
    if (lane == 0) {
      *sum = sm;
      *vmin = lo;
      *vmax = hi;
    }
  }
  __syncthreads();
}

// Largest quota a block takes in one iteration: the DATA policy keeps its
// block's initializer list in shared memory.
constexpr unsigned kDataMaxQuota = 8192;
__device__ __forceinline__ unsigned block_quota_cap(int policy) { return policy == POLICY_DATA ? kDataMaxQuota : 0xFFFFFFFFu; }

// Bounded wait of one thread for the generation word (barrier[1]) to move
// past g: the persistent loops' grid barriers. After `timeout` cycles (about
// 1 s by default) the thread sets the abort word (barrier[2]) and
// ERR_BARRIER_TIMEOUT and gives up; a waiter that sees the abort word gives
// up too, so every block leaves its loop at its next barrier and the kernel
// ends with an error status the host reads. Returns true if the generation
// moved and no abort was raised.
__device__ __forceinline__ bool wait_generation(const Params& p, unsigned g, long long timeout) {
  unsigned int* gen = p.barrier + 1;
  unsigned int* abort_word = p.barrier + 2;
  const long long t0 = clock64();
  for (;;) {
    if (*reinterpret_cast<volatile unsigned*>(gen) != g) break;
    if (*reinterpret_cast<volatile unsigned*>(abort_word) != 0u) return false;
    if (clock64() - t0 > timeout) {
      atomicExch(abort_word, 1u);
      atomicOr(&p.ctl->error, ERR_BARRIER_TIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
  return *reinterpret_cast<volatile unsigned*>(abort_word) == 0u;
}

// Per-iteration inputs of a block pass, read in one batch of loads (from
// L2) right after the previous iteration's barrier: the loop condition, the
// fill plan (buffer head, entries taken, whether secondaries may overflow),
// this block's quota, first entry and vacancy count, and this thread's
// chunk vacancy of the first batch (chunk bid + nb * threadIdx.x).
struct BlockIter {
  unsigned long long head, take, prefix, iteration;
  unsigned quota, vtot, vac0;
  bool cont, tight, blocks_ok;
};
__device__ __forceinline__ BlockIter load_block_iter(const Params& p, int bid, int nb) {
  const Ctl* c = p.ctl;
  BlockIter it;
  it.cont = __ldcg(&c->cont) != 0u;
  it.head = __ldcg(&c->head);
  it.take = __ldcg(&c->fill_take);
  it.iteration = __ldcg(&c->iteration);
  it.tight = __ldcg(&c->defer_local) != 0u;
  it.blocks_ok = __ldcg(&c->local_blocks) == (unsigned)nb;
  it.quota = __ldcg(&p.block_quota[bid]);
  it.prefix = __ldcg(&p.block_prefix[bid]);
  it.vtot = __ldcg(&p.block_vacant[bid]);
  const uint32_t n_own = (uint32_t)bid < p.n_chunks ? (p.n_chunks - (uint32_t)bid + nb - 1) / nb : 0u;
  it.vac0 = threadIdx.x < n_own ? __ldcg(&p.vacant[(uint32_t)bid + (uint32_t)nb * threadIdx.x]) : 0u;
  return it;
}

// End of a block pass (LOCAL, DATA). The block's vacancy count is its count
// at the start plus its releases minus its fills (only the block touches its
// chunks). The last block to take a ticket commits the fill, takes the
// vacancy totals from the per-block counts (the per-tile prefix is left to
// the next run of another policy), ends the iteration and plans the next
// fill. In the persistent loop the ticket doubles as the grid barrier: the
// other blocks wait (bounded) for the last one to bump the generation word,
// so an iteration costs one global atomic per block. Returns false if the
// wait gave up (abort word set, ERR_BARRIER_TIMEOUT).
__device__ bool end_block_pass(const Params& p, int bid, int nb, const BlockIter& it, long long vdelta, bool persistent,
                               cudaGraphConditionalHandle handle, int use_handle, long long t_work0) {
  const unsigned long long head = it.head, take = it.take;
  __shared__ long long s_delta;
  __shared__ unsigned s_last, s_gen;
  __shared__ int s_ok;
  Ctl* c = p.ctl;
  unsigned* gen = p.barrier + 1;
  if (threadIdx.x == 0) s_delta = 0;
  __syncthreads();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vdelta += __shfl_xor_sync(0xffffffffu, vdelta, o);
  if ((threadIdx.x & 31) == 0 && vdelta != 0) atomicAdd((unsigned long long*)&s_delta, (unsigned long long)vdelta);
  __syncthreads();
  if (threadIdx.x == 0) {
    p.block_vacant[bid] = (uint32_t)((long long)it.vtot + s_delta);
    if (persistent) {
      atomicMax(&c->iter_max[it.iteration & 1][2], (unsigned long long)(clock64() - t_work0));
      s_gen = *reinterpret_cast<volatile unsigned*>(gen);
    }
    __threadfence();
    const unsigned ticket = atomicAdd(&c->done_c, 1u);
    s_last = (ticket == (unsigned)nb - 1u) ? 1u : 0u;
    if (s_last) *reinterpret_cast<volatile unsigned*>(&c->done_c) = 0u;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    __shared__ uint32_t s_v[kMaxLoopBlocks];
    __shared__ unsigned long long s_sum, s_take;
    __shared__ unsigned s_vmin, s_vmax;
    const long long t0 = clock64();
    if (threadIdx.x == 0) {
      if (c->filled_total != take) c->error |= ERR_VACANCY;
      c->filled_total = 0;
      c->head = head + take;
      c->alive += take;
    }
    load_block_vacancies(p, s_v, nb, &s_sum, &s_vmin, &s_vmax);
    if (threadIdx.x == 0) c->total_vacant = s_sum;
    __syncthreads();
    if (threadIdx.x < 32) loop_ctl_warp(p, &s_take);
    __syncthreads();
    const unsigned long long planned = plan_block_quotas(p, s_v, nb, s_vmin, s_vmax, s_take, block_quota_cap(p.policy));
    if (threadIdx.x == 0) {
      if (planned != s_take) c->fill_take = planned;
      if (use_handle) cudaGraphSetConditional(handle, c->cont);
      c->book_total[1] += (unsigned long long)(clock64() - t0);
    }
    __syncthreads();
    if (persistent && threadIdx.x == 0) {
      __threadfence();
      atomicAdd(gen, 1u);
    }
    return true;
  }
  if (!persistent) return true;
  if (threadIdx.x == 0) {
    const bool ok = wait_generation(p, s_gen, kBarrierTimeoutCycles);
    __threadfence();
    s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  return s_ok != 0;
}

// Plan of one block pass: the first initializer the block takes and how many,
// its vacant slots at the start of the pass, whether secondaries reserve
// their entries by compare-and-swap, and (synchronous loops) this thread's
// chunk vacancy of the first batch, read with the iteration's other inputs.
struct PassPlan {
  unsigned long long first;
  unsigned quota, vtot;
  bool tight, have_vac0;
  unsigned vac0;
};
// Per-thread counts of a pass: tracks ended, deferred, stepped; slots filled.
struct PassCounts {
  unsigned long long killed, n_def, steps, fill;
};

// Copy buffer entry `index` into `slot` as a fresh track. In the asynchronous
// loop the entry may still be in its writer's hands: wait (bounded) until it
// is written, read it from L2, and mark it read. A wait that gives up leaves
// the slot vacant; the run then ends with ERR_BARRIER_TIMEOUT.
template <bool kAsync>
__device__ __forceinline__ void take_initializer(const Params& p, unsigned long long index, uint32_t slot) {
  const Tracks& t = p.trk;
  const unsigned long long i = index & p.ring_mask;
  unsigned code = 0;
  if (kAsync) {
    code = ring_lap_code(p, index) + 1u;
    if (!ring_wait(p, index, code)) return;
  }
  t.x[slot] = __ldcg(&p.ring.x[i]);
  t.y[slot] = __ldcg(&p.ring.y[i]);
  t.z[slot] = __ldcg(&p.ring.z[i]);
  t.ux[slot] = __ldcg(&p.ring.ux[i]);
  t.uy[slot] = __ldcg(&p.ring.uy[i]);
  t.uz[slot] = __ldcg(&p.ring.uz[i]);
  t.E[slot] = __ldcg(&p.ring.E[i]);
  t.tid[slot] = __ldcg(&p.ring.tid[i]);
  t.event[slot] = __ldcg(&p.ring.event[i]);
  t.primary[slot] = __ldcg(&p.ring.primary[i]);
  t.layer[slot] = __ldcg(&p.ring.layer[i]);
  t.ptype[slot] = __ldcg(&p.ring.ptype[i]);
  t.ctr[slot] = 0u;
  t.nmfp[slot] = -1.0;
  t.action[slot] = A_NONE;
  t.status[slot] = ALIVE;
  if (kAsync) st_release_u32(p.ring_state + i, code + 1u);
}

// One pass of the DATA policy (Sec. 3.2, "partitioning track data") over
// block b's chunks b, b + nb, ...: the block takes its initializers (pl);
// among them the neutral ones fill its lowest vacant slots (its chunk order,
// then slot order) and the charged ones its highest, so that neutral and
// charged tracks gather at opposite ends of the block's slots and most warps
// hold one kind. There is no reindexing: each warp takes one of the block's
// chunks that hold or receive tracks, fills it, and runs the step limit,
// along-step and interaction of its live tracks in slot order, masking the
// others (Sec. 2).
template <bool kAsync>
__device__ void data_pass(const Params& p, int bid, int nb, const SharedStatic& ss, const PassPlan& pl,
                          PassCounts& n) {
  __shared__ uint32_t s_chunks[kTile];
  __shared__ uint32_t s_cpre[kTile];
  __shared__ unsigned s_wn[kTile / 32];
  __shared__ unsigned short s_list[kDataMaxQuota];  // offsets in the quota: neutral from the front, charged from the back
  __shared__ unsigned s_acts[A_COUNT];
  Ctl* c = p.ctl;
  const Tracks& t = p.trk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const unsigned lt = (1u << lane) - 1u;
  if (!kAsync && threadIdx.x < A_COUNT) s_acts[threadIdx.x] = 0u;
  const unsigned quota = min(pl.quota, kDataMaxQuota);
  const unsigned long long first = pl.first;
  const unsigned vtot = pl.vtot;  // the block's vacant slots at the start of the pass
  // the block's initializers by kind: offsets of the neutral ones in order
  // from the front of s_list, of the charged ones from the back
  unsigned n_neutral = 0;
  for (unsigned e0 = 0; e0 < quota; e0 += blockDim.x) {
    const unsigned e = e0 + threadIdx.x;
    const bool in = e < quota;
    bool neutral = false;
    if (in) {
      if (!kAsync || ring_wait(p, first + e, ring_lap_code(p, first + e) + 1u))
        neutral = __ldcg(&p.ring.ptype[(first + e) & p.ring_mask]) == GAMMA;
    }
    unsigned round_n = 0;
    const unsigned rn = n_neutral + block_exclusive_scan(neutral ? 1u : 0u, round_n);
    if (neutral) {
      s_list[rn] = (unsigned short)e;
    } else if (in) {
      s_list[quota - 1u - (e - rn)] = (unsigned short)e;  // e - rn charged ones precede it
    }
    n_neutral += round_n;
  }
  const unsigned n_charged = quota - n_neutral;
  __syncthreads();
  const uint32_t n_own = (uint32_t)bid < p.n_chunks ? (p.n_chunks - (uint32_t)bid + nb - 1) / nb : 0u;
  unsigned run = 0;  // the block's vacancies before the next batch (ascending rank)
  for (uint32_t c0 = 0; c0 < n_own; c0 += blockDim.x) {
    const uint32_t m = c0 + threadIdx.x;
    const uint32_t g = (uint32_t)bid + (uint32_t)nb * m;
    unsigned vac = 0, csize = 0;
    if (m < n_own) {
      csize = (p.n_slots - g * 32u) < 32u ? (p.n_slots - g * 32u) : 32u;
      vac = (c0 == 0 && pl.have_vac0) ? pl.vac0 : __ldcg(&p.vacant[g]);
    }
    unsigned batch_vac = 0;
    const unsigned pre = block_exclusive_scan(vac, batch_vac);
    // ascending ranks of the chunk's vacancies: [a, a + vac); it receives a
    // neutral track if a < n_neutral, a charged one if its highest vacancy's
    // descending rank, vtot - (a + vac), is below n_charged
    const unsigned a = run + pre;
    const bool cand = m < n_own && (vac < csize || (vac > 0 && (a < n_neutral || vtot - (a + vac) < n_charged)));
    const unsigned bal = __ballot_sync(0xffffffffu, cand);
    __syncthreads();
    if (lane == 0) s_wn[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, nch = 0;
    for (int w = 0; w < nwarps; ++w) {
      const unsigned cw = s_wn[w];
      before += w < warp ? cw : 0u;
      nch += cw;
    }
    if (cand) {
      s_chunks[before + __popc(bal & lt)] = g;
      s_cpre[before + __popc(bal & lt)] = pre;
    }
    __syncthreads();
    const unsigned run0 = run;
    run += batch_vac;
    for (unsigned j = (unsigned)warp; j < nch; j += (unsigned)nwarps) {
      const uint32_t gc = s_chunks[j];
      const uint32_t slot = gc * 32u + lane;
      const bool real = slot < p.n_slots;
      const bool vac_l = real && t.status[slot] == VACANT;
      const unsigned vb = __ballot_sync(0xffffffffu, vac_l);
      const unsigned r = run0 + s_cpre[j] + __popc(vb & lt);
      int off = -1;
      if (vac_l) {
        if (r < n_neutral) {
          off = s_list[r];
        } else if (vtot - 1u - r < n_charged) {
          off = s_list[quota - 1u - (vtot - 1u - r)];
        }
      }
      if (off >= 0) take_initializer<kAsync>(p, first + (unsigned)off, slot);
      const unsigned nfill = __popc(__ballot_sync(0xffffffffu, off >= 0));
      if (lane == 0 && nfill) {
        atomicSub(&p.vacant[gc], nfill);
        atomicSub(&p.tile_vacant[gc >> 3], nfill);
        n.fill += nfill;
      }
      // the chunk's live tracks: step limit, along-step, interaction
      if (real) {
        const uint8_t st = t.status[slot];
        if (st != VACANT) {
          uint8_t act;
          if (st == ALIVE) {
            act = step_limit(p, slot, ss.tab, ss.zb, ss.lmat);
            ++n.steps;
          } else {
            act = t.action[slot];
          }
          if (!kAsync) atomicAdd(&s_acts[act], 1u);
          if (step_one(p, slot, st, ss, pl.tight, n.n_def)) ++n.killed;
        }
      }
    }
  }
  if (!kAsync) {
    __syncthreads();
    if (threadIdx.x < A_COUNT && s_acts[threadIdx.x] != 0) atomicAdd(&c->action_count[threadIdx.x], s_acts[threadIdx.x]);
  }
}

// One pass of the block-local policy over block b's chunks b, b + nb, ...,
// with no grid barrier between the fill and the step:
//  * fill: the block's lowest vacant slots (its chunk order, then slot order
//    within a chunk) take its initializers (pl);
//  * step limit of each live track of the chunk, by the warp that filled it;
//  * the live tracks gathered into shared memory a few hundred at a time and
//    grouped by key (action and particle type) with a counting sort; each
//    group is cut into pieces of 8, 16 or 32 (the smallest size whose piece
//    count fits the warps) and the pieces are dealt to the warps: every warp
//    runs one kind of along-step and interaction, and few tracks spread over
//    all warps.
// Secondaries go to the buffer's tail while the taken entries are being read:
// the capacity checks count from the uncommitted head (synchronous loops) or
// wait for the entries' readers (asynchronous loop).
template <bool kAsync>
__device__ void local_pass(const Params& p, int bid, int nb, const SharedStatic& ss, const PassPlan& pl,
                           PassCounts& n) {
  constexpr int kCap = 2 * kTile;
  constexpr int kMaxPieces = kCap / 8 + kMaxKeys;
  __shared__ uint32_t s_slot[kCap];
  __shared__ uint32_t s_sorted[kCap];
  __shared__ uint8_t s_key[kCap];
  __shared__ uint32_t s_chunks[kTile];
  __shared__ uint32_t s_cpre[kTile];
  __shared__ unsigned s_wn[kTile / 32];
  __shared__ unsigned s_cnt[kMaxKeys], s_cur[kMaxKeys];
  __shared__ unsigned short s_pstart[kMaxPieces];
  __shared__ unsigned char s_plen[kMaxPieces];
  __shared__ unsigned s_npieces;
  __shared__ unsigned s_acts[A_COUNT];
  Ctl* c = p.ctl;
  const Tracks& t = p.trk;
  const bool tight = pl.tight;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (int)(blockDim.x >> 5);
  const unsigned lt = (1u << lane) - 1u;
  if (!kAsync && threadIdx.x < A_COUNT) s_acts[threadIdx.x] = 0u;
  const unsigned quota = pl.quota;  // initializers this block takes
  const unsigned long long first = pl.first;
  unsigned run = 0;  // the block's vacancies before the next batch
  // group the n gathered slots by key and run them, one piece per warp
  auto flush = [&](unsigned ng) {
    if (threadIdx.x < kMaxKeys) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (unsigned i = threadIdx.x; i < ng; i += blockDim.x) atomicAdd(&s_cnt[s_key[i]], 1u);
    __syncthreads();
    if (threadIdx.x < 32) {
      // one lane per key, keys taken in the order of kPieceOrder (the
      // interactions first: piece q runs on warp q mod nwarps, so the costly
      // pieces get sub-partitions, and FP64 pipes, of their own)
      const int k = lane < kMaxKeys ? (int)kPieceOrder[lane] : 0;
      const unsigned ck = lane < kMaxKeys ? s_cnt[k] : 0u;
      unsigned piece = 32u;
      for (unsigned pc = 8u; pc <= 32u; pc <<= 1) {  // smallest piece size whose pieces fit the warps
        unsigned np = (ck + pc - 1) / pc;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) np += __shfl_xor_sync(0xffffffffu, np, o);
        if (np <= (unsigned)nwarps) {
          piece = pc;
          break;
        }
      }
      const unsigned mine = (ck + piece - 1) / piece;
      unsigned off = ck, pstart = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned a = __shfl_up_sync(0xffffffffu, off, o), b = __shfl_up_sync(0xffffffffu, pstart, o);
        if (lane >= o) {
          off += a;
          pstart += b;
        }
      }
      off -= ck;
      pstart -= mine;
      if (lane < kMaxKeys) {
        s_cur[k] = off;
        for (unsigned q = 0; q < mine; ++q) {
          s_pstart[pstart + q] = (unsigned short)(off + q * piece);
          s_plen[pstart + q] = (unsigned char)(ck - q * piece < piece ? ck - q * piece : piece);
        }
      }
      if (lane == 31) s_npieces = pstart + mine;
    }
    __syncthreads();
    for (unsigned i = threadIdx.x; i < ng; i += blockDim.x) s_sorted[atomicAdd(&s_cur[s_key[i]], 1u)] = s_slot[i];
    __syncthreads();
    const unsigned npieces = s_npieces;
    for (unsigned q = (unsigned)warp; q < npieces; q += (unsigned)nwarps) {
      if ((unsigned)lane >= s_plen[q]) continue;
      const uint32_t sl = s_sorted[s_pstart[q] + lane];
      if (step_one(p, sl, t.status[sl], ss, tight, n.n_def)) ++n.killed;
    }
    __syncthreads();  // the lists are reused by the next gather
  };
  const uint32_t n_own = (uint32_t)bid < p.n_chunks ? (p.n_chunks - (uint32_t)bid + nb - 1) / nb : 0u;
  unsigned pending = 0;  // gathered and not yet run (block-uniform)
  for (uint32_t c0 = 0; c0 < n_own; c0 += blockDim.x) {
    // this batch's chunks: start-of-pass vacancies and their exclusive scan
    // (fill ranks); a chunk is visited if it holds live tracks or receives
    // initializers
    const uint32_t m = c0 + threadIdx.x;
    const uint32_t g = (uint32_t)bid + (uint32_t)nb * m;
    unsigned vac = 0, csize = 0;
    if (m < n_own) {
      csize = (p.n_slots - g * 32u) < 32u ? (p.n_slots - g * 32u) : 32u;
      vac = (c0 == 0 && pl.have_vac0) ? pl.vac0 : __ldcg(&p.vacant[g]);
    }
    unsigned batch_vac = 0;
    const unsigned pre = block_exclusive_scan(vac, batch_vac);
    const bool cand = m < n_own && (vac < csize || (vac > 0 && run + pre < quota));
    const unsigned bal = __ballot_sync(0xffffffffu, cand);
    __syncthreads();  // the previous batch is done with s_wn / s_chunks / s_cpre
    if (lane == 0) s_wn[warp] = __popc(bal);
    __syncthreads();
    unsigned before = 0, nch = 0;
    for (int w = 0; w < nwarps; ++w) {
      const unsigned cw = s_wn[w];
      before += w < warp ? cw : 0u;
      nch += cw;
    }
    if (cand) {
      s_chunks[before + __popc(bal & lt)] = g;
      s_cpre[before + __popc(bal & lt)] = pre;
    }
    __syncthreads();
    const unsigned run0 = run;
    run += batch_vac;
    for (unsigned j0 = 0; j0 < nch; j0 += (unsigned)nwarps) {
      // one chunk per warp: fill, step limit, key; live slots appended after
      // the `pending` entries
      const unsigned j = j0 + (unsigned)warp;
      bool live = false;
      uint32_t slot = 0;
      uint8_t key = 0;
      if (j < nch) {
        const uint32_t gc = s_chunks[j];
        const unsigned q = run0 + s_cpre[j];
        slot = gc * 32u + lane;
        const bool real = slot < p.n_slots;
        if (q < quota) {
          const bool vac_l = real && t.status[slot] == VACANT;
          const unsigned vb = __ballot_sync(0xffffffffu, vac_l);
          const unsigned r = q + __popc(vb & lt);
          if (vac_l && r < quota) take_initializer<kAsync>(p, first + r, slot);
          const unsigned left = quota - q;
          const unsigned nfill = (unsigned)__popc(vb) < left ? (unsigned)__popc(vb) : left;
          if (lane == 0 && nfill) {
            atomicSub(&p.vacant[gc], nfill);
            atomicSub(&p.tile_vacant[gc >> 3], nfill);
            n.fill += nfill;
          }
        }
        if (real) {
          const uint8_t st = t.status[slot];
          uint8_t act = A_NONE;
          if (st == ALIVE) {
            act = step_limit(p, slot, ss.tab, ss.zb, ss.lmat);
            ++n.steps;
          } else if (st == DEFERRED) {
            act = t.action[slot];
          }
          if (st != VACANT) {
            if (!kAsync) atomicAdd(&s_acts[act], 1u);
            live = true;
            key = key_of(POLICY_ACTION_TYPE, t.ptype[slot], act);
          }
        }
      }
      const unsigned lb = __ballot_sync(0xffffffffu, live);
      if (lane == 0) s_wn[warp] = __popc(lb);
      __syncthreads();
      unsigned wb = 0, add = 0;
      for (int w = 0; w < nwarps; ++w) {
        const unsigned cw = s_wn[w];
        wb += w < warp ? cw : 0u;
        add += cw;
      }
      if (live) {
        const unsigned pos = pending + wb + __popc(lb & lt);
        s_slot[pos] = slot;
        s_key[pos] = key;
      }
      pending += add;
      __syncthreads();
      if (pending >= (unsigned)kTile) {
        flush(pending);
        pending = 0;
      }
    }
  }
  if (pending > 0) flush(pending);
  if (!kAsync) {
    __syncthreads();
    if (threadIdx.x < A_COUNT && s_acts[threadIdx.x] != 0) atomicAdd(&c->action_count[threadIdx.x], s_acts[threadIdx.x]);
  }
}

// One whole iteration of a block-pass policy in the synchronous loops: the
// pass over the block's chunks with the fill planned at the end of the
// previous iteration by level filling (plan_block_quotas: a deterministic
// fill that needs no other block's counts during the iteration and spreads
// fresh tracks over all SMs), then the end of the block's pass, where the
// last block to finish commits the fill, scans the per-block and per-tile
// vacancy counts and ends the iteration (which plans the next fill).
__device__ bool block_iteration(const Params& p, int bid, int nb, const SharedStatic& ss,
                                cudaGraphConditionalHandle handle, int use_handle, bool persistent,
                                const BlockIter& it) {
  const long long t_work0 = clock64();
  Ctl* c = p.ctl;
  if (bid == 0 && threadIdx.x == 0 && !it.blocks_ok) atomicOr(&c->error, ERR_VACANCY);
  const PassPlan pl{it.head + it.prefix, it.quota, it.vtot, it.tight, true, it.vac0};
  PassCounts n{0, 0, 0, 0};
  if (p.policy == POLICY_DATA)
    data_pass<false>(p, bid, nb, ss, pl, n);
  else
    local_pass<false>(p, bid, nb, ss, pl, n);
  flush_counter(&c->alive, n.killed, true);
  flush_counter(&c->steps_iter, n.steps, false);
  flush_counter(&c->filled_total, n.fill, false);
  if (n.n_def) atomicAdd(&c->n_deferred, (unsigned)n.n_def);
  return end_block_pass(p, bid, nb, it, (long long)n.killed - (long long)n.fill, persistent, handle, use_handle,
                        t_work0);
}

