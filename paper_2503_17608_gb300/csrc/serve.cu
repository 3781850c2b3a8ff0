// Serving loop (continuous batching of arriving events) and the autotuner
// of the launch configuration, both host code on top of the C ABI.
//
// Serving follows the paper's standalone mode (Sec. 5.1: events mixed in a
// single track array): tracks of every admitted event stay resident in the
// slot store across step iterations, new events are admitted between chunks
// of iterations as slots and initializer-buffer space free up, and finished
// events are collected by their live-track counts.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "celer_gb.h"
#include <cuda_runtime.h>

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0) {
  return std::chrono::duration<double>(Clock::now() - t0).count();
}

struct InFlight {
  uint64_t req;
  uint32_t row;
  double reserved;
};

}  // namespace

extern "C" celer_status celer_serve(celer_ctx* ctx, const celer_request* reqs, uint64_t n,
                                    const celer_serve_options* opt_in, celer_request_result* results,
                                    celer_serve_summary* summary) {
  if (!ctx || (n > 0 && (!reqs || !results))) return CELER_ERR_INVALID;
  celer_serve_options opt{};
  if (opt_in) opt = *opt_in;
  if (opt.chunk_iterations == 0) opt.chunk_iterations = 16;
  if (opt.footprint_per_primary <= 0.0) opt.footprint_per_primary = 40.0;
  for (uint64_t i = 1; i < n; ++i)
    if (reqs[i].arrival_s < reqs[i - 1].arrival_s) return CELER_ERR_INVALID;

  celer_step_stats st{};
  celer_status s = celer_get_stats(ctx, &st);
  if (s != CELER_OK) return s;
  const uint64_t steps0 = st.steps_total;

  // capacity in tracks: the slot store plus the initializer buffer
  uint64_t n_slots = 0, ring = 0, max_events = 0, n_bins = 0;
  {
    celer_problem pb{};
    s = celer_get_problem(ctx, &pb);
    if (s != CELER_OK) return s;
    n_slots = pb.n_slots;
    ring = 1;
    while (ring < pb.init_capacity) ring <<= 1;
    max_events = pb.max_events;
    n_bins = pb.tally_mode == CELER_TALLY_LAYERS ? (uint64_t)pb.n_layers * pb.n_periods : (uint64_t)pb.n_zbins;
  }
  const double capacity = (double)(n_slots + ring);
  std::vector<uint8_t> row_busy(max_events, 0);
  std::vector<uint32_t> live(max_events, 0);
  std::vector<double> tally(n_bins);
  std::vector<InFlight> inflight;
  double reserved = 0.0;

  for (uint64_t i = 0; i < n; ++i) {
    results[i].arrival_s = reqs[i].arrival_s;
    results[i].admit_s = -1.0;
    results[i].done_s = -1.0;
    results[i].edep = 0.0;
    results[i].escaped = 0.0;
  }
  uint64_t next = 0, admitted = 0, completed = 0, chunks = 0;
  const Clock::time_point t0 = Clock::now();
  double last_done = 0.0;

  for (;;) {
    double now = seconds_since(t0);
    // admission, in arrival order, while the head request fits
    while (next < n && reqs[next].arrival_s <= now) {
      const celer_request& q = reqs[next];
      if (opt.stop_admitting_s > 0.0 && now > opt.stop_admitting_s) break;
      if (opt.max_in_flight && inflight.size() >= opt.max_in_flight) break;
      const uint32_t row = (uint32_t)(q.event % max_events);
      if (row_busy[row]) break;
      const double need = std::max((double)q.n, opt.footprint_per_primary * (double)q.n);
      if (!inflight.empty() && reserved + need > capacity) break;
      s = celer_reset_event(ctx, q.event);
      if (s != CELER_OK) return s;
      s = celer_add_primaries(ctx, q.event, q.primaries, q.n);
      if (s == CELER_ERR_CAPACITY && !inflight.empty()) break;  // wait for space
      if (s != CELER_OK) return s;
      row_busy[row] = 1;
      reserved += need;
      inflight.push_back(InFlight{next, row, need});
      results[next].admit_s = seconds_since(t0);
      ++admitted;
      ++next;
    }
    if (inflight.empty()) {
      if (next >= n) break;
      if (opt.stop_admitting_s > 0.0 && seconds_since(t0) > opt.stop_admitting_s) break;
      const double wait = reqs[next].arrival_s - seconds_since(t0);
      if (wait > 2e-4) std::this_thread::sleep_for(std::chrono::duration<double>(wait - 1e-4));
      continue;
    }
    // a chunk of step iterations over every resident track
    uint64_t done = 0;
    s = celer_run_iterations(ctx, opt.mode, opt.chunk_iterations, &done);
    if (s != CELER_OK) return s;
    ++chunks;
    // collect finished events
    s = celer_read_event_live(ctx, 0, (uint32_t)max_events, live.data());
    if (s != CELER_OK) return s;
    for (size_t k = 0; k < inflight.size();) {
      const InFlight f = inflight[k];
      if (live[f.row] != 0u) {
        ++k;
        continue;
      }
      double esc = 0.0;
      s = celer_read_tallies(ctx, reqs[f.req].event, tally.data(), n_bins, &esc);
      if (s != CELER_OK) return s;
      double sum = 0.0;
      for (double v : tally) sum += v;
      celer_request_result& r = results[f.req];
      r.done_s = seconds_since(t0);
      r.edep = sum;
      r.escaped = esc;
      if (opt.tallies_out) std::memcpy(opt.tallies_out + f.req * n_bins, tally.data(), sizeof(double) * n_bins);
      last_done = r.done_s;
      row_busy[f.row] = 0;
      reserved -= f.reserved;
      ++completed;
      inflight[k] = inflight.back();
      inflight.pop_back();
    }
    // nothing left to step but events still counted live: inconsistent state
    if (done == 0 && !inflight.empty()) return CELER_ERR_STATE;
  }
  if (summary) {
    s = celer_get_stats(ctx, &st);
    if (s != CELER_OK) return s;
    summary->wall_s = last_done;
    summary->track_steps = st.steps_total - steps0;
    summary->admitted = admitted;
    summary->completed = completed;
    summary->chunks = chunks;
  }
  return CELER_OK;
}

extern "C" celer_status celer_autotune(const celer_problem* base, const celer_primary* prims, const uint32_t* events,
                                       uint64_t n, const uint64_t* slot_counts, int n_slot_counts,
                                       const int* block_sizes, int n_block_sizes, const int* policies,
                                       int n_policies, const int* modes, int n_modes, celer_tune_trial* trials,
                                       int max_trials, int* n_trials, celer_tune_trial* best) {
  if (!base || !prims || !events || !slot_counts || !block_sizes || !policies || !modes || !best)
    return CELER_ERR_INVALID;
  if (n == 0 || n_slot_counts < 1 || n_block_sizes < 1 || n_policies < 1 || n_modes < 1) return CELER_ERR_INVALID;
  // group primaries by event, in order of first appearance
  std::vector<uint32_t> order;
  std::vector<std::vector<celer_primary>> groups;
  for (uint64_t i = 0; i < n; ++i) {
    auto it = std::find(order.begin(), order.end(), events[i]);
    size_t g = (size_t)(it - order.begin());
    if (it == order.end()) {
      order.push_back(events[i]);
      groups.emplace_back();
    }
    groups[g].push_back(prims[i]);
  }
  cudaStream_t stream = static_cast<cudaStream_t>(base->cuda_stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return CELER_ERR_CUDA;
  int count = 0;
  *best = celer_tune_trial{};
  for (int a = 0; a < n_slot_counts; ++a)
    for (int b = 0; b < n_block_sizes; ++b)
      for (int c = 0; c < n_policies; ++c)
        for (int d = 0; d < n_modes; ++d)
          for (int warps = 1; warps >= 0; --warps) {
            // the asynchronous loop's two schedules for the block-local policy
            if (warps == 0 && !(modes[d] == CELER_LOOP_ASYNC && policies[c] == CELER_SORT_LOCAL)) continue;
            celer_problem pb = *base;
            pb.n_slots = slot_counts[a];
            pb.block_size = block_sizes[b];
            pb.sort_policy = policies[c];
            if (pb.max_events < order.size()) pb.max_events = (uint32_t)order.size();
            celer_tune_trial t{pb.n_slots, pb.block_size, pb.sort_policy, modes[d], 0.0, 0.0, warps};
            // the asynchronous loop runs the block-pass policies only: other
            // pairs are recorded with no throughput
            const bool runnable = modes[d] != CELER_LOOP_ASYNC ||
                                  ((pb.sort_policy == CELER_SORT_LOCAL || pb.sort_policy == CELER_SORT_DATA) &&
                                   !pb.split_actions);
            celer_ctx* ctx = nullptr;
            if (runnable && celer_create(&pb, &ctx) == CELER_OK) {
              bool ok = celer_set_async_warps(ctx, warps) == CELER_OK;
              uint64_t steps = 0;
              for (int rep = 0; rep < 2 && ok; ++rep) {
                for (size_t g = 0; g < order.size() && ok; ++g) {
                  ok = celer_reset_event(ctx, order[g]) == CELER_OK &&
                       celer_add_primaries(ctx, order[g], groups[g].data(), groups[g].size()) == CELER_OK;
                }
                celer_step_stats s0{}, s1{};
                ok = ok && celer_get_stats(ctx, &s0) == CELER_OK;
                cudaEventRecord(e0, stream);
                ok = ok && celer_run_events(ctx, modes[d]) == CELER_OK;
                cudaEventRecord(e1, stream);
                ok = ok && cudaEventSynchronize(e1) == cudaSuccess && celer_get_stats(ctx, &s1) == CELER_OK;
                if (ok && rep == 1) {
                  float ms = 0.f;
                  cudaEventElapsedTime(&ms, e0, e1);
                  steps = s1.steps_total - s0.steps_total;
                  t.ms = ms;
                  t.track_steps_per_s = ms > 0.f ? steps / (ms * 1e-3) : 0.0;
                }
              }
              celer_destroy(ctx);
            }
            if (trials && count < max_trials) trials[count] = t;
            ++count;
            if (t.track_steps_per_s > best->track_steps_per_s) *best = t;
          }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (n_trials) *n_trials = count;
  return best->track_steps_per_s > 0.0 ? CELER_OK : CELER_ERR_STATE;
}
