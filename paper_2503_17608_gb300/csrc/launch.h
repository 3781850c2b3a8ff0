// Host-side launchers of the step-iteration kernels (defined in step.cu).
#pragma once

#include "common.cuh"

namespace celer {

// A primary staged for the initializer buffer (host validated, layer resolved).
struct StagedPrimary {
  double E, x, y, z, ux, uy, uz;
  unsigned long long tid;
  uint32_t event, primary;
  int32_t layer, ptype;
};

struct LaunchShape {
  int tile_grid;       // persistent grid of the tile kernels (fill, step limit, scatter)
  int step_grid;       // persistent grid of the phase-merged step kernel
  int along_grid;      // persistent grid of the per-kind along-step kernels
  int post_grid;       // persistent grid of the per-process interaction kernels
  int loop_grid;       // co-resident grid of the persistent loop kernel
  int block;           // threads per block of the step / along-step / interaction kernels
  size_t static_smem;  // tables + layer planes + layer materials in shared memory
};

cudaError_t configure_kernels(const Params& p, int block, LaunchShape* shape);

// phase-merged launches
void launch_fill_step(const Params& p, const LaunchShape& sh, cudaStream_t s);
void launch_scatter(const Params& p, const LaunchShape& sh, cudaStream_t s);
void launch_step(const Params& p, const LaunchShape& sh, unsigned long long handle, int use_handle, cudaStream_t s);
// block-local policy: one launch per iteration, and the per-block vacancy
// scan a run starts with (both on the loop's grid)
void launch_local(const Params& p, const LaunchShape& sh, unsigned long long handle, int use_handle, cudaStream_t s);
void launch_local_prepare(const Params& p, const LaunchShape& sh, cudaStream_t s);
// per-tile vacancy scan for a slot-order run after block-local iterations
void launch_scan_tiles(const Params& p, cudaStream_t s);
// check of the bounded grid-barrier wait (one block never arrives)
cudaError_t launch_barrier_probe(const Params& p, int blocks, int absent, long long timeout, cudaStream_t s);
// per-action launches
void launch_fill(const Params& p, const LaunchShape& sh, cudaStream_t s);
void launch_pre_step(const Params& p, const LaunchShape& sh, cudaStream_t s);
void launch_along(const Params& p, int charged, const LaunchShape& sh, cudaStream_t s);
void launch_post(const Params& p, int which, const LaunchShape& sh, cudaStream_t s);
void launch_loop_ctl(const Params& p, unsigned long long handle, int use_handle, cudaStream_t s);
// start of a run (iteration budget, last-block tickets)
void launch_begin_run(const Params& p, unsigned long long budget, cudaStream_t s);
// persistent loop
cudaError_t launch_loop(const Params& p, const LaunchShape& sh, cudaStream_t s);
// Asynchronous block loop (block-pass policies): the buffer entries' states,
// then one cooperative launch; p.ring_state must be set.
void launch_async_prepare(const Params& p, cudaStream_t s);
// Check of the asynchronous loop's queue waits (k_queue_wait_probe).
cudaError_t launch_queue_wait_probe(const Params& p, int which, long long timeout, cudaStream_t s);
cudaError_t launch_loop_async(const Params& p, const LaunchShape& sh, cudaStream_t s);
void launch_push_primaries(const Params& p, const StagedPrimary* d_prim, uint32_t n, cudaStream_t s);

// Primary record as laid out by the C ABI (celer_primary).
struct DevicePrimary {
  double E;
  double pos[3];
  double dir[3];
  int32_t ptype, pad;
};
void launch_push_device_primaries(const Params& p, const DevicePrimary* src, uint32_t n, uint32_t event,
                                  unsigned long long tid0, uint32_t prim0, cudaStream_t s);

// Active-lane counters of the instrumented build (-DCELER_LANE_COUNTERS):
// 3 x n_sites values (visits, lanes, cycles) summed over the copies, then
// cleared; cudaErrorNotSupported in the product build.
cudaError_t read_lane_counts(unsigned long long* host_out, int n_sites);

const char* kernel_name(int id);
enum KernelId : int {
  KID_FILL_STEP = 0, KID_SCATTER, KID_STEP, KID_FILL, KID_PRE_STEP, KID_ALONG_NEUTRAL, KID_ALONG_CHARGED,
  KID_POST_COMPTON, KID_POST_PE, KID_POST_PAIR, KID_POST_MOLLER, KID_POST_BREMS, KID_LOOP_CTL, KID_LOOP, KID_LOCAL,
  KID_COUNT
};

}  // namespace celer
