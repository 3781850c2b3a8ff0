// Stable partition of slot indices by key without any device allocation.
//
// The step loop partitions track slots by next action with per-tile key
// counts kept in memory the context allocates. This file offers the same
// partition as a stand-alone call whose only working memory is a fixed
// file-scope device array, for callers that must not allocate device memory
// themselves: code that runs while another framework's caching allocator
// owns the device memory, or latency-critical host loops that cannot afford
// cudaMalloc/cudaFree (cudaFree synchronises the whole device).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "celer_gb.h"

namespace {

constexpr int kNaTile = 256;                  // slots per tile, one thread per slot
constexpr uint32_t kNaMaxSlots = 1u << 20;    // largest n accepted
constexpr int kNaMaxKeys = 16;                // largest n_keys accepted
constexpr uint32_t kNaMaxTiles = kNaMaxSlots / kNaTile;
constexpr int kNaMaxDevices = 64;

// Per-(key, tile) counts, then their exclusive scan, key major:
// 16 x 4096 x 4 bytes = 256 KiB, held by every device that loads the library.
__device__ __align__(256) uint32_t g_partition_scratch[kNaMaxKeys * kNaMaxTiles + kNaMaxKeys + 1];

// Device address of g_partition_scratch per device ordinal, looked up once
// per process. cudaDeviceReset destroys the context this address belongs to,
// so the entry point must not be called on a device after it was reset.
uint32_t* g_scratch_ptr[kNaMaxDevices] = {};
std::mutex g_scratch_mutex;

cudaError_t scratch_for_current_device(uint32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNaMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_partition_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<uint32_t*>(ptr);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// Pass 1: keys per tile (every (key, tile) entry is written, so the scratch
// needs no clearing between calls).
__global__ void __launch_bounds__(kNaTile) k_na_count(const uint8_t* keys, uint32_t n, int n_keys, uint32_t n_tiles,
                                                     uint32_t* counts) {
  __shared__ unsigned s_cnt[kNaMaxKeys];
  const uint32_t tile = blockIdx.x;
  if (threadIdx.x < kNaMaxKeys) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t slot = tile * kNaTile + threadIdx.x;
  if (slot < n) {
    const unsigned key = keys[slot];
    if ((int)key < n_keys) atomicAdd(&s_cnt[key], 1u);
  }
  __syncthreads();
  if ((int)threadIdx.x < n_keys) counts[threadIdx.x * n_tiles + tile] = s_cnt[threadIdx.x];
}

// Pass 2 (one block): exclusive scan of the counts in key-major order, so
// that entry (k, t) becomes the output position of tile t's first key-k slot;
// offsets[k] = first position of key k, offsets[n_keys] = the number of slots
// whose key is below n_keys (n when every key is in range).
__global__ void __launch_bounds__(1024) k_na_scan(uint32_t* counts, int n_keys, uint32_t n_tiles, uint32_t* offsets) {
  __shared__ unsigned s_warp[32];
  __shared__ unsigned s_total;
  const uint32_t total = (uint32_t)n_keys * n_tiles;
  const uint32_t per = (total + blockDim.x - 1) / blockDim.x;
  const uint32_t beg = min(threadIdx.x * per, total);
  const uint32_t end = min(beg + per, total);
  unsigned local = 0;
  for (uint32_t i = beg; i < end; ++i) local += counts[i];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : 0u;
    unsigned wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    s_warp[lane] = wi - w;
    if (lane == 31) s_total = wi;
  }
  __syncthreads();
  unsigned run = s_warp[warp] + incl - local;
  for (uint32_t i = beg; i < end; ++i) {
    const unsigned v = counts[i];
    counts[i] = run;
    run += v;
  }
  __syncthreads();
  if ((int)threadIdx.x < n_keys) offsets[threadIdx.x] = counts[threadIdx.x * n_tiles];
  if ((int)threadIdx.x == n_keys) offsets[n_keys] = s_total;
}

// Pass 3: stable scatter; slots whose key is skip_key (or not below n_keys)
// are left out of perm.
__global__ void __launch_bounds__(kNaTile) k_na_scatter(const uint8_t* keys, uint32_t n, int n_keys, uint32_t n_tiles,
                                                       const uint32_t* positions, int skip_key, uint32_t* perm) {
  __shared__ unsigned s_cnt[kNaTile / 32][kNaMaxKeys];
  const uint32_t tile = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < (kNaTile / 32) * kNaMaxKeys) (&s_cnt[0][0])[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t slot = tile * kNaTile + threadIdx.x;
  unsigned key = slot < n ? keys[slot] : 0xFFFFFFFFu;
  if (key >= (unsigned)n_keys) key = 0xFFFFFFFFu;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  const unsigned rank = __popc(peers & ((1u << lane) - 1u));
  if (key != 0xFFFFFFFFu && lane == __ffs(peers) - 1) s_cnt[warp][key] = __popc(peers);
  __syncthreads();
  if (key != 0xFFFFFFFFu && (int)key != skip_key) {
    unsigned pos = positions[key * n_tiles + tile] + rank;
    for (int w = 0; w < warp; ++w) pos += s_cnt[w][key];
    perm[pos] = slot;
  }
}

}  // namespace

extern "C" celer_status celer_partition_keys_noalloc(const uint8_t* d_keys, uint64_t n, int n_keys, int skip_key,
                                                     uint32_t* d_perm, uint32_t* d_offsets, void* cuda_stream) {
  if (!d_offsets || (n > 0 && (!d_keys || !d_perm))) return CELER_ERR_INVALID;
  if (n > kNaMaxSlots || n_keys < 1 || n_keys > kNaMaxKeys || skip_key >= n_keys) return CELER_ERR_INVALID;
  // An error left pending by earlier work on this thread is not ours to
  // report or clear: launch nothing and leave it in place.
  if (cudaPeekAtLastError() != cudaSuccess) return CELER_ERR_CUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (n == 0) {  // every offset is 0; d_perm is not touched
    return cudaMemsetAsync(d_offsets, 0, sizeof(uint32_t) * (size_t)(n_keys + 1), s) == cudaSuccess ? CELER_OK
                                                                                              : CELER_ERR_CUDA;
  }
  uint32_t* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != cudaSuccess) return CELER_ERR_CUDA;
  const uint32_t n_tiles = (uint32_t)((n + kNaTile - 1) / kNaTile);
  k_na_count<<<n_tiles, kNaTile, 0, s>>>(d_keys, (uint32_t)n, n_keys, n_tiles, scratch);
  k_na_scan<<<1, 1024, 0, s>>>(scratch, n_keys, n_tiles, d_offsets);
  k_na_scatter<<<n_tiles, kNaTile, 0, s>>>(d_keys, (uint32_t)n, n_keys, n_tiles, scratch, skip_key, d_perm);
  // nothing was pending before the launches, so an error now is theirs
  return cudaGetLastError() == cudaSuccess ? CELER_OK : CELER_ERR_CUDA;
}
