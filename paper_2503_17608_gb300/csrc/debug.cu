// Diagnostics for the parity tests: the device Philox4x32-10 on given
// (counter, key) records, cuRAND's Philox4_32_10 generator for
// cross-checking the two against each other and against the CPU oracle, and
// the table-driven log/exp next to CUDA's own.
#include <curand_kernel.h>

#include <vector>

#include "celer_gb.h"
#include "physics.cuh"

namespace {

__global__ void k_philox(const uint32_t* in, uint32_t* out, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t* r = in + 6 * i;
    const uint4 o = celer::philox4x32_10(make_uint4(r[0], r[1], r[2], r[3]), make_uint2(r[4], r[5]));
    out[4 * i + 0] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
  }
}

__global__ void k_curand(unsigned long long seed, unsigned long long sub, unsigned long long offset4, uint32_t* out,
                         uint64_t n) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, sub, 4ull * offset4, &st);
  for (uint64_t i = 0; i < n; ++i) {
    const uint4 o = curand4(&st);
    out[4 * i + 0] = o.x;
    out[4 * i + 1] = o.y;
    out[4 * i + 2] = o.z;
    out[4 * i + 3] = o.w;
  }
}

__global__ void k_math(int fn, const double* mt, const double* x, double* out, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const double v = x[i];
    double r;
    switch (fn) {
      case 0: r = celer::fast_log(v, mt); break;
      case 1: r = celer::fast_exp(v, mt); break;
      case 2: r = log(v); break;
      case 3: r = exp(v); break;
      case 4: { double sn, cs; celer::fast_sincos_2pi(v, mt, &sn, &cs); r = sn; break; }
      case 5: { double sn, cs; celer::fast_sincos_2pi(v, mt, &sn, &cs); r = cs; break; }
      case 6: r = sin(2.0 * celer::kPi * v); break;
      case 7: r = cos(2.0 * celer::kPi * v); break;
      case 8: { double sn, cs; celer::fast_sincos(v, mt, &sn, &cs); r = sn; break; }
      case 9: { double sn, cs; celer::fast_sincos(v, mt, &sn, &cs); r = cs; break; }
      case 10: r = sin(v); break;
      default: r = cos(v); break;
    }
    out[i] = r;
  }
}


// One rejection sample per record: which 0 the FP32-filtered Compton sampler
// of the step kernels, 1 its plain FP64 form, 2 the filtered Moller sampler,
// 3 its plain FP64 form.
__global__ void k_sample(int which, uint32_t seed, uint32_t event, const double* mt, const double* E, double cut,
                         const uint64_t* tid, const uint32_t* ctr, double* eps_out, double* cost_out,
                         uint32_t* ctr_out, uint8_t* ok_out, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    celer::TrackRng rng(seed, event, tid[i], ctr[i]);
    bool ok = false;
    double eps = 0.0, cost = 0.0;
    switch (which) {
      case 0: eps = celer::sample_compton(E[i], rng, cost, ok, mt); break;
      case 1: eps = celer::sample_compton_fp64(E[i], rng, cost, ok, mt); break;
      case 2: eps = celer::sample_moller(E[i], cut, rng, ok); break;
      default: eps = celer::sample_moller_fp64(E[i], cut, rng, ok); break;
    }
    eps_out[i] = eps;
    cost_out[i] = cost;
    ctr_out[i] = rng.ctr;
    ok_out[i] = ok ? 1 : 0;
  }
}

// FP64 throughput probe: every thread runs 8 independent fused multiply-add
// chains, so the FP64 pipes never wait on a result. The sum is written only
// if it equals an impossible value, which keeps the work alive.
__global__ void __launch_bounds__(256) k_fp64_rate(uint64_t iters, double seed, double* out) {
  double a[8];
  const double b = 1.0 - 1e-9 * (double)(threadIdx.x & 7), c = 1e-12 * (double)threadIdx.x;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = seed + j;
  for (uint64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  double sum = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) sum += a[j];
  if (sum == -1.0) out[blockIdx.x] = sum;
}

}  // namespace

extern "C" {

celer_status celer_debug_math(int fn, const double* host_x, uint64_t n, double* host_out) {
  if (!host_x || !host_out || fn < 0 || fn > 11) return CELER_ERR_INVALID;
  if (n == 0) return CELER_OK;
  std::vector<double> table(celer::kMathTableSize);
  celer::build_math_table(table.data());
  double *d_mt = nullptr, *d_x = nullptr, *d_out = nullptr;
  celer_status st = CELER_OK;
  if (cudaMalloc(&d_mt, sizeof(double) * table.size()) != cudaSuccess || cudaMalloc(&d_x, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&d_out, sizeof(double) * n) != cudaSuccess)
    st = CELER_ERR_CUDA;
  if (st == CELER_OK &&
      (cudaMemcpy(d_mt, table.data(), sizeof(double) * table.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_x, host_x, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess))
    st = CELER_ERR_CUDA;
  if (st == CELER_OK) {
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_math<<<grid, 256>>>(fn, d_mt, d_x, d_out, n);
    if (cudaGetLastError() != cudaSuccess) st = CELER_ERR_CUDA;
  }
  if (st == CELER_OK && cudaMemcpy(host_out, d_out, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = CELER_ERR_CUDA;
  cudaFree(d_mt);
  cudaFree(d_x);
  cudaFree(d_out);
  return st;
}

celer_status celer_debug_philox(const uint32_t* host_ctr_key, uint32_t* host_out, uint64_t n) {
  if (!host_ctr_key || !host_out) return CELER_ERR_INVALID;
  if (n == 0) return CELER_OK;
  uint32_t *d_in = nullptr, *d_out = nullptr;
  if (cudaMalloc(&d_in, sizeof(uint32_t) * 6 * n) != cudaSuccess) return CELER_ERR_CUDA;
  if (cudaMalloc(&d_out, sizeof(uint32_t) * 4 * n) != cudaSuccess) {
    cudaFree(d_in);
    return CELER_ERR_CUDA;
  }
  celer_status st = CELER_OK;
  if (cudaMemcpy(d_in, host_ctr_key, sizeof(uint32_t) * 6 * n, cudaMemcpyHostToDevice) != cudaSuccess) st = CELER_ERR_CUDA;
  if (st == CELER_OK) {
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_philox<<<grid, 256>>>(d_in, d_out, n);
    if (cudaGetLastError() != cudaSuccess) st = CELER_ERR_CUDA;
  }
  if (st == CELER_OK && cudaMemcpy(host_out, d_out, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = CELER_ERR_CUDA;
  cudaFree(d_in);
  cudaFree(d_out);
  return st;
}

celer_status celer_debug_curand_philox(uint64_t seed, uint64_t subsequence, uint64_t offset4, uint32_t* host_out,
                                       uint64_t n) {
  if (!host_out) return CELER_ERR_INVALID;
  if (n == 0) return CELER_OK;
  uint32_t* d_out = nullptr;
  if (cudaMalloc(&d_out, sizeof(uint32_t) * 4 * n) != cudaSuccess) return CELER_ERR_CUDA;
  k_curand<<<1, 1>>>(seed, subsequence, offset4, d_out, n);
  celer_status st = cudaGetLastError() == cudaSuccess ? CELER_OK : CELER_ERR_CUDA;
  if (st == CELER_OK && cudaMemcpy(host_out, d_out, sizeof(uint32_t) * 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    st = CELER_ERR_CUDA;
  cudaFree(d_out);
  return st;
}

celer_status celer_debug_sample(int which, uint32_t seed, uint32_t event, const double* host_E, double cut,
                                const uint64_t* host_tid, const uint32_t* host_ctr, uint64_t n, double* eps_out,
                                double* cost_out, uint32_t* ctr_out, uint8_t* ok_out) {
  if (which < 0 || which > 3 || !host_E || !host_tid || !host_ctr || !eps_out || !cost_out || !ctr_out || !ok_out)
    return CELER_ERR_INVALID;
  if (n == 0) return CELER_OK;
  std::vector<double> table(celer::kMathTableSize);
  celer::build_math_table(table.data());
  double *d_mt = nullptr, *d_E = nullptr, *d_eps = nullptr, *d_cost = nullptr;
  uint64_t* d_tid = nullptr;
  uint32_t *d_ctr = nullptr, *d_ctr_out = nullptr;
  uint8_t* d_ok = nullptr;
  celer_status st = CELER_OK;
  if (cudaMalloc(&d_mt, sizeof(double) * table.size()) != cudaSuccess || cudaMalloc(&d_E, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&d_eps, sizeof(double) * n) != cudaSuccess || cudaMalloc(&d_cost, sizeof(double) * n) != cudaSuccess ||
      cudaMalloc(&d_tid, sizeof(uint64_t) * n) != cudaSuccess || cudaMalloc(&d_ctr, sizeof(uint32_t) * n) != cudaSuccess ||
      cudaMalloc(&d_ctr_out, sizeof(uint32_t) * n) != cudaSuccess || cudaMalloc(&d_ok, n) != cudaSuccess)
    st = CELER_ERR_CUDA;
  if (st == CELER_OK &&
      (cudaMemcpy(d_mt, table.data(), sizeof(double) * table.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_E, host_E, sizeof(double) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_tid, host_tid, sizeof(uint64_t) * n, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(d_ctr, host_ctr, sizeof(uint32_t) * n, cudaMemcpyHostToDevice) != cudaSuccess))
    st = CELER_ERR_CUDA;
  if (st == CELER_OK) {
    const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_sample<<<grid, 256>>>(which, seed, event, d_mt, d_E, cut, d_tid, d_ctr, d_eps, d_cost, d_ctr_out, d_ok, n);
    if (cudaGetLastError() != cudaSuccess) st = CELER_ERR_CUDA;
  }
  if (st == CELER_OK && (cudaMemcpy(eps_out, d_eps, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
                         cudaMemcpy(cost_out, d_cost, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
                         cudaMemcpy(ctr_out, d_ctr_out, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
                         cudaMemcpy(ok_out, d_ok, n, cudaMemcpyDeviceToHost) != cudaSuccess))
    st = CELER_ERR_CUDA;
  cudaFree(d_mt);
  cudaFree(d_E);
  cudaFree(d_eps);
  cudaFree(d_cost);
  cudaFree(d_tid);
  cudaFree(d_ctr);
  cudaFree(d_ctr_out);
  cudaFree(d_ok);
  return st;
}

celer_status celer_debug_fp64_rate(int blocks_per_sm, uint64_t iters, double* tflops_out, double* ms_out) {
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters == 0 || iters > (1ull << 32) || !tflops_out)
    return CELER_ERR_INVALID;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CELER_ERR_CUDA;
  const int grid = sms * blocks_per_sm;
  double* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  celer_status st = CELER_OK;
  if (cudaMalloc(&d_out, sizeof(double) * grid) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    st = CELER_ERR_CUDA;
  float ms = 0.0f;
  if (st == CELER_OK) {
    k_fp64_rate<<<grid, 256>>>(iters / 8 + 1, 1.0, d_out);  // warm-up
    cudaEventRecord(e0);
    k_fp64_rate<<<grid, 256>>>(iters, 1.0, d_out);
    cudaEventRecord(e1);
    if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess || ms <= 0.0f)
      st = CELER_ERR_CUDA;
  }
  if (st == CELER_OK) {
    const double flop = 2.0 * 8.0 * (double)iters * (double)grid * 256.0;
    *tflops_out = flop / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(d_out);
  return st;
}

}  // extern "C"
