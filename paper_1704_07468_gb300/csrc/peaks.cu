// Measured ceiling of the sparse accumulation's unit of work.
//
// The on-chip accumulation (countAndUpdate of Alg. 1 for sparse levels)
// spends one 32-bit shared-memory atomic add per pair update.  Its roofline
// is therefore the rate at which the SMs retire shared-memory atomic adds
// when nothing else limits them: every lane of a warp on its own bank (no
// conflicts), many warps per SM, no global traffic.  This probe measures
// that rate on the current device.
#include <cuda_runtime.h>

#include <cstdint>

#include "gakco.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kProbeWords = 8;  // distinct words per thread

// Random columns: each lane adds at pseudo-random words of a 4096-word row
// (a xorshift sequence per lane), the pattern of the accumulation's column
// updates; lanes of a warp then meet in banks as random draws do.
__global__ void __launch_bounds__(kProbeThreads)
k_smem_atomic_probe_random(uint32_t iters, uint32_t* __restrict__ out) {
  constexpr uint32_t kRow = 4096;
  extern __shared__ uint32_t sh[];
  for (uint32_t i = threadIdx.x; i < kRow; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  uint32_t x = 0x9E3779B9u * (blockIdx.x * blockDim.x + threadIdx.x + 1);
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeWords; ++j) {
      x ^= x << 13;
      x ^= x >> 17;
      x ^= x << 5;
      atomicAdd(&sh[x & (kRow - 1)], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t s = 0;
    for (uint32_t t = 0; t < kRow; ++t) s += sh[t];
    out[blockIdx.x * kProbeWords] = s;
  }
}

__global__ void __launch_bounds__(kProbeThreads)
k_smem_atomic_probe(uint32_t iters, uint32_t* __restrict__ out) {
  extern __shared__ uint32_t sh[];
  for (int j = 0; j < kProbeWords; ++j) sh[j * kProbeThreads + threadIdx.x] = 0;
  __syncthreads();
  // Word j * blockDim + tid: the 32 lanes of a warp touch 32 consecutive
  // words, one per bank.
  uint32_t* mine = sh + threadIdx.x;
  const uint32_t inc = 1u + (blockIdx.x & 1u);
  for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kProbeWords; ++j) atomicAdd(mine + j * kProbeThreads, inc);
  }
  __syncthreads();
  if (threadIdx.x < kProbeWords) {
    uint32_t s = 0;
    for (int t = 0; t < kProbeThreads; ++t) s += sh[threadIdx.x * kProbeThreads + t];
    out[blockIdx.x * kProbeWords + threadIdx.x] = s;
  }
}

}  // namespace

extern "C" int gakco_measure_smem_atomics_pattern(void* stream, int random_columns, double* updates_per_s) {
  if (!updates_per_s) return GAKCO_E_INVALID;
  *updates_per_s = 0;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) {
    cudaGetLastError();
    return GAKCO_E_CUDA;
  }
  const size_t smem = (size_t)kProbeWords * kProbeThreads * 4;
  const int blocks = 2 * nsm;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* out = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * kProbeWords * 4);
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  float ms = 0;
  const uint32_t iters = 20000;
  auto launch = [&](uint32_t n) {
    if (random_columns)
      k_smem_atomic_probe_random<<<blocks, kProbeThreads, 4096 * 4, st>>>(n, out);
    else
      k_smem_atomic_probe<<<blocks, kProbeThreads, smem, st>>>(n, out);
  };
  if (e == cudaSuccess) {
    launch(iters / 10);  // warm-up
    e = cudaEventRecord(a, st);
  }
  if (e == cudaSuccess) {
    launch(iters);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (out) cudaFree(out);
  if (e != cudaSuccess || ms <= 0) {
    cudaGetLastError();
    return GAKCO_E_CUDA;
  }
  *updates_per_s = (double)blocks * kProbeThreads * kProbeWords * iters / (ms * 1e-3);
  return GAKCO_OK;
}

extern "C" int gakco_measure_smem_atomics(void* stream, double* updates_per_s) {
  return gakco_measure_smem_atomics_pattern(stream, 0, updates_per_s);
}
