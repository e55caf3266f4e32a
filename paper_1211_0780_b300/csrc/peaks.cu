// Throughput probes of the units the sweep kernels lean on: the special
// function unit (sin/cos, ex2), the FP32 and FP64 FMA pipes, the 32x32->64
// integer multiply used by Philox, and L2 read bandwidth.  Each probe runs
// independent dependency chains (8 per thread) in every thread of a grid
// filling the GPU, so the pipe, not latency, bounds it; the host times it
// with CUDA events and divides the operation count by the time.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/xy.h"

namespace {

constexpr int kChains = 8;

__global__ void k_probe_sincos(int64_t iters, float* sink) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = 0.001f * (threadIdx.x + j);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      float s, c;
      __sincosf(v[j], &s, &c);
      v[j] = s + c;  // one sin + one cos per chain step
    }
  }
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc += v[j];
  if (acc == 12345.f) sink[0] = acc;
}

__global__ void k_probe_ex2(int64_t iters, float* sink) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = -0.001f * (threadIdx.x + j);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = exp2f(-fabsf(v[j]));
  }
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc += v[j];
  if (acc == 12345.f) sink[0] = acc;
}

__global__ void k_probe_ffma(int64_t iters, float* sink) {
  float v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = 1.0f + 1e-7f * (threadIdx.x + j);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = fmaf(v[j], 0.9999999f, 1e-7f);
  }
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc += v[j];
  if (acc == 12345.f) sink[0] = acc;
}

__global__ void k_probe_dfma(int64_t iters, float* sink) {
  double v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = 1.0 + 1e-9 * (threadIdx.x + j);
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) v[j] = fma(v[j], 0.999999999, 1e-9);
  }
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc += v[j];
  if (acc == 12345.0) sink[0] = static_cast<float>(acc);
}

__global__ void k_probe_imad_wide(int64_t iters, float* sink) {
  uint32_t v[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) v[j] = threadIdx.x * 2654435761u + j;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) {
      const unsigned long long p = static_cast<unsigned long long>(v[j]) * 0xD2511F53ull;
      v[j] = static_cast<uint32_t>(p >> 32) ^ static_cast<uint32_t>(p);
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc ^= v[j];
  if (acc == 12345u) sink[0] = static_cast<float>(acc);
}

// Reads `n4` float4 repeatedly (a buffer that fits in L2), summing them.
__global__ void k_probe_l2(const float4* __restrict__ buf, int64_t n4, int reps, float* sink) {
  float acc = 0.f;
  for (int r = 0; r < reps; ++r)
    for (int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x; i < n4;
         i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
      const float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == 12345.f) sink[0] = acc;
}

}  // namespace

extern "C" {

// kind: 0 = MUFU sin+cos pairs (counted as 2 ops), 1 = MUFU ex2, 2 = FP32
// FMA, 3 = FP64 FMA, 4 = 32x32->64 integer multiply, 5 = L2 read bytes.
// d_scratch: >= 64 MiB of device memory for kind 5 (>= 4 bytes otherwise).
int xy_peak_probe(int kind, void* d_scratch, size_t scratch_bytes, double* ops_per_s, void* stream) {
  if (!ops_per_s || !d_scratch || kind < 0 || kind > 5) return XY_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return XY_ERR_CUDA;
  float* sink = static_cast<float*>(d_scratch);
  const int threads = 256, blocks = sms * 8;
  const int64_t iters = 4096;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return XY_ERR_CUDA;
  double ops = 0.0;
  for (int pass = 0; pass < 2; ++pass) {  // pass 0 warms up
    cudaEventRecord(a, st);
    switch (kind) {
      case 0: k_probe_sincos<<<blocks, threads, 0, st>>>(iters, sink); ops = 2.0; break;
      case 1: k_probe_ex2<<<blocks, threads, 0, st>>>(iters, sink); ops = 1.0; break;
      case 2: k_probe_ffma<<<blocks, threads, 0, st>>>(iters, sink); ops = 1.0; break;
      case 3: k_probe_dfma<<<blocks, threads, 0, st>>>(iters / 8, sink); ops = 1.0 / 8; break;
      case 4: k_probe_imad_wide<<<blocks, threads, 0, st>>>(iters, sink); ops = 1.0; break;
      case 5: {
        if (scratch_bytes < (size_t(64) << 20)) return XY_ERR_NOMEM;
        const int64_t n4 = (int64_t(32) << 20) / 16;  // 32 MiB: resident in L2
        k_probe_l2<<<sms * 4, 512, 0, st>>>(static_cast<const float4*>(d_scratch) + 4, n4, 16, sink);
        ops = 0.0;
        break;
      }
    }
    cudaEventRecord(b, st);
  }
  if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) return XY_ERR_CUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  const double total = (kind == 5) ? double(int64_t(32) << 20) * 16
                                   : double(blocks) * threads * kChains * double(iters) * ops;
  *ops_per_s = total / (ms * 1e-3);
  return XY_OK;
}

}  // extern "C"
