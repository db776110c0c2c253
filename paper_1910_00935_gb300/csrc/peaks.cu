// peaks.cu -- mpm_measure_peak: arithmetic peaks of this GPU measured with the library's
// own kernel, the denominators of the ALU rooflines (FP64 and FP32 fused multiply-adds: the
// ratio of the two is why the polar factor's refinement runs in compensated FP32).
//
// The kernel runs 8 independent fused multiply-add chains per thread (enough to hide the
// pipe's latency), on 8 CTAs of 256 threads per SM, for a fixed number of iterations; a
// multiply-add counts as 2 FLOP.  The first launch warms up, the next ones are timed with
// CUDA events on the caller's stream and the best is returned.
#include <cuda_runtime.h>

#include "../../include/mpm.h"
#include "mpm_internal.h"

namespace {

__device__ double g_peak_sink;  // written only when the chains reach an impossible value

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chains_kernel(int iters, T seed) {
  T a[kChains];
  const T b = seed * (T)0.999999, c = seed * (T)1e-7;
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = seed + (T)(threadIdx.x + k);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = a[k] * b + c;  // contracted to one FMA
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == (T)-1.2345e-30) g_peak_sink = (double)s;
}

// float4 reduction throughput: every thread issues `iters` reductions (results unused, so
// they compile to RED) into an L2-resident array of nodes; SPREAD puts the 32 lanes of an
// instruction on 32 different 128-byte lines (the scattered case), else on 32 consecutive
// nodes (4 lines: the best case)
constexpr unsigned kRedNodes = 1u << 18;  // 4 MiB of float4 nodes
__device__ float4 g_red_nodes[kRedNodes];

template <bool SPREAD>
__global__ void __launch_bounds__(kThreads) red_kernel(int iters) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int it = 0; it < iters; ++it) {
    const unsigned base = (warp * 1237u + (unsigned)it * 613u) * 32u;
    const unsigned node = (SPREAD ? base + lane * 8u : base + lane) & (kRedNodes - 1u);
    atomicAdd(&g_red_nodes[node], make_float4(1.0f, 1.0f, 1.0f, 1.0f));
  }
}

template <typename T>
int measure(double* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mpm::set_static_error("mpm_measure_peak: no CUDA device");
    return MPM_ERR_CUDA;
  }
  const int blocks = sms * 8;
  const int iters = sizeof(T) == 8 ? 256 : 4096;  // ~10-30 ms a launch
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    mpm::set_static_error("mpm_measure_peak: cudaEventCreate failed");
    return MPM_ERR_CUDA;
  }
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    fma_chains_kernel<T><<<blocks, kThreads, 0, st>>>(iters, (T)1.0000001);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * kChains * 16.0 * iters * (double)blocks * kThreads;
    if (e == cudaSuccess && rep > 0 && ms > 0.0f && flops / (ms * 1e-3) > best)
      best = flops / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mpm::set_static_error(cudaGetErrorString(e));
    return MPM_ERR_CUDA;
  }
  *out = best;
  return MPM_OK;
}

}  // namespace

template <bool SPREAD>
int measure_red(double* out, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mpm::set_static_error("mpm_measure_peak: no CUDA device");
    return MPM_ERR_CUDA;
  }
  const int blocks = sms * 8, iters = 256;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    mpm::set_static_error("mpm_measure_peak: cudaEventCreate failed");
    return MPM_ERR_CUDA;
  }
  double best = 0.0;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    cudaEventRecord(e0, st);
    red_kernel<SPREAD><<<blocks, kThreads, 0, st>>>(iters);
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    const double updates = (double)iters * blocks * kThreads;
    if (e == cudaSuccess && rep > 0 && ms > 0.0f && updates / (ms * 1e-3) > best)
      best = updates / (ms * 1e-3);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    mpm::set_static_error(cudaGetErrorString(e));
    return MPM_ERR_CUDA;
  }
  *out = best;
  return MPM_OK;
}

extern "C" int mpm_measure_peak(int32_t kind, double* flops_per_s, void* stream) {
  if (!flops_per_s || kind < MPM_PEAK_FP64_FMA || kind > MPM_PEAK_RED_F32X4_SPREAD) {
    mpm::set_static_error("mpm_measure_peak: bad kind or NULL output");
    return MPM_ERR_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  switch (kind) {
    case MPM_PEAK_FP64_FMA: return measure<double>(flops_per_s, s);
    case MPM_PEAK_FP32_FMA: return measure<float>(flops_per_s, s);
    case MPM_PEAK_RED_F32X4: return measure_red<false>(flops_per_s, s);
    default: return measure_red<true>(flops_per_s, s);
  }
}
