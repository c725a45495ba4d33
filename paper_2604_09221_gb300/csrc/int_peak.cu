// int_peak.cu -- measured integer-issue peak of the GPU (the denominator of
// the engine's roofline: the method is integer work on the ALU pipes, with no
// tensor-core or floating-point component).
//
// Every thread runs kChains independent dependency chains of one integer
// instruction kind, unrolled kUnroll times per loop trip, so the SM's
// schedulers always have independent instructions to issue.  The operations
// are written as inline PTX so that the compiler keeps one instruction per
// operation, and each chain value feeds the next operations of its chain so
// that none can be folded away:
//   kind 0  lop3.b32 (majority of three evolving words)
//   kind 1  add.u32  (a Fibonacci-like chain: each value is the sum of the
//                     two before it)
//   kind 2  mad.lo.u32 (a*b + c of evolving words)
//   kind 3  lop3.b32 and mad.lo.u32 alternating (two issue pipes)
// The grid fills every SM with 64 resident warps.  The rate is
// (threads x trips x kChains x kUnroll x 3) lane operations / kernel time.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

namespace {

constexpr int kChains = 4;
constexpr int kUnroll = 16;
constexpr int kThreads = 512;

__device__ __forceinline__ uint32_t op_lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t op_add(uint32_t a, uint32_t b, uint32_t) {
  uint32_t r;
  asm volatile("add.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t op_mad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm volatile("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}

template <int KIND>
__device__ __forceinline__ uint32_t op(int step, uint32_t a, uint32_t b, uint32_t c) {
  if constexpr (KIND == 0) return op_lop3(a, b, c);
  else if constexpr (KIND == 1) return op_add(a, b, c);
  else if constexpr (KIND == 2) return op_mad(a, b, c);
  else return (step & 1) ? op_mad(a, b, c) : op_lop3(a, b, c);
}

template <int KIND>
__global__ void __launch_bounds__(kThreads) int_peak_kernel(uint64_t trips, uint32_t seed,
                                                            uint32_t *sink) {
  uint32_t x[kChains], y[kChains], z[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    x[k] = seed ^ (threadIdx.x * 0x9E3779B9u + k);
    y[k] = seed + blockIdx.x * 0x85EBCA6Bu + 3u * k;
    z[k] = (seed >> 3) ^ (threadIdx.x + 7u * k);
  }
  for (uint64_t t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        x[k] = op<KIND>(u, x[k], y[k], z[k]);
        y[k] = op<KIND>(u + 1, y[k], z[k], x[k]);
        z[k] = op<KIND>(u, z[k], x[k], y[k]);
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) acc ^= x[k] ^ y[k] ^ z[k];
  if (acc == seed) sink[0] = acc;  // keeps the chains live; practically never taken
}

template <int KIND>
cudaError_t run(uint64_t trips, unsigned grid, uint32_t *sink, cudaStream_t st, float *ms) {
  cudaEvent_t a, b;
  cudaError_t e = cudaEventCreate(&a);
  if (e != cudaSuccess) return e;
  e = cudaEventCreate(&b);
  if (e != cudaSuccess) {
    cudaEventDestroy(a);
    return e;
  }
  int_peak_kernel<KIND><<<grid, kThreads, 0, st>>>(trips / 16 + 1, 1u, sink);  // warm-up
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaEventRecord(a, st);
  if (e == cudaSuccess) {
    int_peak_kernel<KIND><<<grid, kThreads, 0, st>>>(trips, 12345u, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(b, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(b);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

}  // namespace

extern "C" ts_status ts_int_issue_peak(int kind, uint64_t trips, double *lane_ops_per_s,
                                       double *ms_out, void *stream) {
  if (kind < 0 || kind > 3 || trips == 0 || trips > (1ull << 24) || !lane_ops_per_s)
    return TS_EINVAL;
  int dev = 0, sms = 0, per_sm_threads = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&per_sm_threads, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (e != cudaSuccess) return TS_ECUDA;
  const unsigned grid = (unsigned)sms * (unsigned)(per_sm_threads / kThreads > 0 ? per_sm_threads / kThreads : 1);
  uint32_t *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) return TS_ENOMEM;
  cudaStream_t st = (cudaStream_t)stream;
  float ms = 0.f;
  switch (kind) {
    case 0: e = run<0>(trips, grid, sink, st, &ms); break;
    case 1: e = run<1>(trips, grid, sink, st, &ms); break;
    case 2: e = run<2>(trips, grid, sink, st, &ms); break;
    default: e = run<3>(trips, grid, sink, st, &ms); break;
  }
  cudaFree(sink);
  if (e != cudaSuccess || ms <= 0.f) return TS_ECUDA;
  const double ops = (double)grid * kThreads * (double)trips * kChains * kUnroll * 3.0;
  *lane_ops_per_s = ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return TS_OK;
}
