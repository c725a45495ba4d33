// Test infrastructure: host definitions of the CUDA qualifiers and
// intrinsics that a generated specialised source uses, so that the source
// compiles as plain C++ and its sweep functions can be run one lane at a time
// on the CPU (tests/test_generated_host.py).  Atomics are plain read-modify-
// writes (one lane runs at a time); __match_any_sync returns the calling lane
// alone, so every lane inserts its own code.
#pragma once
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#define __device__
#define __global__
#define __host__
#define __forceinline__ inline
#define __noinline__
#define __constant__
#define __shared__
#define __restrict__
#define __align__(n) __attribute__((aligned(n)))
#define __launch_bounds__(...)
struct EmuDim { unsigned x, y, z; };
static EmuDim threadIdx{0, 0, 0}, blockIdx{0, 0, 0}, gridDim{1, 1, 1}, blockDim{128, 1, 1};
static inline int __ffs(unsigned x) { return __builtin_ffs(x); }
static inline int __ffsll(unsigned long long x) { return __builtin_ffsll(x); }
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline unsigned atomicAdd(unsigned *p, unsigned v) { unsigned o = *p; *p += v; return o; }
static inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) { auto o = *p; *p += v; return o; }
static inline unsigned atomicOr(unsigned *p, unsigned v) { unsigned o = *p; *p |= v; return o; }
static inline unsigned long long atomicCAS(unsigned long long *p, unsigned long long c, unsigned long long v) { auto o = *p; if (o == c) *p = v; return o; }
static inline void __threadfence() {}
static inline void __nanosleep(unsigned) {}
static inline void __syncthreads() {}
static inline int __syncthreads_or(int v) { return v; }
static inline unsigned __match_any_sync(unsigned, unsigned long long) { return 1u << (threadIdx.x & 31u); }
static inline unsigned long long __shfl_sync(unsigned, unsigned long long v, int) { return v; }
unsigned tc_smem[1 << 18];
