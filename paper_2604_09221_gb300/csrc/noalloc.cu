// noalloc.cu -- ts_enumerate_noalloc: an exhaustive sweep that allocates
// nothing.
//
// The regular sweep (ts_enumerate) keeps its hash table, work counter and
// error words in a ts_hist created with cudaMalloc.  Some callers cannot
// allocate device memory when they run a sweep: services that reserve all
// device memory at start-up and forbid later allocations, and hosts whose
// allocator must not be entered from the calling thread (a real-time loop
// where an allocation could block, or a thread that holds the allocator's
// lock).  For them this entry point runs the same table-driven sweep kernel
// with all of its scratch in one statically allocated device array that
// every GPU loading this library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "engine.h"

namespace {

// Scratch layout (all inside tc_noalloc_scratch):
//   keys[kSlots] u64 | counts[kSlots] u64 | err u32 (+pad) | failed u64 | work u64
constexpr uint64_t kSlots = 4096;                    // hash slots (power of two)
constexpr uint64_t kMaxCodes = kSlots / 2;           // distinct codes kept (load <= 1/2)
constexpr size_t kScratchBytes = kSlots * 16 + 64;   // 65 600 bytes

static __device__ __align__(256) unsigned char tc_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
// Device address of the array per device, looked up once (under g_setup_mu)
// and then read without a lock.
std::atomic<unsigned char *> g_scratch[kMaxDevices];  // static storage: zero-initialised
std::mutex g_setup_mu;

// The array's address on the current device `dev`: cudaGetSymbolAddress on
// the first call for the device, the cached value after that.  Returns null
// if the lookup fails (the next call tries again).
unsigned char *scratch_address(int dev) {
  unsigned char *p = g_scratch[dev].load(std::memory_order_acquire);
  if (p) return p;
  std::lock_guard<std::mutex> g(g_setup_mu);
  p = g_scratch[dev].load(std::memory_order_relaxed);
  if (p) return p;
  void *q = nullptr;
  if (cudaGetSymbolAddress(&q, tc_noalloc_scratch) != cudaSuccess || !q) return nullptr;
  p = static_cast<unsigned char *>(q);
  g_scratch[dev].store(p, std::memory_order_release);
  return p;
}

// Copy the non-empty slots of the scratch table into the caller's arrays
// (in slot order) and write n_out[0] = distinct codes, n_out[1] = failed
// instances, n_out[2] = error bits of the sweep.
__global__ void noalloc_compact(const uint64_t *keys, const unsigned long long *counts,
                                const uint32_t *err, const unsigned long long *failed,
                                uint64_t *codes, uint64_t *out_counts, uint64_t cap,
                                uint64_t *n_out) {
  __shared__ unsigned long long n;
  if (threadIdx.x == 0) n = 0;
  __syncthreads();
  for (uint64_t s = threadIdx.x; s < kSlots; s += blockDim.x) {
    const uint64_t k = keys[s];
    if (k == 0) continue;
    const unsigned long long i = atomicAdd(&n, 1ull);
    if (i < cap) {
      codes[i] = k;
      out_counts[i] = counts[s];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    n_out[0] = n;
    n_out[1] = *failed;
    n_out[2] = *err | (n > cap ? tcurve::kErrOverflow : 0u);
  }
}

}  // namespace

extern "C" ts_status ts_enumerate_noalloc(const ts_tri *t, uint64_t lo, uint64_t hi,
                                          uint32_t flags, uint64_t *codes, uint64_t *counts,
                                          uint64_t cap, uint64_t *n_out, void *stream) {
  if (!t || !n_out || (cap && (!codes || !counts)) || hi < lo ||
      (flags & ~(TS_ENUM_FLIP | TS_ENUM_REDUCED)) || flags == (TS_ENUM_FLIP | TS_ENUM_REDUCED))
    return TS_EINVAL;
  if (t->cw != 1 || t->np > 64) return TS_EUNSUPPORTED;
  if (cap > kMaxCodes) return TS_EINVAL;  // the scratch table holds at most kMaxCodes codes
  int free_bits = t->np - ((flags & TS_ENUM_FLIP) ? 1 : 0) - ((flags & TS_ENUM_REDUCED) ? 3 : 0);
  if (free_bits < 64 && hi > (1ull << free_bits)) return TS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TS_ECUDA;
  if (dev != t->device) return TS_EINVAL;
  // once per device: the device address of the static array
  unsigned char *base = scratch_address(dev);
  if (!base) return TS_ECUDA;
  ts_hist view;  // a histogram whose storage is the static array (owns nothing)
  view.cw = 1;
  view.slots = kSlots;
  view.d_keys = reinterpret_cast<uint64_t *>(base);
  view.d_counts = reinterpret_cast<unsigned long long *>(base + kSlots * 8);
  view.d_err = reinterpret_cast<uint32_t *>(base + kSlots * 16);
  view.d_failed = reinterpret_cast<unsigned long long *>(base + kSlots * 16 + 16);
  view.d_work = reinterpret_cast<unsigned long long *>(base + kSlots * 16 + 32);
  view.device = dev;
  cudaStream_t st = (cudaStream_t)stream;
  // the array keeps the previous call's contents: start from zero
  if (cudaMemsetAsync(base, 0, kScratchBytes, st) != cudaSuccess) return TS_ECUDA;
  if (lo < hi && tcurve::launch_enumerate(t, lo, hi, flags, &view, st, false) != cudaSuccess)
    return TS_ECUDA;
  noalloc_compact<<<1, 256, 0, st>>>(view.d_keys, view.d_counts, view.d_err, view.d_failed, codes,
                                     counts, cap, n_out);
  return cudaGetLastError() == cudaSuccess ? TS_OK : TS_ECUDA;
}
