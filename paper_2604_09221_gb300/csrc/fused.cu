// fused.cu -- one persistent launch for a whole mixed-degree batch.
//
// The fused batch kernel serves the jobs of every degree of a ts_batch in
// one launch: blocks pull work items from one counter over all jobs (sorted
// by degree), stage the job's tables into shared memory with cp.async.bulk
// on an mbarrier (bounded wait) when they move to another triangulation,
// draw the job's splitmix64 sign vectors on the device (or read the
// caller's, ts_batch_set_signs), classify them with Algorithm 1 (Sec. 2)
// and add the codes to the job's device histogram.  The degree of a job
// selects the code path inside the kernel (a switch over degree-templated
// bodies), and each degree has a tile of its own:
//
//   thread per instance  (TS_KERNEL_TABLE)  every thread classifies its own
//        sign vector with the table-driven sweep: the label slots in shared
//        memory, found through the staged fan entries' offsets, the rest
//        of the per-thread scratch in global memory (word-interleaved,
//        L1/L2-resident);
//   warp per instance    (TS_KERNEL_WARP)   the 32 lanes of a warp classify
//        one sign vector together (lock-free union-find in shared memory,
//        tc_warp_sweep.cuh), 32 sign vectors per warp between histogram
//        inserts;
//
// plus the sign vectors per work item.  A kernel is compiled for a range of
// degrees 1..DHI with a register budget that keeps the resident blocks of
// that range's table-driven bodies (tiers below); the batch takes the tier
// of its largest degree, or the widest tier's kernel with warp bodies when
// a degree has a warp tile.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "tc_layout.h"
#include "tc_stage.cuh"
#include "tc_table_sweep.cuh"
#include "tc_warp_sweep.cuh"

namespace tcurve {
namespace {

constexpr u32 kFT = kFusedThreads;  // threads per block: 4 warps

// Register tiers: (largest degree, resident 128-thread blocks per SM its
// register budget is set for).  The budgets are the ones the per-degree
// table-driven kernels get without a bound (40, 48, 64 and 80 registers).
constexpr int kTierD[kFusedTiers] = {6, 9, 11, 16};
constexpr int kTierMinB[kFusedTiers] = {12, 10, 8, 6};

// Largest per-thread scratch (words) of the table-driven bodies up to dhi.
constexpr u32 slab_words_upto(int dhi) {
  u32 m = 0;
  for (int d = 1; d <= dhi; ++d) {
    const u32 w = (u32)tc_layout(d, true, (int)kFT).words;
    m = w > m ? w : m;
  }
  return m;
}
template <int DHI>
struct FusedSlab {
  static constexpr u32 WORDS = slab_words_upto(DHI);
};

// Sign vector idx of job J: the caller's (J.signs, W words each) or word w
// of the splitmix64 stream, splitmix64((base + idx) * W + w); bits >= |A|
// cleared.
template <u32 W, u32 NPOINTS>
__device__ __forceinline__ TcSig<W> job_sig(const FusedJob &__restrict__ J, u64 idx) {
  TcSig<W> sg;
  if (J.signs) {
#pragma unroll
    for (u32 w = 0; w < W; ++w) sg.w[w] = J.signs[idx * W + w];
  } else {
#pragma unroll
    for (u32 w = 0; w < W; ++w) sg.w[w] = tc_splitmix64((J.base + idx) * W + w);
  }
  sg.w[W - 1] &= tc_top_mask(NPOINTS, W);
  return sg;
}

// Thread per instance: chunk sign vectors of job J from index `first`.  The
// label slots of the sweep (one load per fan entry) sit in shared memory
// (ls: this thread's word 0, word i at ls[i * 128]), and the staged fan
// entries carry their slots' byte offsets; the rest of the scratch is in
// global memory.
template <int D>
__device__ __forceinline__ void thread_item(const FusedJob &__restrict__ J, u64 first, const u32 *tab,
                                            u32 *gslab, u32 *ls, u32 *err_word, u32 &err,
                                            unsigned long long &failed) {
  typedef TcTableK<D, (int)kFT, true> K;
  const TcScratch<K> S{gslab + threadIdx.x};
  const u32 lane = threadIdx.x & 31u;
  for (u32 k = 0; k < J.chunk; k += kFT) {
    const u64 idx = first + k + threadIdx.x;
    TcCodeOut<K> key{};
    if (idx < J.n) {
      const TcSig<K::W> sg = job_sig<K::W, K::NPOINTS>(J, idx);
      key = tc_table_classify<K, true>(sg, tab, J.off_fan, J.off_vext, S, err, ls);
      u64 any = 0;
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) {
        any |= key.w[w];
        if (J.codes) J.codes[idx * K::CW + w] = key.w[w];
      }
      failed += any == 0;
    }
    if constexpr (K::CW == 1) {
      const unsigned peers = __match_any_sync(0xffffffffu, key.w[0]);
      if (key.w[0] != 0 && lane == (u32)(__ffs(peers) - 1))
        tc_global_add(J.hkeys, J.hcnt, J.hslots, err_word, key.w[0],
                      (unsigned long long)__popc(peers));
    } else {
      tc_hist_add_wide<K::CW>(key.w, J.hkeys, J.hcnt, J.hslots, err_word);
    }
  }
}

// Warp per instance: warp w of the block takes sign vectors first + g + r,
// g = 32 w, 32 w + 128, ..., r < 32, one at a time; lane r keeps the code of
// the r-th and the warp inserts its 32 codes together.
template <int D>
__device__ __forceinline__ void warp_item(const FusedJob &__restrict__ J, u64 first, const u32 *tab, u32 *ws,
                                          u32 *err_word, u32 &err, unsigned long long &failed) {
  typedef TcWarpK<D> K;
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  for (u32 g = warp * 32u; g < J.chunk; g += kFT) {
    u64 mine[K::CW];
#pragma unroll
    for (u32 w = 0; w < K::CW; ++w) mine[w] = 0;
    for (u32 r = 0; r < 32u; ++r) {
      const u64 idx = first + g + r;
      if (idx >= J.n) break;  // warp-uniform
      const TcSig<K::W> sg = job_sig<K::W, K::NPOINTS>(J, idx);
      u64 code[K::CW];
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
      err |= tc_warp_classify<D>(sg, tab + J.wl.off_v, tab + J.wl.off_e, J.wl.E,
                                 tab + J.wl.off_anti, J.wl.nanti, tab + J.wl.off_bedge,
                                 J.wl.nbedge, ws, code);
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) {
        const u64 c = __shfl_sync(0xffffffffu, code[w], 0);  // lane 0 holds the code
        if (lane == 0 && J.codes) J.codes[idx * K::CW + w] = c;
        mine[w] = lane == r ? c : mine[w];
      }
    }
    u64 any = 0;
#pragma unroll
    for (u32 w = 0; w < K::CW; ++w) any |= mine[w];
    failed += first + g + lane < J.n && any == 0;
    if constexpr (K::CW == 1) {
      const unsigned peers = __match_any_sync(0xffffffffu, mine[0]);
      if (mine[0] != 0 && lane == (u32)(__ffs(peers) - 1))
        tc_global_add(J.hkeys, J.hcnt, J.hslots, err_word, mine[0],
                      (unsigned long long)__popc(peers));
    } else {
      tc_hist_add_wide<K::CW>(mine, J.hkeys, J.hcnt, J.hslots, err_word);
    }
  }
}

// Work item of a degree-D job (D <= DHI): the job's tile decides the body.
// Only the WARP kernel has warp bodies (from d = 7; below, the table-driven
// body keeps its whole scratch in a few lines per thread and the warp's
// shared-memory union-find has nothing to gain): their register pressure
// made the narrower tiers spill.
template <int D, int DHI, bool WARP>
__device__ __forceinline__ void run_item(const FusedJob &__restrict__ J, u64 first, const u32 *tab,
                                         u32 *gslab, u32 *ls, u32 *ws, u32 *err_word, u32 &err,
                                         unsigned long long &failed) {
  if constexpr (D <= DHI) {
    if constexpr (WARP && D >= kFusedWarpFrom) {
      if (J.warp) {
        warp_item<D>(J, first, tab, ws, err_word, err, failed);
        return;
      }
    }
    thread_item<D>(J, first, tab, gslab, ls, err_word, err, failed);
  }
}

// smem: [tables (toff bytes)] [mbarrier | work slot (128 bytes)] [label
// slots: ls_words x 128 words] [warp states: 4 x ws_stride words, warp
// tiles only].
template <int DHI, int MINB, bool WARP>
__global__ void __launch_bounds__(kFT, MINB)
    fused_jobs_kernel(const FusedJob *__restrict__ jobs, u32 njobs, u64 total_items,
                      unsigned long long *work, u32 *err_word, unsigned long long *failed_word,
                      u32 *gscratch, u32 toff, u32 ls_words, u32 ws_stride) {
  extern __shared__ __align__(128) uint8_t smem[];
  constexpr u32 SLAB = FusedSlab<DHI>::WORDS;
  u32 *tab = reinterpret_cast<u32 *>(smem);
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + toff);
  unsigned long long *slot = reinterpret_cast<unsigned long long *>(smem + toff + 64);
  u32 *ls = reinterpret_cast<u32 *>(smem + toff + 128) + threadIdx.x;
  u32 *ws = reinterpret_cast<u32 *>(smem + toff + 128) + ls_words * kFT +
            (threadIdx.x >> 5) * ws_stride;
  u32 *gslab = gscratch + (size_t)blockIdx.x * SLAB * kFT;
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  const u32 *cur = nullptr;
  u32 phase = 0, err = 0;
  unsigned long long failed = 0;
  for (;;) {
    if (threadIdx.x == 0) *slot = atomicAdd(work, 1ull);
    __syncthreads();
    const u64 c = *slot;
    __syncthreads();  // also: every thread is done with the previous tables
    if (c >= total_items) break;
    u32 lo = 0, hi = njobs;  // the job holding item c: last j with item0 <= c
    while (hi - lo > 1) {
      const u32 mid = (lo + hi) / 2;
      if (jobs[mid].item0 <= c) lo = mid; else hi = mid;
    }
    const FusedJob &J = jobs[lo];  // fields read where used (L1): no copy to keep live
    if (J.tab != cur) {  // stage the job's tables (cp.async.bulk, bounded wait)
      if (threadIdx.x == 0) {
        mbar_expect_tx(bar, J.tab_words * 4u);
        bulk_g2s(tab, J.tab, J.tab_words * 4u, bar);
      }
      bool ok = false;
      for (long it = 0; it < kWaitIters && !ok; ++it) ok = mbar_try_wait(bar, phase);
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(err_word, kErrTimeout);
        // let a late copy land before the block's shared memory is released
        for (long it = 0; it < kWaitIters && !ok; ++it) ok = mbar_try_wait(bar, phase);
        return;
      }
      phase ^= 1u;
      cur = J.tab;
      if (!J.warp) {  // thread tiles find a fan entry's label slot by its offset
        const u32 d = J.d, lb = 2 * d * d + 2 * d + 1 <= 126 ? 1u : 2u;  // tc_layout's lbytes
        tc_fan_to_offsets(tab + J.off_fan, J.off_vext - J.off_fan, 4u / lb, lb, kFT, threadIdx.x,
                          kFT);
        __syncthreads();
      }
    }
    const u64 first = (c - J.item0) * (u64)J.chunk;
    switch (J.d) {
#define TC_FUSED_CASE(d) \
  case d: run_item<d, DHI, WARP>(J, first, tab, gslab, ls, ws, err_word, err, failed); break;
      TC_FUSED_CASE(1) TC_FUSED_CASE(2) TC_FUSED_CASE(3) TC_FUSED_CASE(4) TC_FUSED_CASE(5)
      TC_FUSED_CASE(6) TC_FUSED_CASE(7) TC_FUSED_CASE(8) TC_FUSED_CASE(9) TC_FUSED_CASE(10)
      TC_FUSED_CASE(11) TC_FUSED_CASE(12) TC_FUSED_CASE(13) TC_FUSED_CASE(14)
      TC_FUSED_CASE(15) TC_FUSED_CASE(16)
#undef TC_FUSED_CASE
      default: err |= kErrInternal; break;
    }
  }
  if (err) atomicOr(err_word, err);
  if (failed) atomicAdd(failed_word, failed);
}

typedef void (*FusedFn)(const FusedJob *, u32, u64, unsigned long long *, u32 *,
                        unsigned long long *, u32 *, u32, u32, u32);

// Tiers 0..3 thread per instance only; kFusedWarpTier: the widest tier
// with warp bodies (any batch with a warp tile runs it).
FusedFn tier_fn(int tier) {
  switch (tier) {
    case 0: return fused_jobs_kernel<kTierD[0], kTierMinB[0], false>;
    case 1: return fused_jobs_kernel<kTierD[1], kTierMinB[1], false>;
    case 2: return fused_jobs_kernel<kTierD[2], kTierMinB[2], false>;
    case 3: return fused_jobs_kernel<kTierD[3], kTierMinB[3], false>;
    case kFusedWarpTier: return fused_jobs_kernel<kTierD[3], kTierMinB[3], true>;
    default: return nullptr;
  }
}

template <int D>
u32 warp_words_d() {
  return TcWarpK<D>::WORDS;
}

}  // namespace

int fused_tier(int dmax) {
  for (int t = 0; t < kFusedTiers; ++t)
    if (dmax <= kTierD[t]) return t;
  return -1;
}

int fused_tier_degree(int tier) {
  if (tier == kFusedWarpTier) return kTierD[kFusedTiers - 1];
  return tier >= 0 && tier < kFusedTiers ? kTierD[tier] : 0;
}

uint32_t fused_slab_words(int tier) {
  switch (tier) {
    case 0: return FusedSlab<kTierD[0]>::WORDS;
    case 1: return FusedSlab<kTierD[1]>::WORDS;
    case 2: return FusedSlab<kTierD[2]>::WORDS;
    case 3:
    case kFusedWarpTier: return FusedSlab<kTierD[3]>::WORDS;
    default: return 0;
  }
}

uint32_t fused_warp_words(int d) {
  switch (d) {
#define TC_WW(x) \
  case x: return warp_words_d<x>();
    TC_WW(1) TC_WW(2) TC_WW(3) TC_WW(4) TC_WW(5) TC_WW(6) TC_WW(7) TC_WW(8) TC_WW(9) TC_WW(10)
    TC_WW(11) TC_WW(12) TC_WW(13) TC_WW(14) TC_WW(15) TC_WW(16)
#undef TC_WW
    default: return 0;
  }
}

cudaError_t fused_occupancy(int tier, size_t smem, int *blocks_per_sm) {
  const FusedFn fn = tier_fn(tier);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute((const void *)fn,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, (const void *)fn, (int)kFT,
                                                       smem);
}

cudaError_t fused_attrs(int tier, int *regs, int *local_bytes) {
  const FusedFn fn = tier_fn(tier);
  if (!fn) return cudaErrorInvalidValue;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaFuncGetAttributes(&fa, (const void *)fn);
  if (e != cudaSuccess) return e;
  *regs = fa.numRegs;
  *local_bytes = (int)fa.localSizeBytes;
  return cudaSuccess;
}

cudaError_t fused_launch(int tier, unsigned grid, size_t smem, uint32_t toff, uint32_t ls_words,
                         uint32_t ws_stride, const FusedJob *jobs, uint32_t njobs, uint64_t items,
                         unsigned long long *work, uint32_t *err, unsigned long long *failed,
                         uint32_t *scratch, cudaStream_t st) {
  const FusedFn fn = tier_fn(tier);
  if (!fn) return cudaErrorInvalidValue;
  fn<<<grid, kFT, smem, st>>>(jobs, njobs, items, work, err, failed, scratch, toff, ls_words,
                              ws_stride);
  return cudaGetLastError();
}

}  // namespace tcurve
