// warp_kernels.cu -- warp-per-instance kernels of the T-curve real-scheme
// engine (TS_KERNEL_WARP): one kernel per degree (1..16), any triangulation
// of that degree.
//
// Each warp classifies one sign vector at a time with Algorithm 1 (Sec. 2),
// its 32 lanes sharing the work (tc_warp_sweep.cuh): signs of all diamond
// vertices, a lock-free union-find over the same-sign edges, the antipodal
// joins, regions and region tree, the root and the canonical code.  The
// whole state of one instance (about 5.5 KB at d = 16) sits in the warp's
// part of shared memory, so no scratch goes to global memory, unlike the
// table-driven kernels, which keep 32 instances per warp there from d = 7.
// The tables (vertex descriptors, edges, antipodal pairs, boundary edges;
// WarpLayout in engine.h) are staged once per block by cp.async.bulk on an
// mbarrier with a bounded wait (tc_stage.cuh).  Sweeps collect the codes of
// 32 instances per warp and insert them with the warp-aggregated histogram
// inserts of the other kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "tc_layout.h"
#include "tc_stage.cuh"
#include "tc_warp_sweep.cuh"

namespace tcurve {
namespace {

constexpr u32 kWarpThreads = 256;  // 8 warps per block, one instance each at a time
constexpr u32 kWarps = kWarpThreads / 32;
constexpr u32 kGrab = 128;         // instances a warp takes from the work counter at once
constexpr int kWarpMinBlocks = 4;  // register budget: 4 resident blocks (64 registers)

template <int D>
struct WarpSmem {
  typedef TcWarpK<D> K;
  static constexpr u32 HASH = K::CW == 1 ? (u32)K::L.hash : 0u;
  static size_t bytes(u32 table_words, bool with_codes) {
    return ((size_t)table_words * 4 + 127) / 128 * 128 + 128 + (size_t)kWarps * K::WORDS * 4 +
           (with_codes ? (size_t)kWarps * 32 * K::CW * 8 + (size_t)HASH * 16 : 0);
  }
  u32 *tab;
  uint64_t *bar;
  u32 *ws;     // kWarps x K::WORDS
  u64 *codes;  // kWarps x 32 x K::CW (sweeps)
  u64 *hkeys;
  unsigned long long *hcnt;
  __device__ WarpSmem(uint8_t *smem, u32 table_words) {
    size_t off = 0;
    tab = reinterpret_cast<u32 *>(smem);
    off += ((size_t)table_words * 4 + 127) / 128 * 128;
    bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 128;
    ws = reinterpret_cast<u32 *>(smem + off);
    off += (size_t)kWarps * K::WORDS * 4;
    off = (off + 7) & ~(size_t)7;
    codes = reinterpret_cast<u64 *>(smem + off);
    off += (size_t)kWarps * 32 * K::CW * 8;
    hkeys = reinterpret_cast<u64 *>(smem + off);
    hcnt = reinterpret_cast<unsigned long long *>(smem + off + (size_t)HASH * 8);
  }
};

template <int D>
__device__ __forceinline__ u32 warp_classify(const TcSig<TcWarpK<D>::W> &sg, const WarpLayout &L,
                                             const u32 *tab, u32 *ws, u64 *code) {
  return tc_warp_classify<D>(sg, tab + L.off_v, tab + L.off_e, L.E, tab + L.off_anti, L.nanti,
                             tab + L.off_bedge, L.nbedge, ws, code);
}

template <int D>
__global__ void __launch_bounds__(kWarpThreads, kWarpMinBlocks)
    warp_real_schemes_kernel(WarpLayout L, const u32 *__restrict__ gtab,
                             const uint64_t *__restrict__ signs, uint64_t n, uint64_t *codes,
                             uint32_t *err_word) {
  typedef TcWarpK<D> K;
  extern __shared__ __align__(128) uint8_t smem[];
  const WarpSmem<D> M(smem, L.words);
  if (!stage_tables(M.tab, gtab, L.words * 4, M.bar, err_word)) return;
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  u32 *ws = M.ws + warp * K::WORDS;
  u32 err = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kWarps + warp; i < n; i += (uint64_t)gridDim.x * kWarps) {
    TcSig<K::W> sg;
#pragma unroll
    for (u32 w = 0; w < K::W; ++w) sg.w[w] = signs[i * K::W + w];
    u64 code[K::CW];
    err |= warp_classify<D>(sg, L, M.tab, ws, code);
    if (lane == 0) {
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) codes[i * K::CW + w] = code[w];
    }
  }
  if (err) atomicOr(err_word, err);
}

template <int D>
__global__ void __launch_bounds__(kWarpThreads, kWarpMinBlocks)
    warp_enumerate_kernel(WarpLayout L, const u32 *__restrict__ gtab, uint64_t lo, uint64_t total,
                          uint32_t flags, ts_hist h) {
  typedef TcWarpK<D> K;
  typedef WarpSmem<D> SM;
  extern __shared__ __align__(128) uint8_t smem[];
  const SM M(smem, L.words);
  if constexpr (SM::HASH > 0)
    for (u32 s = threadIdx.x; s < SM::HASH; s += kWarpThreads) {
      M.hkeys[s] = 0;
      M.hcnt[s] = 0;
    }
  if (!stage_tables(M.tab, gtab, L.words * 4, M.bar, h.d_err)) return;
  const u32 warp = threadIdx.x >> 5, lane = threadIdx.x & 31u;
  u32 *ws = M.ws + warp * K::WORDS;
  u64 *wcodes = M.codes + (size_t)warp * 32 * K::CW;
  u32 err = 0;
  unsigned long long failed = 0;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(h.d_work, (unsigned long long)kGrab);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) break;
    for (u32 g = 0; g < kGrab; g += 32) {
      // 32 instances one after another, lane 0 keeps the codes
      for (u32 j = 0; j < 32; ++j) {
        const uint64_t idx = base + g + j;
        u64 code[K::CW];
#pragma unroll
        for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
        if (idx < total) err |= warp_classify<D>(tc_enum_sig<K::W>(lo + idx, flags, D), L, M.tab, ws, code);
        if (lane == 0) {
#pragma unroll
          for (u32 w = 0; w < K::CW; ++w) wcodes[j * K::CW + w] = code[w];
        }
      }
      __syncwarp();
      // lane j inserts instance j's code (warp-aggregated)
      u64 key[K::CW];
      u64 any = 0;
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) {
        key[w] = wcodes[lane * K::CW + w];
        any |= key[w];
      }
      failed += base + g + lane < total && any == 0;
      if constexpr (K::CW == 1)
        tc_hist_add<SM::HASH>(key[0], M.hkeys, M.hcnt, reinterpret_cast<u64 *>(h.d_keys), h.d_counts,
                              h.slots, h.d_err);
      else
        tc_hist_add_wide<K::CW>(key, reinterpret_cast<u64 *>(h.d_keys), h.d_counts, h.slots, h.d_err);
      __syncwarp();
    }
  }
  __syncthreads();
  if constexpr (SM::HASH > 0)
    for (u32 s = threadIdx.x; s < SM::HASH; s += kWarpThreads)
      if (M.hkeys[s])
        tc_global_add(reinterpret_cast<u64 *>(h.d_keys), h.d_counts, h.slots, h.d_err, M.hkeys[s],
                      M.hcnt[s]);
  if (err) atomicOr(h.d_err, err);
  if (failed) atomicAdd(h.d_failed, failed);
}

int sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Grid of a persistent launch: resident blocks per SM x SMs, at most `want`.
template <class F>
cudaError_t warp_grid(F fn, size_t smem, uint64_t want, unsigned *grid) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWarpThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t cap = (uint64_t)per_sm * sms();
  *grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  return cudaSuccess;
}

template <int D>
cudaError_t real_schemes_w(const ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                           cudaStream_t st) {
  const size_t smem = WarpSmem<D>::bytes(t->wlay.words, false);
  unsigned grid = 0;
  cudaError_t e = warp_grid(warp_real_schemes_kernel<D>, smem, (n + kWarps - 1) / kWarps, &grid);
  if (e != cudaSuccess) return e;
  warp_real_schemes_kernel<D><<<grid, kWarpThreads, smem, st>>>(t->wlay, t->d_wtables, signs, n,
                                                                 codes, t->d_err);
  return cudaGetLastError();
}

template <int D>
cudaError_t enumerate_w(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                        cudaStream_t st) {
  const size_t smem = WarpSmem<D>::bytes(t->wlay.words, true);
  const uint64_t total = hi - lo;
  unsigned grid = 0;
  cudaError_t e = warp_grid(warp_enumerate_kernel<D>, smem,
                            (total + (uint64_t)kWarps * kGrab - 1) / ((uint64_t)kWarps * kGrab), &grid);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  warp_enumerate_kernel<D><<<grid, kWarpThreads, smem, st>>>(t->wlay, t->d_wtables, lo, total, flags,
                                                              *h);
  return cudaGetLastError();
}

}  // namespace

#define TC_WARP_DEGREES(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)

cudaError_t launch_real_schemes_warp(const ts_tri *t, const uint64_t *signs, uint64_t n,
                                     uint64_t *codes, cudaStream_t st) {
  switch (t->d) {
#define TC_CASE(d) \
  case d: return real_schemes_w<d>(t, signs, n, codes, st);
    TC_WARP_DEGREES(TC_CASE)
#undef TC_CASE
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_enumerate_warp(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags,
                                  ts_hist *h, cudaStream_t st) {
  switch (t->d) {
#define TC_CASE(d) \
  case d: return enumerate_w<d>(t, lo, hi, flags, h, st);
    TC_WARP_DEGREES(TC_CASE)
#undef TC_CASE
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace tcurve
