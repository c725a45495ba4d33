// kernels.cu -- table-driven sm_103a kernels of the T-curve real-scheme
// engine (TS_KERNEL_TABLE): one kernel per degree (1..16), any triangulation
// of that degree, no compilation at load time.
//
// One thread classifies one sign vector with Algorithm 1 (Sec. 2):
//   (a) the triangulation tables (host.cpp; format in tc_runtime.cuh) are
//       copied global -> shared once per block with cp.async.bulk completing
//       on an mbarrier (plain bulk copy, no multicast; bounded wait);
//   (b) the sign of a diamond vertex is bit k(v) of sigma xor the Eq. 2
//       parity constant c(v);
//   (c) an edge is crossed iff its end points' signs differ;
//   (d) Alg. 1 lines 3-4: tc_sweep_table gives every vertex the label of its
//       first same-sign earlier neighbour (or a fresh label); joins between
//       labels (several same-sign runs in a vertex's fan, antipodal pairs)
//       are appended without branching and applied on a static schedule;
//   (e)-(f) Alg. 1 lines 5-11: tc_backend / tc_backend_wide (regions, region
//       tree from the regions' smallest labels, root, AHU code).  Sweeps add
//       codes to a block-private shared-memory hash table (warp-aggregated)
//       that is merged into the device hash table at the end (multi-word
//       codes: straight into the device table).
// Per-thread scratch (tc_layout.h) is interleaved by 32-bit word across the
// block, in shared memory or, from d = 7 by default, in global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "engine.h"
#include "tc_layout.h"
#include "tc_stage.cuh"
#include "tc_table_sweep.cuh"

namespace tcurve {
namespace {

// Scratch placement: shared memory (block size from the layout: the
// largest of which two blocks fit an SM), or global memory, L1/L2-resident,
// with 128-thread blocks (more warps per SM for the large degrees, whose
// per-thread scratch leaves room for one or two warps in shared memory).
template <int D, bool G>
using TableK = TcTableK<D, G ? 128 : 256, G>;

// With global scratch the label slots of the sweep (one load per fan
// entry) stay in shared memory: ceil(nslots / labels per word) words per
// thread, interleaved like the scratch.
template <class K>
__host__ __device__ constexpr uint32_t slot_words(uint32_t nslots) {
  return (nslots + TcScratch<K>::EPW - 1) / TcScratch<K>::EPW;
}

template <class K, bool G>
constexpr size_t smem_bytes(uint32_t table_words, uint32_t nslots, bool with_hash) {
  return ((size_t)table_words * 4 + 127) / 128 * 128 + 128 +
         (G ? (size_t)slot_words<K>(nslots) * 4 * K::THREADS : (size_t)K::WORDS * 4 * K::THREADS) +
         (with_hash ? (size_t)K::HASH * 16 : 0);
}

struct SmemLayout {
  uint32_t *tab;
  uint64_t *bar;
  unsigned long long *chunk;  // work-chunk broadcast slot (inside the barrier line)
  u32 *scratch;
  u32 *slots;  // label slots in shared memory (global scratch), else null
  u64 *hkeys;
  unsigned long long *hcnt;
};

template <class K, bool G>
__device__ SmemLayout carve(uint8_t *smem, uint32_t table_words, uint32_t nslots, u32 *gscratch) {
  SmemLayout s;
  size_t off = 0;
  s.tab = reinterpret_cast<uint32_t *>(smem);
  off += ((size_t)table_words * 4 + 127) / 128 * 128;
  s.bar = reinterpret_cast<uint64_t *>(smem + off);
  s.chunk = reinterpret_cast<unsigned long long *>(smem + off + 64);
  off += 128;
  if (G) {
    s.scratch = gscratch + (size_t)blockIdx.x * K::WORDS * K::THREADS;
    s.slots = reinterpret_cast<u32 *>(smem + off);
    off += (size_t)slot_words<K>(nslots) * 4 * K::THREADS;
  } else {
    s.scratch = reinterpret_cast<u32 *>(smem + off);
    s.slots = nullptr;
    off += (size_t)K::WORDS * 4 * K::THREADS;
  }
  s.hkeys = reinterpret_cast<u64 *>(smem + off);
  s.hcnt = reinterpret_cast<unsigned long long *>(smem + off + K::HASH * 8);
  return s;
}

// With global scratch the label slots are in shared memory and the staged
// fan entries are rewritten to their slots' byte offsets (the whole block,
// then a barrier).
template <class K>
__device__ __forceinline__ void fan_offsets(u32 *tab, const TableLayout &L) {
  tc_fan_to_offsets(tab + L.off_fan, L.NF, TcScratch<K>::EPW, K::LBYTES, K::THREADS, threadIdx.x,
                    K::THREADS);
  __syncthreads();
}

// ----------------------------------------------------- query kernel ----

template <int D, bool G>
__global__ void __launch_bounds__(TableK<D, G>::THREADS)
    real_schemes_kernel(TableLayout L, const uint32_t *__restrict__ gtab,
                        const uint64_t *__restrict__ signs, uint64_t n, uint64_t *codes,
                        uint32_t *err_word, u32 *gscratch) {
  typedef TableK<D, G> K;
  extern __shared__ __align__(128) uint8_t smem[];
  SmemLayout M = carve<K, G>(smem, L.words, L.nslots, gscratch);
  if (!stage_tables(M.tab, gtab, L.words * 4, M.bar, err_word)) return;
  const TcScratch<K> S{M.scratch + threadIdx.x};
  u32 *const ls = G ? M.slots + threadIdx.x : nullptr;
  if (G) fan_offsets<K>(M.tab, L);
  const u64 *sg = reinterpret_cast<const u64 *>(signs);
  uint32_t err = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * K::THREADS + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * K::THREADS) {
    const TcCodeOut<K> c =
        tc_table_classify<K, G>(tc_load_sig<K>(sg, i), M.tab, L.off_fan, L.off_vext, S, err, ls);
#pragma unroll
    for (u32 w = 0; w < K::CW; ++w) codes[i * K::CW + w] = c.w[w];
  }
  if (err) atomicOr(err_word, err);
}

// ----------------------------------------------- enumeration kernel ----

template <int D, bool G>
__global__ void __launch_bounds__(TableK<D, G>::THREADS)
    enumerate_kernel(TableLayout L, const uint32_t *__restrict__ gtab, uint64_t lo, uint64_t total,
                     uint32_t flags, ts_hist h, u32 *gscratch) {
  typedef TableK<D, G> K;
  constexpr uint32_t kChunk = K::THREADS * 16;
  extern __shared__ __align__(128) uint8_t smem[];
  SmemLayout M = carve<K, G>(smem, L.words, L.nslots, gscratch);
  for (int s = threadIdx.x; s < (int)K::HASH; s += K::THREADS) {
    M.hkeys[s] = 0;
    M.hcnt[s] = 0;
  }
  if (!stage_tables(M.tab, gtab, L.words * 4, M.bar, h.d_err)) return;
  const TcScratch<K> S{M.scratch + threadIdx.x};
  u32 *const ls = G ? M.slots + threadIdx.x : nullptr;
  if (G) fan_offsets<K>(M.tab, L);
  uint32_t err = 0;
  unsigned long long failed = 0;
  for (;;) {
    if (threadIdx.x == 0) *M.chunk = atomicAdd(h.d_work, (unsigned long long)kChunk);
    __syncthreads();
    const uint64_t base = *M.chunk;
    __syncthreads();
    if (base >= total) break;
    for (uint32_t j = 0; j < kChunk; j += K::THREADS) {
      const uint64_t idx = base + j + threadIdx.x;
      TcCodeOut<K> key{};
      if (idx < total) {
        key = tc_table_classify<K, G>(tc_enum_sig<K::W>(lo + idx, flags, D), M.tab, L.off_fan,
                                      L.off_vext, S, err, ls);
        u64 any = 0;
#pragma unroll
        for (u32 w = 0; w < K::CW; ++w) any |= key.w[w];
        failed += any == 0;
      }
      if constexpr (K::CW == 1)
        tc_hist_add<K::HASH>(key.w[0], M.hkeys, M.hcnt, reinterpret_cast<u64 *>(h.d_keys),
                             h.d_counts, h.slots, h.d_err);
      else
        tc_hist_add_wide<K::CW>(key.w, reinterpret_cast<u64 *>(h.d_keys), h.d_counts, h.slots,
                                h.d_err);
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < (int)K::HASH; s += K::THREADS)
    if (M.hkeys[s])
      tc_global_add(reinterpret_cast<u64 *>(h.d_keys), h.d_counts, h.slots, h.d_err, M.hkeys[s],
                    M.hcnt[s]);
  if (err) atomicOr(h.d_err, err);
  if (failed) atomicAdd(h.d_failed, failed);
}

// Word w of sign vector i is splitmix64((base + i) * W + w); the top word is
// cut to the |A| - 64 (W - 1) bits that exist.
__global__ void splitmix_masks_kernel(uint64_t base, uint64_t n, uint32_t npoints, uint64_t *out) {
  const uint32_t W = (npoints + 63) / 64;
  const uint64_t top = tc_top_mask(npoints, W);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    for (uint32_t w = 0; w < W; ++w) {
      const uint64_t x = tc_splitmix64((base + i) * W + w);
      out[i * W + w] = w + 1 == W ? x & top : x;
    }
}

// Self-test of the bounded waits: the only wait is on an mbarrier that
// nothing completes (no arrival, no copy), polled at most `iters` times; the
// kernel reports kErrTimeout and returns.
__global__ void selftest_wait_kernel(unsigned long long iters, uint32_t *err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);
  __syncthreads();
  bool ok = false;
  for (unsigned long long it = 0; it < iters && !ok; ++it) ok = mbar_try_wait(&bar, 0);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(err, kErrTimeout);
}

__global__ void hist_clear_kernel(ts_hist h) {
  const uint64_t n = h.slots;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    for (int w = 0; w < h.cw; ++w) h.d_keys[i * h.cw + w] = 0;
    h.d_counts[i] = 0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *h.d_err = 0;
    *h.d_failed = 0;
  }
}

// Pack occupied slots (a nonzero key word) into the compaction buffers: one
// atomic per warp, lanes ranked by a ballot.
__global__ void hist_compact_kernel(ts_hist h) {
  const uint64_t n = h.slots;
  const u32 lane = threadIdx.x & 31u;
  for (uint64_t base = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) & ~31ull; base < n;
       base += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t s = base + lane;
    bool nz = false;
    if (s < n)
      for (int w = 0; w < h.cw; ++w) nz |= h.d_keys[s * h.cw + w] != 0;
    const unsigned ball = __ballot_sync(0xffffffffu, nz);
    unsigned long long first = 0;
    if (lane == 0 && ball) first = atomicAdd(h.d_cn, (unsigned long long)__popc(ball));
    first = __shfl_sync(0xffffffffu, first, 0);
    if (nz) {
      const uint64_t o = first + __popc(ball & ((1u << lane) - 1u));
      for (int w = 0; w < h.cw; ++w) h.d_ckeys[o * h.cw + w] = h.d_keys[s * h.cw + w];
      h.d_ccnt[o] = h.d_counts[s] & ((1ull << 62) - 1);
    }
  }
}

// ----------------------------------------------------------- launch ----

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Grid of a persistent launch: resident blocks per SM x SMs, at most `want`.
template <class F>
cudaError_t persistent_grid(F fn, int threads, size_t smem, uint64_t want, unsigned *grid) {
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t cap = (uint64_t)per_sm * sm_count();
  *grid = (unsigned)(want < cap ? (want ? want : 1) : cap);
  return cudaSuccess;
}

// Global scratch of a launch: stream-ordered allocation, freed after it.
struct GlobalScratch {
  u32 *p = nullptr;
  cudaStream_t st;
  explicit GlobalScratch(cudaStream_t s) : st(s) {}
  cudaError_t alloc(size_t bytes) { return scratch_alloc((void **)&p, bytes, st); }
  ~GlobalScratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

template <int D, bool G>
cudaError_t real_schemes_dg(const ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                            cudaStream_t st) {
  typedef TableK<D, G> K;
  const size_t smem = smem_bytes<K, G>(t->lay.words, t->lay.nslots, false);
  unsigned grid = 0;
  cudaError_t e = persistent_grid(real_schemes_kernel<D, G>, K::THREADS, smem,
                                  (n + K::THREADS - 1) / K::THREADS, &grid);
  if (e != cudaSuccess) return e;
  GlobalScratch gs(st);
  if (G && (e = gs.alloc((size_t)grid * K::WORDS * K::THREADS * 4)) != cudaSuccess) return e;
  real_schemes_kernel<D, G><<<grid, K::THREADS, smem, st>>>(t->lay, t->d_tables, signs, n, codes,
                                                            t->d_err, gs.p);
  return cudaGetLastError();
}

template <int D, bool G>
cudaError_t enumerate_dg(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                         cudaStream_t st) {
  typedef TableK<D, G> K;
  const size_t smem = smem_bytes<K, G>(t->lay.words, t->lay.nslots, true);
  const uint64_t total = hi - lo;
  const uint64_t chunk = (uint64_t)K::THREADS * 16;
  unsigned grid = 0;
  cudaError_t e = persistent_grid(enumerate_kernel<D, G>, K::THREADS, smem, (total + chunk - 1) / chunk,
                                  &grid);
  if (e != cudaSuccess) return e;
  GlobalScratch gs(st);
  if (G && (e = gs.alloc((size_t)grid * K::WORDS * K::THREADS * 4)) != cudaSuccess) return e;
  e = cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  enumerate_kernel<D, G><<<grid, K::THREADS, smem, st>>>(t->lay, t->d_tables, lo, total, flags, *h,
                                                         gs.p);
  return cudaGetLastError();
}

// Global scratch from d = 7 unless the triangulation asks otherwise.
bool global_scratch(const ts_tri *t) {
  if (t->scratch == TS_SCRATCH_SHARED) return false;
  if (t->scratch == TS_SCRATCH_GLOBAL) return true;
  return t->d >= kGlobalScratchFrom;
}

template <int D>
cudaError_t real_schemes_d(const ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                           cudaStream_t st) {
  return global_scratch(t) ? real_schemes_dg<D, true>(t, signs, n, codes, st)
                           : real_schemes_dg<D, false>(t, signs, n, codes, st);
}

template <int D>
cudaError_t enumerate_d(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                        cudaStream_t st, bool allow_global) {
  return allow_global && global_scratch(t) ? enumerate_dg<D, true>(t, lo, hi, flags, h, st)
                                           : enumerate_dg<D, false>(t, lo, hi, flags, h, st);
}

}  // namespace

// The device's default pool is told to keep freed memory (release threshold
// at its maximum), so repeated launches reuse it instead of mapping it again.
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t st) {
  static std::once_flag once[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64)
    std::call_once(once[dev], [dev] {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
      }
    });
  return cudaMallocAsync(p, bytes, st);
}

cudaError_t launch_real_schemes(const ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                                cudaStream_t st) {
  switch (t->d) {
    case 1: return real_schemes_d<1>(t, signs, n, codes, st);
    case 2: return real_schemes_d<2>(t, signs, n, codes, st);
    case 3: return real_schemes_d<3>(t, signs, n, codes, st);
    case 4: return real_schemes_d<4>(t, signs, n, codes, st);
    case 5: return real_schemes_d<5>(t, signs, n, codes, st);
    case 6: return real_schemes_d<6>(t, signs, n, codes, st);
    case 7: return real_schemes_d<7>(t, signs, n, codes, st);
    case 8: return real_schemes_d<8>(t, signs, n, codes, st);
    case 9: return real_schemes_d<9>(t, signs, n, codes, st);
    case 10: return real_schemes_d<10>(t, signs, n, codes, st);
    case 11: return real_schemes_d<11>(t, signs, n, codes, st);
    case 12: return real_schemes_d<12>(t, signs, n, codes, st);
    case 13: return real_schemes_d<13>(t, signs, n, codes, st);
    case 14: return real_schemes_d<14>(t, signs, n, codes, st);
    case 15: return real_schemes_d<15>(t, signs, n, codes, st);
    case 16: return real_schemes_d<16>(t, signs, n, codes, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_enumerate(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                             cudaStream_t st, bool allow_global) {
  switch (t->d) {
    case 1: return enumerate_d<1>(t, lo, hi, flags, h, st, allow_global);
    case 2: return enumerate_d<2>(t, lo, hi, flags, h, st, allow_global);
    case 3: return enumerate_d<3>(t, lo, hi, flags, h, st, allow_global);
    case 4: return enumerate_d<4>(t, lo, hi, flags, h, st, allow_global);
    case 5: return enumerate_d<5>(t, lo, hi, flags, h, st, allow_global);
    case 6: return enumerate_d<6>(t, lo, hi, flags, h, st, allow_global);
    case 7: return enumerate_d<7>(t, lo, hi, flags, h, st, allow_global);
    case 8: return enumerate_d<8>(t, lo, hi, flags, h, st, allow_global);
    case 9: return enumerate_d<9>(t, lo, hi, flags, h, st, allow_global);
    case 10: return enumerate_d<10>(t, lo, hi, flags, h, st, allow_global);
    case 11: return enumerate_d<11>(t, lo, hi, flags, h, st, allow_global);
    case 12: return enumerate_d<12>(t, lo, hi, flags, h, st, allow_global);
    case 13: return enumerate_d<13>(t, lo, hi, flags, h, st, allow_global);
    case 14: return enumerate_d<14>(t, lo, hi, flags, h, st, allow_global);
    case 15: return enumerate_d<15>(t, lo, hi, flags, h, st, allow_global);
    case 16: return enumerate_d<16>(t, lo, hi, flags, h, st, allow_global);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_splitmix_masks(int d, uint64_t base, uint64_t n, uint64_t *out, cudaStream_t st) {
  const uint64_t blocks = (n + 255) / 256;
  splitmix_masks_kernel<<<(unsigned)(blocks < 4096 ? (blocks ? blocks : 1) : 4096), 256, 0, st>>>(
      base, n, (uint32_t)((d + 1) * (d + 2) / 2), out);
  return cudaGetLastError();
}

cudaError_t launch_hist_compact(ts_hist *h, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(h->d_cn, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const uint64_t blocks = (h->slots + 255) / 256;
  hist_compact_kernel<<<(unsigned)(blocks < 2048 ? blocks : 2048), 256, 0, st>>>(*h);
  return cudaGetLastError();
}

cudaError_t launch_selftest_wait(unsigned long long iters, uint32_t *err, cudaStream_t st) {
  selftest_wait_kernel<<<1, 32, 0, st>>>(iters, err);
  return cudaGetLastError();
}

cudaError_t launch_hist_clear(ts_hist *h, cudaStream_t st) {
  hist_clear_kernel<<<64, 256, 0, st>>>(*h);
  return cudaGetLastError();
}

}  // namespace tcurve
