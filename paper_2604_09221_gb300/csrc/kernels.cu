// kernels.cu -- table-driven sm_103a kernels of the T-curve real-scheme
// engine (TS_KERNEL_TABLE): one kernel per degree, any triangulation of that
// degree, no compilation at load time.
//
// One thread classifies one sign vector with Algorithm 1 (Sec. 2):
//   (a) the triangulation tables (host.cpp, layout in engine.h) are copied
//       global -> shared once per block with cp.async.bulk completing on an
//       mbarrier (plain bulk copy, no multicast; bounded wait);
//   (b) the sign of a diamond vertex is bit k(v) of sigma xor the Eq. 2
//       parity constant c(v);
//   (c) an edge is crossed iff its end points' signs differ;
//   (d) Alg. 1 lines 3-4: a sweep of T^diamond in the fixed order of the
//       tables gives every vertex the label of its first same-sign earlier
//       neighbour (or a fresh label); joins between labels (several same-sign
//       runs in a vertex's fan, antipodal pairs) are appended without
//       branching and applied after the sweep (tc_runtime.cuh);
//   (e)-(f) Alg. 1 lines 5-11: tc_backend (regions, region tree from the
//       regions' smallest labels, root, AHU code).  Sweeps add codes to a
//       block-private shared-memory hash table (warp-aggregated) that is merged
//       into the device hash table at the end.
// Per-thread scratch lives in shared memory, interleaved by 32-bit word
// (tc_layout.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"
#include "tc_layout.h"
#include "tc_runtime.cuh"

namespace tcurve {
namespace {

constexpr long kWaitIters = 1L << 22;  // bounded spin on the table mbarrier

// Traits of the table-driven kernels of degree D (scratch with one label per
// vertex, since the sweep is not unrolled).
template <int D_>
struct TableK {
  static constexpr TcLayout L = tc_layout(D_, true, 256);
  static constexpr u32 D = D_, V = L.V, NPOINTS = (D_ + 1) * (D_ + 2) / 2, RMAX = L.rmax,
                       NB = L.nb, THREADS = L.threads, HASH = L.hash, LBYTES = L.lbytes,
                       CODE64 = L.code64, PCAP = L.pcap, WODD = L.wodd, WORDS = L.words,
                       OFF_LPAR = L.off_lpar, OFF_CAND = L.off_cand, OFF_LAB = L.off_lab,
                       OFF_BPAIR = L.off_bpair, OFF_PEND = L.off_pend, OFF_ADJ = L.off_adj,
                       OFF_RLAB = L.off_rlab, OFF_TPAR = L.off_tpar, OFF_ORDER = L.off_order,
                       OFF_CLEN = L.off_clen, OFF_ODD = L.off_odd, OFF_CODE = L.off_code;
  static_assert(L.ok, "scratch layout");
};

// ---------------------------------------------------------------- PTX ----

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                         uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Stage the triangulation tables into shared memory (step (a)).  Every wait
// is bounded; on time-out the block reports kErrTimeout and returns false.
__device__ bool stage_tables(uint32_t *stab, const uint32_t *gtab, uint32_t bytes, uint64_t *bar,
                             uint32_t *err) {
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, bytes);
    bulk_g2s(stab, gtab, bytes, bar);
  }
  bool ok = false;
  for (long it = 0; it < kWaitIters && !ok; ++it) ok = mbar_try_wait(bar, 0);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(err, kErrTimeout);
    // let a late copy land before the block's shared memory is released
    for (long it = 0; it < kWaitIters && !ok; ++it) ok = mbar_try_wait(bar, 0);
    return false;
  }
  return true;
}

// ------------------------------------------------------------- sweep ----

__device__ __forceinline__ u32 sign_bit(u64 sigma, u32 k, u32 c) {
  return ((u32)(sigma >> k) & 1u) ^ c;
}

// Algorithm 1 for one sign vector; returns the code or 0 (err bits set).
template <class K>
__device__ u64 classify(u64 sigma, const u32 *__restrict__ tab, const TableLayout &L,
                        const TcScratch<K> &S, u32 &err) {
  const u32 *vdesc = tab + L.off_vdesc;
  const u32 *fan = tab + L.off_fan;
  const u32 *vext = tab + L.off_vext;
  u32 nl = 0, nb = 0, np = 0;
  tc_clear_odd(S);
  for (u32 v = 0; v < K::V; ++v) {
    const u32 desc = vdesc[v];
    const u32 sv = sign_bit(sigma, desc & 63u, (desc >> 6) & 1u);
    const u32 m = (desc >> 7) & 63u, fs = desc >> 16;
    if (np + m + 1 > K::PCAP) {  // at most m - 1 run joins and one antipodal join at v
      tc_unions(S, np);
      np = 0;
    }
    u32 lv = 0, l0 = TcScratch<K>::NONE, any = 0, prev = 0;
    for (u32 i = 0; i < m; ++i) {
      const u32 f = fan[fs + i];
      const u32 lu = *S.lab(K::OFF_LAB, f & 255u);
      const u32 e = sign_bit(sigma, (f >> 8) & 63u, (f >> 14) & 1u) ^ sv ^ 1u;
      const u32 st = e & ~(((f >> 15) & 1u) & prev) & 1u;  // e starts a run of the fan
      l0 = i == 0 ? lu : l0;
      // a run after the first: join its label with the vertex's label
      S.word(K::OFF_PEND, np) = lv | (lu << 16);
      np += st & any;
      lv = any ? lv : (st ? lu : lv);
      any |= st;
      prev = e;
    }
    if (!any) {
      lv = nl;
      tc_newlab(S, nl, l0);
      ++nl;
    }
    *S.lab(K::OFF_LAB, v) = (typename TcScratch<K>::lab_t)lv;
    const u32 x = vext[v];
    if ((x & 255u) != 255u) {  // the antipodal partner, reached earlier
      S.word(K::OFF_PEND, np) = (u32)*S.lab(K::OFF_LAB, x & 255u) | (lv << 16) | 0x80000000u;
      ++np;
    }
    if (K::D % 2) {  // crossed boundary edges, for the pseudoline's region
#pragma unroll
      for (u32 sh = 8; sh <= 16; sh += 8) {
        const u32 b = (x >> sh) & 255u;
        if (b == 255u) continue;
        const u32 db = vdesc[b];
        if (sign_bit(sigma, db & 63u, (db >> 6) & 1u) != sv) {
          tc_bpair(S, nb, *S.lab(K::OFF_LAB, b), lv);
          ++nb;
        }
      }
    }
  }
  tc_unions(S, np);
  return tc_backend(S, nl, nb, err);
}

template <class K>
constexpr size_t smem_bytes(uint32_t table_words, bool with_hash) {
  return ((size_t)table_words * 4 + 127) / 128 * 128 + 128 + (size_t)K::WORDS * 4 * K::THREADS +
         (with_hash ? (size_t)K::HASH * 16 : 0);
}

struct SmemLayout {
  uint32_t *tab;
  uint64_t *bar;
  unsigned long long *chunk;  // work-chunk broadcast slot (inside the barrier line)
  u32 *scratch;
  u64 *hkeys;
  unsigned long long *hcnt;
};

template <class K>
__device__ SmemLayout carve(uint8_t *smem, uint32_t table_words) {
  SmemLayout s;
  size_t off = 0;
  s.tab = reinterpret_cast<uint32_t *>(smem);
  off += ((size_t)table_words * 4 + 127) / 128 * 128;
  s.bar = reinterpret_cast<uint64_t *>(smem + off);
  s.chunk = reinterpret_cast<unsigned long long *>(smem + off + 64);
  off += 128;
  s.scratch = reinterpret_cast<u32 *>(smem + off);
  off += (size_t)K::WORDS * 4 * K::THREADS;
  s.hkeys = reinterpret_cast<u64 *>(smem + off);
  s.hcnt = reinterpret_cast<unsigned long long *>(smem + off + K::HASH * 8);
  return s;
}

// ----------------------------------------------------- query kernel ----

template <int D>
__global__ void __launch_bounds__(TableK<D>::THREADS)
    real_schemes_kernel(TableLayout L, const uint32_t *__restrict__ gtab,
                        const uint64_t *__restrict__ signs, uint64_t n, uint64_t *codes,
                        uint32_t *err_word) {
  typedef TableK<D> K;
  extern __shared__ __align__(128) uint8_t smem[];
  SmemLayout M = carve<K>(smem, L.words);
  if (!stage_tables(M.tab, gtab, L.words * 4, M.bar, err_word)) return;
  const TcScratch<K> S{M.scratch + threadIdx.x};
  const uint64_t valid = K::NPOINTS >= 64 ? ~0ull : ((1ull << (K::NPOINTS & 63)) - 1);
  uint32_t err = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * K::THREADS + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * K::THREADS)
    codes[i] = classify<K>(signs[i] & valid, M.tab, L, S, err);
  if (err) atomicOr(err_word, err);
}

// ----------------------------------------------- enumeration kernel ----

template <int D>
__global__ void __launch_bounds__(TableK<D>::THREADS)
    enumerate_kernel(TableLayout L, const uint32_t *__restrict__ gtab, uint64_t lo, uint64_t total,
                     uint32_t flags, ts_hist h) {
  typedef TableK<D> K;
  constexpr uint32_t kChunk = K::THREADS * 16;
  extern __shared__ __align__(128) uint8_t smem[];
  SmemLayout M = carve<K>(smem, L.words);
  for (int s = threadIdx.x; s < (int)K::HASH; s += K::THREADS) {
    M.hkeys[s] = 0;
    M.hcnt[s] = 0;
  }
  if (!stage_tables(M.tab, gtab, L.words * 4, M.bar, h.d_err)) return;
  const TcScratch<K> S{M.scratch + threadIdx.x};
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
      uint64_t key = 0;
      if (idx < total) {
        key = classify<K>(tc_enum_mask(lo + idx, flags, D), M.tab, L, S, err);
        failed += key == 0;
      }
      tc_hist_add<K::HASH>(key, M.hkeys, M.hcnt, reinterpret_cast<u64 *>(h.d_keys), h.d_counts,
                           h.slots, h.d_err);
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

// Sign vectors splitmix64(base + i), cut to npoints bits (input generation).
__global__ void splitmix_masks_kernel(uint64_t base, uint64_t n, uint32_t npoints, uint64_t *out) {
  const uint64_t valid = npoints >= 64 ? ~0ull : ((1ull << npoints) - 1);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = tc_splitmix64(base + i) & valid;
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

// ----------------------------------------------------------- launch ----

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int D>
cudaError_t real_schemes_d(const ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                           cudaStream_t st) {
  typedef TableK<D> K;
  const size_t smem = smem_bytes<K>(t->lay.words, false);
  cudaError_t e = cudaFuncSetAttribute(real_schemes_kernel<D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, real_schemes_kernel<D>, K::THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t want = (n + K::THREADS - 1) / K::THREADS;
  uint64_t cap = (uint64_t)per_sm * sm_count();
  unsigned grid = (unsigned)(want < cap ? want : cap);
  real_schemes_kernel<D><<<grid, K::THREADS, smem, st>>>(t->lay, t->d_tables, signs, n, codes, t->d_err);
  return cudaGetLastError();
}

template <int D>
cudaError_t enumerate_d(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                        cudaStream_t st) {
  typedef TableK<D> K;
  const size_t smem = smem_bytes<K>(t->lay.words, true);
  cudaError_t e = cudaFuncSetAttribute(enumerate_kernel<D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enumerate_kernel<D>, K::THREADS, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t total = hi - lo;
  const uint64_t chunk = (uint64_t)K::THREADS * 16;
  uint64_t want = (total + chunk - 1) / chunk;
  uint64_t cap = (uint64_t)per_sm * sm_count();
  unsigned grid = (unsigned)(want < cap ? want : cap);
  e = cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  enumerate_kernel<D><<<grid, K::THREADS, smem, st>>>(t->lay, t->d_tables, lo, total, flags, *h);
  return cudaGetLastError();
}

}  // namespace

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
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_enumerate(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                             cudaStream_t st) {
  switch (t->d) {
    case 1: return enumerate_d<1>(t, lo, hi, flags, h, st);
    case 2: return enumerate_d<2>(t, lo, hi, flags, h, st);
    case 3: return enumerate_d<3>(t, lo, hi, flags, h, st);
    case 4: return enumerate_d<4>(t, lo, hi, flags, h, st);
    case 5: return enumerate_d<5>(t, lo, hi, flags, h, st);
    case 6: return enumerate_d<6>(t, lo, hi, flags, h, st);
    case 7: return enumerate_d<7>(t, lo, hi, flags, h, st);
    case 8: return enumerate_d<8>(t, lo, hi, flags, h, st);
    case 9: return enumerate_d<9>(t, lo, hi, flags, h, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_splitmix_masks(int d, uint64_t base, uint64_t n, uint64_t *out, cudaStream_t st) {
  const uint64_t blocks = (n + 255) / 256;
  splitmix_masks_kernel<<<(unsigned)(blocks < 4096 ? (blocks ? blocks : 1) : 4096), 256, 0, st>>>(
      base, n, (uint32_t)((d + 1) * (d + 2) / 2), out);
  return cudaGetLastError();
}

cudaError_t launch_hist_clear(ts_hist *h, cudaStream_t st) {
  hist_clear_kernel<<<64, 256, 0, st>>>(*h);
  return cudaGetLastError();
}

}  // namespace tcurve
