// kernels.cu -- sm_103a kernels of the T-curve real-scheme engine.
//
// One thread classifies one sign vector with Algorithm 1 (Sec. 2):
//   (a) the triangulation tables (built on the host, see host.cpp) are
//       copied global -> shared once per block with cp.async.bulk and an
//       mbarrier (plain bulk copy, no multicast);
//   (b) the sign of a diamond vertex is bit k(v) of sigma xor the Eq. 2
//       parity constant c(v);
//   (c) an edge is crossed iff its end points' signs differ;
//   (d) Alg. 1 lines 3-4: union-find over the vertices of T^diamond in a
//       fixed sweep order; each vertex links to its first same-sign earlier
//       neighbour, and only the rare vertex whose same-sign earlier
//       neighbours form several runs of its (angularly ordered) fan needs a
//       real union.  Roots are always the smallest vertex of their set, so a
//       single forward pass flattens the forest into component ids.  The
//       2d antipodal pairs then join components into regions with a parity
//       union-find (each antipodal identification reverses orientation);
//   (e) Alg. 1 lines 5-10: the region adjacency graph.  The first (smallest)
//       vertex of every component has only opposite-sign earlier neighbours;
//       its first earlier neighbour gives one crossed edge to a component
//       with a smaller first vertex.  These edges connect all components,
//       hence all regions, so their projection contains every edge of the
//       region tree.  The root is the region with an odd antipodal cycle
//       (even d) or the region on both sides of a crossed boundary edge,
//       i.e. the side of the pseudoline (odd d);
//   (f) Alg. 1 line 11: AHU canonical form of the tree rooted there; codes
//       of subtrees are left-aligned 64-bit strings, children concatenated
//       in descending order.  The enumeration kernel adds each code to a
//       block-private shared-memory hash table (warp-aggregated) and merges
//       it into the device hash table at the end.
//
// Per-thread scratch lives in shared memory, interleaved by 32-bit word
// (word w of thread t at [w * blockDim + t]) so that any per-thread index
// pattern is free of bank conflicts.
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.h"

namespace tcurve {
namespace {

constexpr int kThreads = 128;
constexpr int kHashSlots = 1024;  // block-private histogram slots (power of 2)
constexpr uint32_t kNone = 0xFFu;
constexpr long kWaitIters = 1L << 22;  // bounded spin on the table mbarrier

template <int D>
struct Dims {
  static constexpr int V = 2 * D * D + 2 * D + 1;          // |A^diamond|
  static constexpr int M = (D - 1) * (D - 2) / 2 + 1;      // Harnack's bound
  static constexpr int NMAX = (D % 2 == 0) ? M : M - 1;    // ovals
  static constexpr int RMAX = NMAX + 1;                     // regions
  static constexpr int VW = (V + 3) / 4;                    // words per V-byte array
  static constexpr int RW = (RMAX + 3) / 4;
  // byte arrays: parent/comp, cand, rpar, rflg (V each); clen, order, tpar (RMAX)
  static constexpr int W32 = 4 * VW + 3 * RW;
  // u64 arrays: adj, code (RMAX each)
  static constexpr int W64 = 2 * RMAX;
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

// ------------------------------------------------ interleaved scratch ----

struct Bytes {  // a per-thread byte array inside the word-interleaved region
  uint8_t *base;  // &region[0 * kThreads + tid] as bytes
  __device__ __forceinline__ uint32_t get(uint32_t i) const {
    return base[(i >> 2) * (4 * kThreads) + (i & 3)];
  }
  __device__ __forceinline__ void set(uint32_t i, uint32_t v) const {
    base[(i >> 2) * (4 * kThreads) + (i & 3)] = (uint8_t)v;
  }
};

struct Words64 {
  uint64_t *base;  // &region[0 * kThreads + tid]
  __device__ __forceinline__ uint64_t get(uint32_t i) const { return base[i * kThreads]; }
  __device__ __forceinline__ void set(uint32_t i, uint64_t v) const { base[i * kThreads] = v; }
};

__device__ __forceinline__ uint32_t sign_bit(uint64_t sigma, uint32_t k, uint32_t c) {
  return ((uint32_t)(sigma >> k) & 1u) ^ c;
}

__device__ __forceinline__ uint32_t uf_find(const Bytes &p, uint32_t x) {
  // path halving; parent[x] <= x is preserved
  uint32_t px = p.get(x);
  while (px != x) {
    uint32_t g = p.get(px);
    p.set(x, g);
    x = g;
    px = p.get(x);
  }
  return x;
}

__device__ __forceinline__ void uf_unite(const Bytes &p, uint32_t a, uint32_t b) {
  uint32_t ra = uf_find(p, a), rb = uf_find(p, b);
  if (ra == rb) return;
  if (ra < rb) p.set(rb, ra);
  else p.set(ra, rb);
}

// Returns the canonical code of one instance, or 0 (and sets err bits).
template <int D>
__device__ uint64_t classify(uint64_t sigma, const uint32_t *__restrict__ tab, const TableLayout &L,
                             uint32_t *s32, uint64_t *s64, uint32_t &err) {
  using K = Dims<D>;
  const uint32_t *vdesc = tab + L.off_vdesc;
  const uint32_t *fan = tab + L.off_fan;
  uint8_t *b8 = reinterpret_cast<uint8_t *>(s32);
  const Bytes parent{b8};
  const Bytes cand{b8 + 1 * K::VW * 4 * kThreads};
  const Bytes rpar{b8 + 2 * K::VW * 4 * kThreads};
  const Bytes rflg{b8 + 3 * K::VW * 4 * kThreads};
  const Bytes clen{b8 + 4 * K::VW * 4 * kThreads};
  const Bytes order{b8 + (4 * K::VW + K::RW) * 4 * kThreads};
  const Bytes tpar{b8 + (4 * K::VW + 2 * K::RW) * 4 * kThreads};
  const Words64 adj{s64};
  const Words64 code{s64 + K::RMAX * kThreads};

  // ---- (b)-(d): same-sign components in one sweep ----
  for (uint32_t v = 0; v < (uint32_t)K::V; ++v) {
    const uint32_t desc = vdesc[v];
    const uint32_t sv = sign_bit(sigma, desc & 63u, (desc >> 6) & 1u);
    const uint32_t m = (desc >> 7) & 63u, fs = desc >> 16;
    uint32_t p = v, runs = 0, prev = 0;
    for (uint32_t i = 0; i < m; ++i) {
      const uint32_t f = fan[fs + i];
      const uint32_t same = sign_bit(sigma, (f >> 8) & 63u, (f >> 14) & 1u) == sv;
      const uint32_t start = same & ~(((f >> 15) & 1u) & prev) & 1u;
      if (start && runs == 0) p = f & 255u;
      runs += start;
      prev = same;
    }
    parent.set(v, p);
    if (runs >= 2) {
      // same-sign earlier neighbours in several runs: join the later runs
      prev = 0;
      uint32_t first = 1;
      for (uint32_t i = 0; i < m; ++i) {
        const uint32_t f = fan[fs + i];
        const uint32_t same = sign_bit(sigma, (f >> 8) & 63u, (f >> 14) & 1u) == sv;
        const uint32_t start = same & ~(((f >> 15) & 1u) & prev) & 1u;
        if (start) {
          if (!first) uf_unite(parent, v, f & 255u);
          first = 0;
        }
        prev = same;
      }
    }
  }

  // ---- flatten into component ids; candidate crossed edge per component ----
  uint32_t C = 0;
  for (uint32_t v = 0; v < (uint32_t)K::V; ++v) {
    const uint32_t p = parent.get(v);
    if (p == v) {
      const uint32_t desc = vdesc[v];
      const uint32_t m = (desc >> 7) & 63u;
      parent.set(v, C);
      cand.set(C, m ? parent.get(fan[desc >> 16] & 255u) : kNone);
      ++C;
    } else {
      parent.set(v, parent.get(p));
    }
  }

  // ---- regions: antipodal pairs with orientation parity ----
  for (uint32_t c = 0; c < C; ++c) {
    rpar.set(c, c);
    rflg.set(c, 0);
  }
  const uint32_t *anti = tab + L.off_anti;
  for (uint32_t a = 0; a < L.n_anti; ++a) {
    const uint32_t e = anti[a];
    uint32_t x = parent.get(e & 255u), y = parent.get((e >> 8) & 255u);
    uint32_t px = 0, py = 0, r;
    while ((r = rpar.get(x)) != x) { px ^= rflg.get(x) & 1u; x = r; }
    while ((r = rpar.get(y)) != y) { py ^= rflg.get(y) & 1u; y = r; }
    if (x == y) {
      if (px == py) rflg.set(x, rflg.get(x) | 2u);  // odd cycle: non-orientable
    } else {
      const uint32_t lo = x < y ? x : y, hi = x < y ? y : x;
      const uint32_t fh = rflg.get(hi);
      rpar.set(hi, lo);
      rflg.set(hi, (fh & 2u) | (px ^ py ^ 1u));
      if (fh & 2u) rflg.set(lo, rflg.get(lo) | 2u);
    }
  }
  uint32_t R = 0;
  uint64_t oddmask = 0;
  for (uint32_t c = 0; c < C; ++c) {
    const uint32_t r = rpar.get(c);
    if (r == c) {
      if (R >= (uint32_t)K::RMAX) { err |= kErrOverflow; return 0; }
      if (rflg.get(c) & 2u) oddmask |= 1ull << R;
      rpar.set(c, R);
      ++R;
    } else {
      rpar.set(c, rpar.get(r));
    }
  }

  // ---- (e) region tree from the candidate edges; root ----
  for (uint32_t r = 0; r < R; ++r) adj.set(r, 0);
  for (uint32_t c = 1; c < C; ++c) {
    const uint32_t cb = cand.get(c);
    if (cb == kNone) continue;
    const uint32_t a = rpar.get(c), b = rpar.get(cb);
    if (a != b) {
      adj.set(a, adj.get(a) | (1ull << b));
      adj.set(b, adj.get(b) | (1ull << a));
    }
  }
  int root = -1;
  if (D % 2 == 0) {
    if (__popcll(oddmask) != 1) { err |= kErrInternal; return 0; }
    root = __ffsll(oddmask) - 1;
  } else {
    const uint32_t *bedge = tab + L.off_bedge;
    for (uint32_t a = 0; a < L.n_bedge; ++a) {
      const uint32_t e = bedge[a];
      const uint32_t sa = sign_bit(sigma, (e >> 16) & 63u, (e >> 22) & 1u);
      const uint32_t sb = sign_bit(sigma, (e >> 23) & 63u, (e >> 29) & 1u);
      if (sa == sb) continue;
      const uint32_t ra = rpar.get(parent.get(e & 255u)), rb = rpar.get(parent.get((e >> 8) & 255u));
      if (ra != rb) continue;
      if (root >= 0 && root != (int)ra) { err |= kErrInternal; return 0; }
      root = (int)ra;
    }
    if (root < 0) { err |= kErrInternal; return 0; }
  }
  uint32_t deg2 = 0;
  for (uint32_t r = 0; r < R; ++r) deg2 += __popcll(adj.get(r));
  if (deg2 != 2 * (R - 1)) { err |= kErrInternal; return 0; }

  // ---- (f) BFS from the root, then AHU codes bottom-up ----
  order.set(0, root);
  tpar.set(root, kNone);
  uint64_t seen = 1ull << root;
  uint32_t n = 1;
  for (uint32_t q = 0; q < n; ++q) {
    const uint32_t x = order.get(q);
    uint64_t kids = adj.get(x) & ~seen;
    seen |= kids;
    while (kids) {
      const uint32_t y = __ffsll(kids) - 1;
      kids &= kids - 1;
      order.set(n++, y);
      tpar.set(y, x);
    }
  }
  if (n != R) { err |= kErrInternal; return 0; }
  uint64_t bits = 0;
  uint32_t nbits = 0;
  for (int q = (int)n - 1; q >= 0; --q) {
    const uint32_t x = order.get(q);
    const uint32_t px = tpar.get(x);
    uint64_t kids = adj.get(x) & ~(px == kNone ? 0ull : (1ull << px));
    uint64_t v = 0;
    uint32_t len = 0;
    while (kids) {
      uint32_t best = __ffsll(kids) - 1;
      uint64_t bv = code.get(best);
      for (uint64_t rest = kids & (kids - 1); rest; rest &= rest - 1) {
        const uint32_t y = __ffsll(rest) - 1;
        const uint64_t cy = code.get(y);
        if (cy > bv) { bv = cy; best = y; }
      }
      v |= len < 64 ? (bv >> len) : 0;
      len += clen.get(best);
      kids &= ~(1ull << best);
    }
    if (px != kNone) {
      code.set(x, (1ull << 63) | (v >> 1));
      clen.set(x, len + 2);
    } else {
      bits = v;
      nbits = len;
    }
  }
  if (nbits != 2 * (R - 1) || nbits > 62) { err |= kErrInternal; return 0; }
  return (1ull << nbits) | (nbits ? bits >> (64 - nbits) : 0ull);
}

template <int D>
constexpr size_t smem_bytes(uint32_t table_words, bool with_hash) {
  return ((size_t)table_words * 4 + 127) / 128 * 128 + 128 +
         (size_t)Dims<D>::W32 * 4 * kThreads + (size_t)Dims<D>::W64 * 8 * kThreads +
         (with_hash ? (size_t)kHashSlots * 16 : 0);
}

struct SmemLayout {
  uint32_t *tab;
  uint64_t *bar;
  uint32_t *s32;
  uint64_t *s64;
  uint64_t *hkeys;
  unsigned long long *hcnt;
  unsigned long long *chunk;  // work-chunk broadcast slot (inside the barrier line)
};

template <int D>
__device__ SmemLayout carve(uint8_t *smem, uint32_t table_words) {
  SmemLayout s;
  size_t off = 0;
  s.tab = reinterpret_cast<uint32_t *>(smem);
  off += ((size_t)table_words * 4 + 127) / 128 * 128;
  s.bar = reinterpret_cast<uint64_t *>(smem + off);
  s.chunk = reinterpret_cast<unsigned long long *>(smem + off + 64);
  off += 128;
  s.s32 = reinterpret_cast<uint32_t *>(smem + off) + threadIdx.x;
  off += (size_t)Dims<D>::W32 * 4 * kThreads;
  s.s64 = reinterpret_cast<uint64_t *>(smem + off) + threadIdx.x;
  off += (size_t)Dims<D>::W64 * 8 * kThreads;
  s.hkeys = reinterpret_cast<uint64_t *>(smem + off);
  s.hcnt = reinterpret_cast<unsigned long long *>(smem + off + kHashSlots * 8);
  return s;
}

// ----------------------------------------------------- query kernel ----

template <int D>
__global__ void __launch_bounds__(kThreads) real_schemes_kernel(TableLayout L,
                                                                 const uint32_t *__restrict__ gtab,
                                                                 const uint64_t *__restrict__ signs,
                                                                 uint64_t n, uint64_t *codes,
                                                                 uint32_t *err_word) {
  extern __shared__ __align__(128) uint8_t smem[];
  SmemLayout S = carve<D>(smem, L.words);
  if (!stage_tables(S.tab, gtab, L.words * 4, S.bar, err_word)) return;
  constexpr int kPoints = (D + 1) * (D + 2) / 2;
  const uint64_t valid = kPoints >= 64 ? ~0ull : ((1ull << (kPoints & 63)) - 1);
  uint32_t err = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * kThreads) {
    const uint64_t sigma = signs[i] & valid;
    codes[i] = classify<D>(sigma, S.tab, L, S.s32, S.s64, err);
  }
  if (err) atomicOr(err_word, err);
}

// ----------------------------------------------- enumeration kernel ----

__device__ __forceinline__ uint32_t hash_slot(uint64_t key, uint64_t mask) {
  return (uint32_t)(((key * 0x9E3779B97F4A7C15ull) >> 32) & mask);
}

__device__ void global_add(ts_hist h, uint64_t key, unsigned long long cnt) {
  const uint64_t mask = h.slots - 1;
  uint64_t s = hash_slot(key, mask);
  for (uint64_t probe = 0; probe < h.slots; ++probe) {
    unsigned long long *kp = reinterpret_cast<unsigned long long *>(h.d_keys + s);
    unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(kp);
    if (k == 0) k = atomicCAS(kp, 0ull, (unsigned long long)key);
    if (k == 0 || k == key) {
      atomicAdd(h.d_counts + s, cnt);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(h.d_err, kErrOverflow);
}

__device__ void shared_add(uint64_t *keys, unsigned long long *cnt, const ts_hist &h, uint64_t key,
                           unsigned long long n) {
  uint32_t s = hash_slot(key, kHashSlots - 1);
  for (int probe = 0; probe < kHashSlots; ++probe) {
    unsigned long long *kp = reinterpret_cast<unsigned long long *>(keys + s);
    unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(kp);
    if (k == 0) k = atomicCAS(kp, 0ull, (unsigned long long)key);
    if (k == 0 || k == key) {
      atomicAdd(cnt + s, n);
      return;
    }
    s = (s + 1) & (kHashSlots - 1);
  }
  global_add(h, key, n);  // block table full: go straight to the device table
}

__device__ __forceinline__ uint64_t enum_mask(uint64_t k, uint32_t flags, int d) {
  if (flags & TS_ENUM_FLIP) return k << 1;
  if (flags & TS_ENUM_REDUCED)
    return ((k & ((1ull << (d - 1)) - 1)) << 2) | ((k >> (d - 1)) << (d + 2));
  return k;
}

constexpr uint32_t kChunk = kThreads * 16;

template <int D>
__global__ void __launch_bounds__(kThreads) enumerate_kernel(TableLayout L,
                                                              const uint32_t *__restrict__ gtab,
                                                              uint64_t lo, uint64_t total,
                                                              uint32_t flags, ts_hist h) {
  extern __shared__ __align__(128) uint8_t smem[];
  SmemLayout S = carve<D>(smem, L.words);
  for (int s = threadIdx.x; s < kHashSlots; s += kThreads) {
    S.hkeys[s] = 0;
    S.hcnt[s] = 0;
  }
  if (!stage_tables(S.tab, gtab, L.words * 4, S.bar, h.d_err)) return;
  const uint32_t lane = threadIdx.x & 31u;
  uint32_t err = 0;
  unsigned long long failed = 0;
  for (;;) {
    if (threadIdx.x == 0) *S.chunk = atomicAdd(h.d_work, (unsigned long long)kChunk);
    __syncthreads();
    const uint64_t base = *S.chunk;
    __syncthreads();
    if (base >= total) break;
    for (uint32_t j = 0; j < kChunk; j += kThreads) {
      const uint64_t idx = base + j + threadIdx.x;
      uint64_t key = 0;
      if (idx < total) {
        key = classify<D>(enum_mask(lo + idx, flags, D), S.tab, L, S.s32, S.s64, err);
        failed += key == 0;
      }
      const unsigned peers = __match_any_sync(0xffffffffu, key);
      if (key != 0 && lane == (uint32_t)(__ffs(peers) - 1))
        shared_add(S.hkeys, S.hcnt, h, key, (unsigned long long)__popc(peers));
    }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < kHashSlots; s += kThreads)
    if (S.hkeys[s]) global_add(h, S.hkeys[s], S.hcnt[s]);
  if (err) atomicOr(h.d_err, err);
  if (failed) atomicAdd(h.d_failed, failed);
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
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int D>
cudaError_t real_schemes_d(const ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                           cudaStream_t st) {
  const size_t smem = smem_bytes<D>(t->lay.words, false);
  cudaError_t e = cudaFuncSetAttribute(real_schemes_kernel<D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, real_schemes_kernel<D>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  uint64_t want = (n + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)per_sm * sm_count();
  unsigned grid = (unsigned)(want < cap ? want : cap);
  real_schemes_kernel<D><<<grid, kThreads, smem, st>>>(t->lay, t->d_tables, signs, n, codes, t->d_err);
  return cudaGetLastError();
}

template <int D>
cudaError_t enumerate_d(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                        cudaStream_t st) {
  const size_t smem = smem_bytes<D>(t->lay.words, true);
  cudaError_t e = cudaFuncSetAttribute(enumerate_kernel<D>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, enumerate_kernel<D>, kThreads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const uint64_t total = hi - lo;
  uint64_t want = (total + kChunk - 1) / kChunk;
  uint64_t cap = (uint64_t)per_sm * sm_count();
  unsigned grid = (unsigned)(want < cap ? want : cap);
  e = cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  enumerate_kernel<D><<<grid, kThreads, smem, st>>>(t->lay, t->d_tables, lo, total, flags, *h);
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

cudaError_t launch_hist_clear(ts_hist *h, cudaStream_t st) {
  hist_clear_kernel<<<64, 256, 0, st>>>(*h);
  return cudaGetLastError();
}

}  // namespace tcurve
