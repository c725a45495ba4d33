// jit_device.cuh -- device runtime of the triangulation-specialised kernels.
//
// jit.cpp generates, for one loaded triangulation, the sweep of Algorithm 1
// lines 1-4 as straight-line code (the fans of T^diamond become immediate
// bit positions, provisional component labels live in registers) and splices
// it into this file at the marker line.  The prelude defines:
//   TC_D, TC_V, TC_RMAX (regions), TC_NB (boundary-edge slots), TC_THREADS,
//   TC_HASH_SLOTS, TC_LABEL_BYTES (1 or 2), TC_CODE64 (0/1), TC_PCAP
//   (pending-union slots), TC_OFF_LPAR, TC_OFF_CAND, TC_OFF_BPAIR,
//   TC_OFF_PEND, TC_OFF_ADJ, TC_OFF_CODE, TC_OFF_CLEN, TC_OFF_ORDER,
//   TC_OFF_TPAR, TC_OFF_RLAB, TC_OFF_ODD, TC_WODD, TC_WORDS (per-thread scratch, in
//   32-bit words), TC_NPOINTS, TC_B (middle-row bits: the lattice points
//   (i, 0), i <= d, are bits 0..d of a mask).
//
// Labels.  The sweep gives a vertex the label of its first same-sign earlier
// neighbour, or a fresh label when it has none; the fresh label remembers the
// label of the vertex's first earlier neighbour (a crossed edge, "cand").
// Labels are joined in a union-find with orientation parity: parity 0 for two
// labels of one component (a vertex whose same-sign earlier neighbours form
// several runs of its fan), parity 1 across an antipodal boundary pair.  The
// sweep only appends the joins to a per-thread list without branching; one
// loop after the sweep applies them (a full list is applied early), so the
// warp's lanes stay converged during the sweep.  An
// inconsistent join marks the set as containing an odd antipodal cycle, i.e.
// the non-orientable region (Alg. 1 lines 6-7).  The back end turns the sets
// into regions and builds the region tree from the cand edges of the regions'
// smallest labels (see tc_backend), finds the root, and writes the AHU code
// (Alg. 1 line 11).
//
// Scratch words are interleaved across the block's threads (word i of thread
// t at [i * TC_THREADS + t]) so every per-thread access pattern is free of
// shared-memory bank conflicts.

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;
typedef unsigned char u8;

#if TC_LABEL_BYTES == 1
typedef u8 lab_t;
#define TC_EPW 4u
#define TC_TOP 0x80u
#else
typedef u16 lab_t;
#define TC_EPW 2u
#define TC_TOP 0x8000u
#endif
#define TC_LOW (TC_TOP - 1u)
#define TC_NONE TC_LOW

#define TC_ERR_INTERNAL 1u
#define TC_ERR_OVERFLOW 2u

struct TcScratch {
  u32 *w;  // word 0 of this thread
  __device__ __forceinline__ lab_t *lab(u32 off, u32 i) const {
    return reinterpret_cast<lab_t *>(w + (off + i / TC_EPW) * TC_THREADS) + (i % TC_EPW);
  }
  __device__ __forceinline__ u8 *byte(u32 off, u32 i) const {
    return reinterpret_cast<u8 *>(w + (off + (i >> 2)) * TC_THREADS) + (i & 3u);
  }
  __device__ __forceinline__ u32 &word(u32 off, u32 i) const { return w[(off + i) * TC_THREADS]; }
  __device__ __forceinline__ u32 lpar(u32 i) const { return *lab(TC_OFF_LPAR, i); }
  __device__ __forceinline__ void set_lpar(u32 i, u32 v) const { *lab(TC_OFF_LPAR, i) = (lab_t)v; }
  __device__ __forceinline__ u32 cand(u32 i) const { return *lab(TC_OFF_CAND, i); }
  __device__ __forceinline__ void set_cand(u32 i, u32 v) const { *lab(TC_OFF_CAND, i) = (lab_t)v; }
};

__device__ __forceinline__ void tc_newlab(const TcScratch &S, u32 l, u32 c) {
  S.set_lpar(l, l);
  S.set_cand(l, c);
}

__device__ __forceinline__ u32 tc_find(const TcScratch &S, u32 x, u32 &par) {
  par = 0;
  u32 e = S.lpar(x);
  while ((e & TC_LOW) != x) {
    par ^= (e & TC_TOP) ? 1u : 0u;
    x = e & TC_LOW;
    e = S.lpar(x);
  }
  return x;
}

// Odd-cycle flags of the label sets (valid at set roots), one bit per label.
__device__ __forceinline__ u32 tc_odd(const TcScratch &S, u32 l) {
  return (S.word(TC_OFF_ODD, l >> 5) >> (l & 31u)) & 1u;
}
__device__ __forceinline__ void tc_set_odd(const TcScratch &S, u32 l) {
  S.word(TC_OFF_ODD, l >> 5) |= 1u << (l & 31u);
}

// Join labels a and b with relative orientation parity p.
__device__ __forceinline__ void tc_unite(const TcScratch &S, u32 a, u32 b, u32 p) {
  u32 pa, pb;
  const u32 ra = tc_find(S, a, pa), rb = tc_find(S, b, pb);
  const u32 q = (pa ^ pb ^ p) & 1u;
  if (ra == rb) {
    if (q) tc_set_odd(S, ra);  // odd cycle
    return;
  }
  const u32 lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
  S.set_lpar(hi, lo | (q ? TC_TOP : 0u));
  if (tc_odd(S, hi)) tc_set_odd(S, lo);
}

__device__ __forceinline__ void tc_bpair(const TcScratch &S, u32 i, u32 la, u32 lb) {
  S.word(TC_OFF_BPAIR, i) = la | (lb << 16);
}

__device__ __forceinline__ void tc_clear_odd(const TcScratch &S) {
#pragma unroll
  for (u32 w = 0; w < TC_WODD; ++w) S.word(TC_OFF_ODD, w) = 0;
}

// Pending joins: a | b << 16 | parity << 31.
__device__ __noinline__ void tc_unions(const TcScratch &S, u32 np) {
  for (u32 i = 0; i < np; ++i) {
    const u32 e = S.word(TC_OFF_PEND, i);
    tc_unite(S, e & 0xFFFFu, (e >> 16) & 0x7FFFu, e >> 31);
  }
}

#if TC_CODE64
typedef u64 code_t;
#define TC_CODE_BITS 64u
__device__ __forceinline__ code_t tc_code(const TcScratch &S, u32 r) {
  return (u64)S.word(TC_OFF_CODE, 2 * r) | ((u64)S.word(TC_OFF_CODE, 2 * r + 1) << 32);
}
__device__ __forceinline__ void tc_set_code(const TcScratch &S, u32 r, code_t v) {
  S.word(TC_OFF_CODE, 2 * r) = (u32)v;
  S.word(TC_OFF_CODE, 2 * r + 1) = (u32)(v >> 32);
}
#else
typedef u32 code_t;
#define TC_CODE_BITS 32u
__device__ __forceinline__ code_t tc_code(const TcScratch &S, u32 r) { return S.word(TC_OFF_CODE, r); }
__device__ __forceinline__ void tc_set_code(const TcScratch &S, u32 r, code_t v) {
  S.word(TC_OFF_CODE, r) = v;
}
#endif

// Concatenated codes of the regions in `kids`: the non-leaves in descending
// order of their codes (left-aligned bit strings), then '10' once per leaf
// (the smallest code, so leaves always come last).
__device__ __forceinline__ code_t tc_concat(const TcScratch &S, u32 kids, u32 leaves, u32 &len) {
  const code_t rep10 = (code_t)(0xAAAAAAAAAAAAAAAAull >> (64u - TC_CODE_BITS));
  u32 big = kids & ~leaves;
  const u32 nleaf = __popc(kids & leaves);
  code_t v = 0;
  len = 0;
  while (big) {
    u32 best = __ffs(big) - 1;
    code_t bv = tc_code(S, best);
    for (u32 rest = big & (big - 1); rest; rest &= rest - 1) {
      const u32 y = __ffs(rest) - 1;
      const code_t cy = tc_code(S, y);
      if (cy > bv) { bv = cy; best = y; }
    }
    v |= len < TC_CODE_BITS ? (bv >> len) : (code_t)0;
    len += *S.byte(TC_OFF_CLEN, best);
    big &= ~(1u << best);
  }
  if (nleaf) {
    const code_t pat = rep10 & ~(((code_t)~(code_t)0) >> (2 * nleaf));
    v |= len < TC_CODE_BITS ? (pat >> len) : (code_t)0;
    len += 2 * nleaf;
  }
  return v;
}

// enc(region) = '1' . children . '0', stored left-aligned with its length.
__device__ __forceinline__ void tc_store_node(const TcScratch &S, u32 x, code_t v, u32 len) {
  tc_set_code(S, x, ((code_t)1 << (TC_CODE_BITS - 1)) | (v >> 1));
  *S.byte(TC_OFF_CLEN, x) = (u8)(len + 2);
}

// Regions, region tree, root and canonical code from the label sets.
//
// Regions are numbered in the order of their smallest label, which is the
// root of their label set (joins always keep the smaller root).  The smallest
// label of a region r > 0 was created at a vertex whose earlier neighbours all
// have the other sign; its cand label lies in a region with a smaller
// smallest label, i.e. a region p < r across a crossed edge.  These R - 1
// edges join every region to region 0, so they span the region adjacency
// graph; that graph is a tree (each oval separates RP^2), hence they are all
// of it, already oriented towards region 0.  Re-rooting at the non-orientable
// region (or the pseudoline's region) reverses the path between the two.
__device__ __noinline__ u64 tc_backend(const TcScratch &S, u32 nl, u32 nb, u32 &err) {
  // 1. region ids over lpar (label order), odd-cycle flags, smallest labels
  u32 R = 0;
  u64 odd = 0;
  for (u32 l = 0; l < nl; ++l) {
    const u32 p = S.lpar(l) & TC_LOW;
    const u32 is_root = p == l;
    const u32 rp = S.lpar(p);  // p < l holds its region id already
    if (is_root) {
      if (R >= TC_RMAX) { err |= TC_ERR_OVERFLOW; return 0; }
      odd |= (u64)tc_odd(S, l) << R;
      *S.byte(TC_OFF_RLAB, R) = (u8)l;
    }
    S.set_lpar(l, is_root ? R : rp);
    R += is_root;
  }
  // 2. root: odd antipodal cycle (even d) / both sides of the pseudoline (odd d)
  int root = -1;
#if TC_D % 2 == 0
  if (__popcll(odd) != 1) { err |= TC_ERR_INTERNAL; return 0; }
  root = __ffsll(odd) - 1;
#else
  for (u32 i = 0; i < nb; ++i) {
    const u32 e = S.word(TC_OFF_BPAIR, i);
    const u32 ra = S.lpar(e & 0xFFFFu), rb = S.lpar(e >> 16);
    if (ra != rb) continue;
    if (root >= 0 && root != (int)ra) { err |= TC_ERR_INTERNAL; return 0; }
    root = (int)ra;
  }
  if (root < 0) { err |= TC_ERR_INTERNAL; return 0; }
#endif
  // 3. the tree hanging from region 0: parent(r) = region of cand(smallest label of r)
  for (u32 r = 0; r < R; ++r) S.word(TC_OFF_ADJ, r) = 0;
  u32 internal = 0;
  for (u32 r = 1; r < R; ++r) {
    const u32 c = S.cand(*S.byte(TC_OFF_RLAB, r)) & TC_LOW;
    if (c == TC_NONE) { err |= TC_ERR_INTERNAL; return 0; }
    const u32 p = S.lpar(c);
    if (p >= r) { err |= TC_ERR_INTERNAL; return 0; }
    *S.byte(TC_OFF_TPAR, r) = (u8)p;
    S.word(TC_OFF_ADJ, p) |= 1u << r;
    internal |= 1u << p;
  }
  // 4. the path root -> region 0, reversed by re-rooting
  u32 k = 0, path = 1u;
  *S.byte(TC_OFF_ORDER, 0) = (u8)root;
  for (u32 x = (u32)root; x != 0;) {
    x = *S.byte(TC_OFF_TPAR, x);
    *S.byte(TC_OFF_ORDER, ++k) = (u8)x;
    path |= 1u << x;
  }
  // 5. AHU: internal regions off the path (higher index = deeper first), then
  //    the path from region 0 up to the root
  const u32 all = R >= 32 ? ~0u : ((1u << R) - 1);
  u32 leaves = all & ~internal & ~path;
  for (u32 todo = internal & ~path; todo;) {
    const u32 x = 31 - __clz(todo);
    todo &= ~(1u << x);
    u32 len;
    const code_t v = tc_concat(S, S.word(TC_OFF_ADJ, x), leaves, len);
    tc_store_node(S, x, v, len);
  }
  code_t bits = 0;
  u32 nbits = 0;
  for (int i = (int)k; i >= 0; --i) {
    const u32 x = *S.byte(TC_OFF_ORDER, i);
    u32 kids = S.word(TC_OFF_ADJ, x);
    if (i > 0) kids &= ~(1u << *S.byte(TC_OFF_ORDER, i - 1));
    if (i < (int)k) kids |= 1u << *S.byte(TC_OFF_ORDER, i + 1);
    if (i > 0 && !kids) { leaves |= 1u << x; continue; }
    u32 len;
    const code_t v = tc_concat(S, kids, leaves, len);
    if (i > 0) {
      tc_store_node(S, x, v, len);
    } else {
      bits = v;
      nbits = len;
    }
  }
  if (nbits != 2 * (R - 1) || nbits > TC_CODE_BITS - 2) { err |= TC_ERR_INTERNAL; return 0; }
  return (1ull << nbits) | (nbits ? (u64)(bits >> (TC_CODE_BITS - nbits)) : 0ull);
}

__device__ __forceinline__ u32 tc_hash_slot(u64 key, u64 mask) {
  return (u32)(((key * 0x9E3779B97F4A7C15ull) >> 32) & mask);
}

__device__ void tc_global_add(u64 *gkeys, unsigned long long *gcnt, u64 gslots, u32 *gerr, u64 key,
                              unsigned long long cnt) {
  const u64 mask = gslots - 1;
  u64 s = tc_hash_slot(key, mask);
  for (u64 probe = 0; probe < gslots; ++probe) {
    unsigned long long *kp = reinterpret_cast<unsigned long long *>(gkeys + s);
    unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(kp);
    if (k == 0) k = atomicCAS(kp, 0ull, (unsigned long long)key);
    if (k == 0 || k == key) {
      atomicAdd(gcnt + s, cnt);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(gerr, TC_ERR_OVERFLOW);
}

// Warp-aggregated insert into the block's hash table (all 32 lanes call it).
__device__ __forceinline__ void tc_hist_add(u64 key, u64 *hkeys, unsigned long long *hcnt, u64 *gkeys,
                                            unsigned long long *gcnt, u64 gslots, u32 *gerr) {
  const u32 lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (key != 0 && lane == (u32)(__ffs(peers) - 1)) {
    const unsigned long long cnt = (unsigned long long)__popc(peers);
    u32 s = tc_hash_slot(key, TC_HASH_SLOTS - 1);
    for (u32 probe = 0; probe < TC_HASH_SLOTS; ++probe) {
      unsigned long long *kp = reinterpret_cast<unsigned long long *>(hkeys + s);
      unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(kp);
      if (k == 0) k = atomicCAS(kp, 0ull, (unsigned long long)key);
      if (k == 0 || k == key) {
        atomicAdd(hcnt + s, cnt);
        return;
      }
      s = (s + 1) & (TC_HASH_SLOTS - 1);
    }
    tc_global_add(gkeys, gcnt, gslots, gerr, key, cnt);
  }
}

#define TC_BIT(k) ((k) < 32 ? ((slo >> ((k) & 31)) & 1u) : ((shi >> ((k) & 31)) & 1u))

__device__ __forceinline__ u64 tc_classify(u64 sig, const TcScratch &S, u32 &err);
__device__ __forceinline__ void tc_sweep_amortised(u64 sig_hi, u32 ishift, u32 ireps,
                                                   const TcScratch &S, u32 &err,
                                                   u64 *hkeys, unsigned long long *hcnt,
                                                   u64 *gkeys, unsigned long long *gcnt, u64 gslots,
                                                   u32 *gerr, unsigned long long &failed);

//@@SPLICE@@

// ---------------------------------------------------------------- kernels

__device__ __forceinline__ TcScratch tc_scratch(u32 *smem) { return TcScratch{smem + threadIdx.x}; }

extern "C" __global__ void __launch_bounds__(TC_THREADS, 2)
    tc_real_schemes(const u64 *__restrict__ signs, u64 n, u64 *__restrict__ codes, u32 *err_word) {
  extern __shared__ __align__(16) u32 tc_smem[];
  const TcScratch S = tc_scratch(tc_smem);
  const u64 valid = TC_NPOINTS >= 64 ? ~0ull : ((1ull << (TC_NPOINTS & 63)) - 1);
  u32 err = 0;
  for (u64 i = (u64)blockIdx.x * TC_THREADS + threadIdx.x; i < n; i += (u64)gridDim.x * TC_THREADS)
    codes[i] = tc_classify(signs[i] & valid, S, err);
  if (err) atomicOr(err_word, err);
}

__device__ __forceinline__ u64 tc_enum_mask(u64 k, u32 flags) {
  if (flags & 1u) return k << 1;
  if (flags & 2u) return ((k & ((1ull << (TC_D - 1)) - 1)) << 2) | ((k >> (TC_D - 1)) << (TC_D + 2));
  return k;
}

#define TC_CHUNK (TC_THREADS * 16)

extern "C" __global__ void __launch_bounds__(TC_THREADS, 2)
    tc_enumerate(u64 lo, u64 total, u32 flags, u64 *gkeys, unsigned long long *gcnt, u64 gslots,
                 u32 *gerr, unsigned long long *gfailed, unsigned long long *work) {
  extern __shared__ __align__(16) u32 tc_smem[];
  u64 *hkeys = reinterpret_cast<u64 *>(tc_smem + TC_WORDS * TC_THREADS);
  unsigned long long *hcnt = reinterpret_cast<unsigned long long *>(hkeys + TC_HASH_SLOTS);
  unsigned long long *chunk = hcnt + TC_HASH_SLOTS;
  const TcScratch S = tc_scratch(tc_smem);
  for (u32 s = threadIdx.x; s < TC_HASH_SLOTS; s += TC_THREADS) {
    hkeys[s] = 0;
    hcnt[s] = 0;
  }
  __syncthreads();
  u32 err = 0;
  unsigned long long failed = 0;
  for (;;) {
    if (threadIdx.x == 0) *chunk = atomicAdd(work, (unsigned long long)TC_CHUNK);
    __syncthreads();
    const u64 base = *chunk;
    __syncthreads();
    if (base >= total) break;
    for (u32 j = 0; j < TC_CHUNK; j += TC_THREADS) {
      const u64 idx = base + j + threadIdx.x;
      u64 key = 0;
      if (idx < total) {
        key = tc_classify(tc_enum_mask(lo + idx, flags), S, err);
        failed += key == 0;
      }
      tc_hist_add(key, hkeys, hcnt, gkeys, gcnt, gslots, gerr);
    }
  }
  __syncthreads();
  for (u32 s = threadIdx.x; s < TC_HASH_SLOTS; s += TC_THREADS)
    if (hkeys[s]) tc_global_add(gkeys, gcnt, gslots, gerr, hkeys[s], hcnt[s]);
  if (err) atomicOr(gerr, err);
  if (failed) atomicAdd(gfailed, failed);
}

// Exhaustive sweep of whole middle-row blocks: masks (h << oshift) |
// (t << ishift) for h in [hi0, hi0 + n_hi) and every t < 32 * ireps.  Each
// warp takes one h at a time; the two half-diamonds depend on h only and are
// swept once, then every lane classifies ireps middle-row patterns
// (tc_sweep_amortised).
extern "C" __global__ void __launch_bounds__(TC_THREADS, 2)
    tc_enumerate_blocks(u64 hi0, u64 n_hi, u32 oshift, u32 ishift, u32 ireps, u64 *gkeys,
                        unsigned long long *gcnt, u64 gslots,
                        u32 *gerr, unsigned long long *gfailed, unsigned long long *work) {
  extern __shared__ __align__(16) u32 tc_smem[];
  u64 *hkeys = reinterpret_cast<u64 *>(tc_smem + TC_WORDS * TC_THREADS);
  unsigned long long *hcnt = reinterpret_cast<unsigned long long *>(hkeys + TC_HASH_SLOTS);
  const TcScratch S = tc_scratch(tc_smem);
  for (u32 s = threadIdx.x; s < TC_HASH_SLOTS; s += TC_THREADS) {
    hkeys[s] = 0;
    hcnt[s] = 0;
  }
  __syncthreads();
  const u32 lane = threadIdx.x & 31u;
  u32 err = 0;
  unsigned long long failed = 0;
  for (;;) {
    unsigned long long h = 0;
    if (lane == 0) h = atomicAdd(work, 1ull);
    h = __shfl_sync(0xffffffffu, h, 0);
    if (h >= n_hi) break;
    tc_sweep_amortised((hi0 + h) << oshift, ishift, ireps, S, err, hkeys, hcnt, gkeys, gcnt, gslots,
                       gerr, failed);
  }
  __syncthreads();
  for (u32 s = threadIdx.x; s < TC_HASH_SLOTS; s += TC_THREADS)
    if (hkeys[s]) tc_global_add(gkeys, gcnt, gslots, gerr, hkeys[s], hcnt[s]);
  if (err) atomicOr(gerr, err);
  if (failed) atomicAdd(gfailed, failed);
}
