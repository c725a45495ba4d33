// tc_runtime.cuh -- per-instance runtime of the label-sweep kernels: the
// label union-find, the back end (regions, region tree, root, canonical code)
// and the block-private hash histogram.  Included by kernels.cu (nvcc, the
// table-driven kernels) and embedded in every generated source (NVRTC, the
// triangulation-specialised kernels).  Everything is a template on a traits
// class K that carries the degree, the block size and the scratch layout of
// tc_layout.h as static constexpr members (D, V, THREADS, HASH, RMAX, LBYTES,
// CODE64, PCAP, WODD, OFF_LPAR, OFF_CAND, OFF_LAB, OFF_BPAIR, OFF_PEND,
// OFF_ADJ, OFF_RLAB, OFF_TPAR, OFF_ORDER, OFF_CLEN, OFF_ODD, OFF_CODE).
//
// Labels.  A sweep of T^diamond (Alg. 1, lines 1-4) gives each vertex the
// label of its first same-sign earlier neighbour, or a fresh label when it
// has none; a fresh label remembers the label of the vertex's first earlier
// neighbour, across a crossed edge ("cand").  Labels are joined in a
// union-find with orientation parity: parity 0 for two labels of one
// component (a vertex whose same-sign earlier neighbours form several runs of
// its fan), parity 1 across an antipodal boundary pair.  Sweeps append joins
// to a per-thread list without branching and tc_unions applies them, which
// keeps a warp's lanes converged.  An inconsistent join marks the set as
// containing an odd antipodal cycle: the non-orientable region (Alg. 1, lines
// 6-7; proof of Thm. 2).
#pragma once

typedef unsigned long long u64;
typedef unsigned int u32;
typedef unsigned short u16;
typedef unsigned char u8;

template <u32 B>
struct TcLab;
template <>
struct TcLab<1> {
  typedef u8 T;
  static constexpr u32 EPW = 4, TOP = 0x80u;
};
template <>
struct TcLab<2> {
  typedef u16 T;
  static constexpr u32 EPW = 2, TOP = 0x8000u;
};

constexpr u32 TC_ERR_INTERNAL = 1u;
constexpr u32 TC_ERR_OVERFLOW = 2u;

template <class K>
struct TcScratch {
  typedef typename TcLab<K::LBYTES>::T lab_t;
  static constexpr u32 EPW = TcLab<K::LBYTES>::EPW;
  static constexpr u32 TOP = TcLab<K::LBYTES>::TOP;  // parity bit of a parent link
  static constexpr u32 LOW = TOP - 1u;
  static constexpr u32 NONE = LOW;                   // "no cand label"
  u32 *w;                                            // word 0 of this thread
  __device__ __forceinline__ lab_t *lab(u32 off, u32 i) const {
    return reinterpret_cast<lab_t *>(w + (off + i / EPW) * K::THREADS) + (i % EPW);
  }
  __device__ __forceinline__ u8 *byte(u32 off, u32 i) const {
    return reinterpret_cast<u8 *>(w + (off + (i >> 2)) * K::THREADS) + (i & 3u);
  }
  __device__ __forceinline__ u32 &word(u32 off, u32 i) const { return w[(off + i) * K::THREADS]; }
  __device__ __forceinline__ u32 lpar(u32 i) const { return *lab(K::OFF_LPAR, i); }
  __device__ __forceinline__ void set_lpar(u32 i, u32 v) const { *lab(K::OFF_LPAR, i) = (lab_t)v; }
  __device__ __forceinline__ u32 cand(u32 i) const { return *lab(K::OFF_CAND, i); }
  __device__ __forceinline__ void set_cand(u32 i, u32 v) const { *lab(K::OFF_CAND, i) = (lab_t)v; }
};

template <class K>
__device__ __forceinline__ void tc_newlab(const TcScratch<K> &S, u32 l, u32 c) {
  S.set_lpar(l, l);
  S.set_cand(l, c);
}

template <class K>
__device__ __forceinline__ u32 tc_find(const TcScratch<K> &S, u32 x, u32 &par) {
  par = 0;
  u32 e = S.lpar(x);
  while ((e & TcScratch<K>::LOW) != x) {
    par ^= (e & TcScratch<K>::TOP) ? 1u : 0u;
    x = e & TcScratch<K>::LOW;
    e = S.lpar(x);
  }
  return x;
}

// Odd-cycle flags of the label sets (valid at set roots), one bit per label.
template <class K>
__device__ __forceinline__ u32 tc_odd(const TcScratch<K> &S, u32 l) {
  return (S.word(K::OFF_ODD, l >> 5) >> (l & 31u)) & 1u;
}
template <class K>
__device__ __forceinline__ void tc_set_odd(const TcScratch<K> &S, u32 l) {
  S.word(K::OFF_ODD, l >> 5) |= 1u << (l & 31u);
}
template <class K>
__device__ __forceinline__ void tc_clear_odd(const TcScratch<K> &S) {
#pragma unroll
  for (u32 w = 0; w < K::WODD; ++w) S.word(K::OFF_ODD, w) = 0;
}

// Join labels a and b with relative orientation parity p.
template <class K>
__device__ __forceinline__ void tc_unite(const TcScratch<K> &S, u32 a, u32 b, u32 p) {
  u32 pa, pb;
  const u32 ra = tc_find(S, a, pa), rb = tc_find(S, b, pb);
  const u32 q = (pa ^ pb ^ p) & 1u;
  if (ra == rb) {
    if (q) tc_set_odd(S, ra);  // odd cycle
    return;
  }
  const u32 lo = ra < rb ? ra : rb, hi = ra < rb ? rb : ra;
  S.set_lpar(hi, lo | (q ? TcScratch<K>::TOP : 0u));
  if (tc_odd(S, hi)) tc_set_odd(S, lo);
}

template <class K>
__device__ __forceinline__ void tc_bpair(const TcScratch<K> &S, u32 i, u32 la, u32 lb) {
  S.word(K::OFF_BPAIR, i) = la | (lb << 16);
}

// Apply the pending joins (a | b << 16 | parity << 31).
template <class K>
__device__ __noinline__ void tc_unions(const TcScratch<K> &S, u32 np) {
  for (u32 i = 0; i < np; ++i) {
    const u32 e = S.word(K::OFF_PEND, i);
    tc_unite(S, e & 0xFFFFu, (e >> 16) & 0x7FFFu, e >> 31);
  }
}

template <u32 C64>
struct TcCode;
template <>
struct TcCode<0> {
  typedef u32 T;
  static constexpr u32 BITS = 32;
};
template <>
struct TcCode<1> {
  typedef u64 T;
  static constexpr u32 BITS = 64;
};

template <class K>
__device__ __forceinline__ typename TcCode<K::CODE64>::T tc_code(const TcScratch<K> &S, u32 r) {
  if (K::CODE64)
    return (typename TcCode<K::CODE64>::T)((u64)S.word(K::OFF_CODE, 2 * r) |
                                           ((u64)S.word(K::OFF_CODE, 2 * r + 1) << 32));
  return (typename TcCode<K::CODE64>::T)S.word(K::OFF_CODE, r);
}
template <class K>
__device__ __forceinline__ void tc_set_code(const TcScratch<K> &S, u32 r,
                                            typename TcCode<K::CODE64>::T v) {
  if (K::CODE64) {
    S.word(K::OFF_CODE, 2 * r) = (u32)v;
    S.word(K::OFF_CODE, 2 * r + 1) = (u32)((u64)v >> 32);
  } else {
    S.word(K::OFF_CODE, r) = (u32)v;
  }
}

// Concatenated codes of the regions in `kids`: the non-leaves in descending
// order of their codes (left-aligned bit strings), then '10' once per leaf
// (the smallest code, so leaves always come last).
template <class K>
__device__ __forceinline__ typename TcCode<K::CODE64>::T tc_concat(const TcScratch<K> &S, u32 kids,
                                                                  u32 leaves, u32 &len) {
  typedef typename TcCode<K::CODE64>::T code_t;
  constexpr u32 BITS = TcCode<K::CODE64>::BITS;
  const code_t rep10 = (code_t)(0xAAAAAAAAAAAAAAAAull >> (64u - BITS));
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
      if (cy > bv) {
        bv = cy;
        best = y;
      }
    }
    v |= len < BITS ? (bv >> len) : (code_t)0;
    len += *S.byte(K::OFF_CLEN, best);
    big &= ~(1u << best);
  }
  if (nleaf) {
    const code_t pat = rep10 & ~(((code_t)~(code_t)0) >> (2 * nleaf));
    v |= len < BITS ? (pat >> len) : (code_t)0;
    len += 2 * nleaf;
  }
  return v;
}

// enc(region) = '1' . children . '0', stored left-aligned with its length.
template <class K>
__device__ __forceinline__ void tc_store_node(const TcScratch<K> &S, u32 x,
                                              typename TcCode<K::CODE64>::T v, u32 len) {
  constexpr u32 BITS = TcCode<K::CODE64>::BITS;
  tc_set_code(S, x, ((typename TcCode<K::CODE64>::T)1 << (BITS - 1)) | (v >> 1));
  *S.byte(K::OFF_CLEN, x) = (u8)(len + 2);
}

// Regions, region tree, root and canonical code from the label sets
// (Alg. 1, lines 5-11).
//
// Regions are numbered in the order of their smallest label, which is the
// root of their label set (joins keep the smaller root).  The smallest label
// of a region r > 0 was created at a vertex whose earlier neighbours all have
// the other sign; its cand label lies in a region with a smaller smallest
// label, i.e. a region p < r across a crossed edge.  These R - 1 edges join
// every region to region 0, so they span the region adjacency graph; that
// graph is a tree (each oval separates RP^2), hence they are all of it,
// already oriented towards region 0.  Re-rooting at the non-orientable region
// (even d) or the pseudoline's region (odd d) reverses the path between the
// two.  AHU codes follow, internal regions only: a leaf's code is '10'.
template <class K>
__device__ __noinline__ u64 tc_backend(const TcScratch<K> &S, u32 nl, u32 nb, u32 &err) {
  typedef typename TcCode<K::CODE64>::T code_t;
  constexpr u32 BITS = TcCode<K::CODE64>::BITS;
  // 1. region ids over lpar (label order), odd-cycle flags, smallest labels
  u32 R = 0;
  u64 odd = 0;
  for (u32 l = 0; l < nl; ++l) {
    const u32 p = S.lpar(l) & TcScratch<K>::LOW;
    const u32 is_root = p == l;
    const u32 rp = S.lpar(p);  // p < l holds its region id already
    if (is_root) {
      if (R >= K::RMAX) {
        err |= TC_ERR_OVERFLOW;
        return 0;
      }
      odd |= (u64)tc_odd(S, l) << R;
      *S.byte(K::OFF_RLAB, R) = (u8)l;
    }
    S.set_lpar(l, is_root ? R : rp);
    R += is_root;
  }
  // 2. root: odd antipodal cycle (even d) / both sides of the pseudoline (odd d)
  int root = -1;
  if (K::D % 2 == 0) {
    if (__popcll(odd) != 1) {
      err |= TC_ERR_INTERNAL;
      return 0;
    }
    root = __ffsll(odd) - 1;
  } else {
    for (u32 i = 0; i < nb; ++i) {
      const u32 e = S.word(K::OFF_BPAIR, i);
      const u32 ra = S.lpar(e & 0xFFFFu), rb = S.lpar(e >> 16);
      if (ra != rb) continue;
      if (root >= 0 && root != (int)ra) {
        err |= TC_ERR_INTERNAL;
        return 0;
      }
      root = (int)ra;
    }
    if (root < 0) {
      err |= TC_ERR_INTERNAL;
      return 0;
    }
  }
  // 3. the tree hanging from region 0: parent(r) = region of cand(smallest label of r)
  for (u32 r = 0; r < R; ++r) S.word(K::OFF_ADJ, r) = 0;
  u32 internal = 0;
  for (u32 r = 1; r < R; ++r) {
    const u32 c = S.cand(*S.byte(K::OFF_RLAB, r)) & TcScratch<K>::LOW;
    if (c == TcScratch<K>::NONE) {
      err |= TC_ERR_INTERNAL;
      return 0;
    }
    const u32 p = S.lpar(c);
    if (p >= r) {
      err |= TC_ERR_INTERNAL;
      return 0;
    }
    *S.byte(K::OFF_TPAR, r) = (u8)p;
    S.word(K::OFF_ADJ, p) |= 1u << r;
    internal |= 1u << p;
  }
  // 4. the path root -> region 0, reversed by re-rooting
  u32 k = 0, path = 1u;
  *S.byte(K::OFF_ORDER, 0) = (u8)root;
  for (u32 x = (u32)root; x != 0;) {
    x = *S.byte(K::OFF_TPAR, x);
    *S.byte(K::OFF_ORDER, ++k) = (u8)x;
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
    const code_t v = tc_concat(S, S.word(K::OFF_ADJ, x), leaves, len);
    tc_store_node(S, x, v, len);
  }
  code_t bits = 0;
  u32 nbits = 0;
  for (int i = (int)k; i >= 0; --i) {
    const u32 x = *S.byte(K::OFF_ORDER, i);
    u32 kids = S.word(K::OFF_ADJ, x);
    if (i > 0) kids &= ~(1u << *S.byte(K::OFF_ORDER, i - 1));
    if (i < (int)k) kids |= 1u << *S.byte(K::OFF_ORDER, i + 1);
    if (i > 0 && !kids) {
      leaves |= 1u << x;
      continue;
    }
    u32 len;
    const code_t v = tc_concat(S, kids, leaves, len);
    if (i > 0) {
      tc_store_node(S, x, v, len);
    } else {
      bits = v;
      nbits = len;
    }
  }
  if (nbits != 2 * (R - 1) || nbits > BITS - 2) {
    err |= TC_ERR_INTERNAL;
    return 0;
  }
  return (1ull << nbits) | (nbits ? (u64)(bits >> (BITS - nbits)) : 0ull);
}

// ------------------------------------------------------------ histogram ----

__device__ __forceinline__ u32 tc_hash_slot(u64 key, u64 mask) {
  return (u32)(((key * 0x9E3779B97F4A7C15ull) >> 32) & mask);
}

// Add cnt to key in the device hash table (open addressing, 0 = empty).
__device__ __forceinline__ void tc_global_add(u64 *gkeys, unsigned long long *gcnt, u64 gslots,
                                              u32 *gerr, u64 key, unsigned long long cnt) {
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

// Warp-aggregated insert into the block's hash table (all 32 lanes call it;
// key 0 means "nothing to add").
template <u32 HASH>
__device__ __forceinline__ void tc_hist_add(u64 key, u64 *hkeys, unsigned long long *hcnt, u64 *gkeys,
                                            unsigned long long *gcnt, u64 gslots, u32 *gerr) {
  const u32 lane = threadIdx.x & 31u;
  const unsigned peers = __match_any_sync(0xffffffffu, key);
  if (key != 0 && lane == (u32)(__ffs(peers) - 1)) {
    const unsigned long long cnt = (unsigned long long)__popc(peers);
    u32 s = tc_hash_slot(key, HASH - 1);
    for (u32 probe = 0; probe < HASH; ++probe) {
      unsigned long long *kp = reinterpret_cast<unsigned long long *>(hkeys + s);
      unsigned long long k = *reinterpret_cast<volatile unsigned long long *>(kp);
      if (k == 0) k = atomicCAS(kp, 0ull, (unsigned long long)key);
      if (k == 0 || k == key) {
        atomicAdd(hcnt + s, cnt);
        return;
      }
      s = (s + 1) & (HASH - 1);
    }
    tc_global_add(gkeys, gcnt, gslots, gerr, key, cnt);
  }
}

__device__ __forceinline__ u64 tc_splitmix64(u64 x) {
  u64 z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Enumeration masks (ts_enumerate flags): k, k << 1, k with zero bits
// inserted at positions 0, 1 and d + 1, or splitmix64(k) cut to |A| bits.
__device__ __forceinline__ u64 tc_enum_mask(u64 k, u32 flags, u32 d) {
  if (flags & 4u) {
    const u32 np = (d + 1) * (d + 2) / 2;
    return tc_splitmix64(k) & (np >= 64 ? ~0ull : ((1ull << np) - 1));
  }
  if (flags & 1u) return k << 1;
  if (flags & 2u) return ((k & ((1ull << (d - 1)) - 1)) << 2) | ((k >> (d - 1)) << (d + 2));
  return k;
}
