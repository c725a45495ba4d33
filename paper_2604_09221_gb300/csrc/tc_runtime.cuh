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

// Attribute of the join pass and the narrow back end: out of line by
// default (the table-driven kernels, where inlining measured 9 % slower at
// d = 7 and 23 % at d = 9); the generated specialised sources define it as
// __forceinline__ (measured faster there: the calls' register saves cost
// more than the larger code).
#ifndef TC_HEAVY_FN
#define TC_HEAVY_FN __noinline__
#endif

constexpr u32 TC_ERR_INTERNAL = 1u;
constexpr u32 TC_ERR_OVERFLOW = 2u;
constexpr u32 TC_ERR_TIMEOUT = 4u;

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
  __device__ __forceinline__ u16 *half(u32 off, u32 i) const {
    return reinterpret_cast<u16 *>(w + (off + (i >> 1)) * K::THREADS) + (i & 1u);
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

// Root of x without the parity (odd degrees, where no parity is read).
template <class K>
__device__ __forceinline__ u32 tc_find_root(const TcScratch<K> &S, u32 x) {
  u32 e = S.lpar(x);
  while ((e & TcScratch<K>::LOW) != x) {
    x = e & TcScratch<K>::LOW;
    e = S.lpar(x);
  }
  return x;
}

// Odd-cycle flags of the label sets (valid at set roots), one bit per label.
// Only even degrees read them (the non-orientable region is the root there);
// for odd d the root comes from the pseudoline, and neither flags nor the
// parities of the links are kept.
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
  if constexpr (K::D % 2 == 0) {
#pragma unroll
    for (u32 w = 0; w < K::WODD; ++w) S.word(K::OFF_ODD, w) = 0;
  }
}

// Join labels a and b with relative orientation parity p.
template <class K>
__device__ __forceinline__ void tc_unite(const TcScratch<K> &S, u32 a, u32 b, u32 p) {
  if constexpr (K::D % 2 == 1) {  // no parity, no odd flags
    const u32 ra = tc_find_root(S, a), rb = tc_find_root(S, b);
    if (ra != rb) S.set_lpar(ra < rb ? rb : ra, ra < rb ? ra : rb);
    return;
  }
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

// Point every label straight at the root of its set, with the parity of the
// whole path (one pass in label order: a parent is smaller than its child,
// so it is already flat when the child is visited; roots keep themselves).
template <class K>
__device__ __forceinline__ void tc_flatten(const TcScratch<K> &S, u32 nl) {
  for (u32 l = 0; l < nl; ++l) {
    const u32 e = S.lpar(l);
    const u32 pe = S.lpar(e & TcScratch<K>::LOW);
    S.set_lpar(l, (pe & TcScratch<K>::LOW) | ((e ^ pe) & TcScratch<K>::TOP));
  }
}

template <class K>
__device__ __forceinline__ void tc_bpair(const TcScratch<K> &S, u32 i, u32 la, u32 lb) {
  S.word(K::OFF_BPAIR, i) = la | (lb << 16);
}

// Apply the pending joins (a | b << 16 | parity << 31).
template <class K>
__device__ TC_HEAVY_FN void tc_unions(const TcScratch<K> &S, u32 np) {
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
// Region of a label after step 1 of tc_backend: labels in `skip` (below 32)
// were passed over; their parent link points straight at their root.
template <class K>
__device__ __forceinline__ u32 tc_region_of(const TcScratch<K> &S, u32 x, u32 skip) {
  const bool via_root = x < 32u && ((skip >> x) & 1u);
  return S.lpar(via_root ? (S.lpar(x) & TcScratch<K>::LOW) : x);
}

// skip: labels below 32 known not to be roots whose parent link is their
// root (the half-diamond labels of a block sweep, flattened once per warp);
// the region pass leaves them out and lookups go through their root.
template <class K>
__device__ TC_HEAVY_FN u64 tc_backend(const TcScratch<K> &S, u32 nl, u32 nb, u32 &err,
                                      u32 skip = 0u) {
  typedef typename TcCode<K::CODE64>::T code_t;
  constexpr u32 BITS = TcCode<K::CODE64>::BITS;
  // 1. region ids over lpar (label order), odd-cycle flags, smallest labels
  u32 R = 0;
  u64 odd = 0;
  auto visit = [&](u32 l) -> bool {
    const u32 p = S.lpar(l) & TcScratch<K>::LOW;
    const u32 is_root = p == l;
    const u32 rp = S.lpar(p);  // p < l holds its region id already
    if (is_root) {
      if (R >= K::RMAX) return false;
      odd |= (u64)tc_odd(S, l) << R;
      *S.byte(K::OFF_RLAB, R) = (u8)l;
    }
    S.set_lpar(l, is_root ? R : rp);
    R += is_root;
    return true;
  };
  bool fits = true;
  if (!skip) {
    for (u32 l = 0; l < nl && fits; ++l) fits = visit(l);
  } else {  // the labels below 32 not in skip, in order, then the rest
    for (u32 todo = ~skip & (nl >= 32u ? ~0u : ((1u << nl) - 1u)); todo && fits; todo &= todo - 1u)
      fits = visit(__ffs(todo) - 1u);
    for (u32 l = 32; l < nl && fits; ++l) fits = visit(l);
  }
  if (!fits) {
    err |= TC_ERR_OVERFLOW;
    return 0;
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
      const u32 ra = tc_region_of(S, e & 0xFFFFu, skip), rb = tc_region_of(S, e >> 16, skip);
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
    const u32 p = tc_region_of(S, c, skip);
    if (p >= r) {
      err |= TC_ERR_INTERNAL;
      return 0;
    }
    *S.byte(K::OFF_TPAR, r) = (u8)p;
    S.word(K::OFF_ADJ, p) |= 1u << r;
    internal |= 1u << p;
  }
  // a star around the root (every oval outermost; nine in ten random sign
  // vectors at d = 7): the code is '10' once per oval, no AHU needed
  if (!(internal & ~(1u | (1u << root))) &&
      (root == 0 || S.word(K::OFF_ADJ, 0) == (1u << root))) {
    const u32 nb2 = 2 * (R - 1);
    return (1ull << nb2) | (0xAAAAAAAAAAAAAAAAull & ((1ull << nb2) - 1));
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

// ------------------------------------------------- wide back end (d >= 10) --
//
// Up to 107 regions and 213-bit codes.  The region tree is built as in
// tc_backend, then re-rooted by reversing the parent links on the path from
// the root to region 0, and stored as first-child / next-sibling bytes.  AHU
// codes are produced in post order without a stack (parent and sibling links
// give the next node).  When a node is finished, the codes of its non-leaf
// children are the most recent entries of a packed bit arena (the codes of
// disjoint finished subtrees, 2 * (R - 1) bits at most); they are written in
// descending order behind a '1' into a build area, followed by '10' per leaf
// child and a '0', and the result replaces them in the arena.  Bit strings
// are MSB first: string bit p is bit 31 - p % 32 of word p / 32.

template <class K>
__device__ __forceinline__ u64 tc_get64(const TcScratch<K> &S, u32 off, u32 p) {
  const u32 w = p >> 5, sh = p & 31u;
  const u64 hi = ((u64)S.word(off, w) << 32) | S.word(off, w + 1);
  return sh ? (hi << sh) | (S.word(off, w + 2) >> (32u - sh)) : hi;
}

// OR the 64-bit MSB-first chunk x into the bit string at position q.
template <class K>
__device__ __forceinline__ void tc_or64(const TcScratch<K> &S, u32 off, u32 q, u64 x) {
  const u32 w = q >> 5, sh = q & 31u;
  S.word(off, w) |= (u32)(x >> (32u + sh));
  S.word(off, w + 1) |= (u32)(x >> sh);
  if (sh) S.word(off, w + 2) |= (u32)(x << (32u - sh));
}

// Append n bits starting at position p of one string at position q of another.
template <class K>
__device__ __forceinline__ void tc_append(const TcScratch<K> &S, u32 src, u32 p, u32 n, u32 dst,
                                          u32 q) {
  for (u32 i = 0; i < n; i += 64) {
    u64 x = tc_get64(S, src, p + i);
    if (n - i < 64) x &= ~0ull << (64 - (n - i));
    tc_or64(S, dst, q + i, x);
  }
}

// Lexicographic comparison of two codes (prefix-free, so equal over the
// shorter length means equal).
template <class K>
__device__ __forceinline__ int tc_cmp(const TcScratch<K> &S, u32 off, u32 pa, u32 la, u32 pb,
                                      u32 lb) {
  const u32 n = la < lb ? la : lb;
  for (u32 i = 0; i < n; i += 64) {
    u64 a = tc_get64(S, off, pa + i), b = tc_get64(S, off, pb + i);
    if (n - i < 64) {
      const u64 mk = ~0ull << (64 - (n - i));
      a &= mk;
      b &= mk;
    }
    if (a != b) return a > b ? 1 : -1;
  }
  return 0;
}

// The canonical code of a region tree (wide back end, steps after the
// parents): on entry wpar[r] (r = 1 .. R-1) is the parent of region r in the
// tree hanging from region 0 (parent(r) < r) and root is the region the tree
// is rooted at (the non-orientable region, or the pseudoline's); re-roots
// the tree there, builds first-child / next-sibling links and writes the
// AHU code of the rooted tree to code[0 .. CW-1] (all zero and err set on
// failure).  Shared by tc_backend_wide and the warp-per-instance kernels.
template <class K>
__device__ __noinline__ void tc_wide_tree_code(const TcScratch<K> &S, u32 R, int root, u32 &err,
                                               u64 *code) {
  constexpr u32 NONE8 = 0xFFu, ENT_CAP = K::RMAX / 2 + 2, ABITS = 32 * (K::WARENA - 3);
#pragma unroll
  for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
  *S.byte(K::OFF_WPAR, 0) = (u8)NONE8;
  for (u32 x = (u32)root, prev = NONE8, it = 0; it < R; ++it) {
    const u32 nx = *S.byte(K::OFF_WPAR, x);
    *S.byte(K::OFF_WPAR, x) = (u8)prev;
    if (x == 0) break;
    prev = x;
    x = nx;
  }
  for (u32 r = 0; r < R; ++r) *S.byte(K::OFF_WFC, r) = (u8)NONE8;
  for (u32 r = 0; r < R; ++r) {
    const u32 p = *S.byte(K::OFF_WPAR, r);
    if (p == NONE8) continue;
    *S.byte(K::OFF_WNS, r) = *S.byte(K::OFF_WFC, p);
    *S.byte(K::OFF_WFC, p) = (u8)r;
  }
  // a star around the root (every oval outermost): '10' once per oval
  bool star = true;
  for (u32 r = 0; r < R; ++r) star &= r == (u32)root || *S.byte(K::OFF_WFC, r) == NONE8;
  if (star) {
    const u32 q = 2 * (R - 1);
#pragma unroll
    for (u32 j = 0; j < K::CW; ++j) {
      const int left = (int)q - 64 * (int)j;  // pattern bits in this word
      code[j] = left >= 64 ? 0xAAAAAAAAAAAAAAAAull
                           : (left > 0 ? 0xAAAAAAAAAAAAAAAAull & ((1ull << left) - 1) : 0ull);
    }
    code[q >> 6] |= 1ull << (q & 63u);
    return;
  }
  // 4. AHU in post order
  u32 top = 0, aend = 0, qroot = 0;
  u32 x = (u32)root;
  for (u32 it = 0; it < R && *S.byte(K::OFF_WFC, x) != NONE8; ++it) x = *S.byte(K::OFF_WFC, x);
  for (u32 it = 0; it < R; ++it) {
    if (*S.byte(K::OFF_WFC, x) != NONE8) {
      u32 k = 0, nleaf = 0;
      for (u32 c = *S.byte(K::OFF_WFC, x); c != NONE8; c = *S.byte(K::OFF_WNS, c)) {
        if (*S.byte(K::OFF_WFC, c) == NONE8) ++nleaf;
        else ++k;
      }
      if (k > top || k > 63) {
        err |= TC_ERR_INTERNAL;
        return;
      }
      const u32 first = top - k;
      const u32 start = k ? *S.half(K::OFF_WENT, first) : aend;
      const bool is_root = x == (u32)root;
#pragma unroll
      for (u32 w = 0; w < K::WARENA; ++w) S.word(K::OFF_WTEMP, w) = 0;
      u32 q = 0;
      if (!is_root) {
        tc_or64(S, K::OFF_WTEMP, 0, 1ull << 63);
        q = 1;
      }
      u64 used = 0;
      for (u32 s = 0; s < k; ++s) {
        u32 best = 0, bp = 0, bl = 0;
        bool have = false;
        for (u32 i = 0; i < k; ++i) {
          if ((used >> i) & 1ull) continue;
          const u32 p = *S.half(K::OFF_WENT, first + i);
          const u32 l = (first + i + 1 < top ? (u32)*S.half(K::OFF_WENT, first + i + 1) : aend) - p;
          if (!have || tc_cmp(S, K::OFF_WARENA, p, l, bp, bl) > 0) {
            best = i;
            bp = p;
            bl = l;
            have = true;
          }
        }
        used |= 1ull << best;
        if (q + bl > ABITS) {
          err |= TC_ERR_OVERFLOW;
          return;
        }
        tc_append(S, K::OFF_WARENA, bp, bl, K::OFF_WTEMP, q);
        q += bl;
      }
      if (q + 2 * nleaf + 1 > ABITS) {
        err |= TC_ERR_OVERFLOW;
        return;
      }
      for (u32 i = 0; i < nleaf; i += 32) {
        const u32 m = nleaf - i < 32 ? nleaf - i : 32;
        u64 pat = 0xAAAAAAAAAAAAAAAAull;
        if (m < 32) pat &= ~0ull << (64 - 2 * m);
        tc_or64(S, K::OFF_WTEMP, q, pat);
        q += 2 * m;
      }
      if (is_root) {
        qroot = q;
        break;
      }
      q += 1;  // the closing '0'
      if (start + q > ABITS || first >= ENT_CAP) {
        err |= TC_ERR_OVERFLOW;
        return;
      }
      // the children's codes are dead: overwrite them with the node's code
      const u32 w0 = start >> 5, sh = start & 31u;
      S.word(K::OFF_WARENA, w0) &= sh ? ~(0xFFFFFFFFu >> sh) : 0u;
      for (u32 w = w0 + 1; w < K::WARENA; ++w) S.word(K::OFF_WARENA, w) = 0;
      tc_append(S, K::OFF_WTEMP, 0, q, K::OFF_WARENA, start);
      *S.half(K::OFF_WENT, first) = (u16)start;
      top = first + 1;
      aend = start + q;
    }
    if (x == (u32)root) break;
    if (*S.byte(K::OFF_WNS, x) != NONE8) {
      x = *S.byte(K::OFF_WNS, x);
      for (u32 j = 0; j < R && *S.byte(K::OFF_WFC, x) != NONE8; ++j) x = *S.byte(K::OFF_WFC, x);
    } else {
      x = *S.byte(K::OFF_WPAR, x);
    }
  }
  // 5. code = (1 << nbits) | bits, little-endian words
  if (qroot != 2 * (R - 1) || qroot + 1 > 64 * K::CW) {
    err |= TC_ERR_INTERNAL;
    return;
  }
#pragma unroll
  for (u32 j = 0; j < K::CW; ++j) {
    const int hiend = (int)qroot - 64 * (int)j;  // end of this word's bits in the string
    if (hiend >= 64) code[j] = tc_get64(S, K::OFF_WTEMP, (u32)(hiend - 64));
    else if (hiend > 0) code[j] = tc_get64(S, K::OFF_WTEMP, 0) >> (64 - hiend);
  }
  code[qroot >> 6] |= 1ull << (qroot & 63u);
}

template <class K>
__device__ __noinline__ void tc_backend_wide(const TcScratch<K> &S, u32 nl, u32 nb, u32 &err,
                                             u64 *code) {
  constexpr u32 NONE8 = 0xFFu;
  typedef TcScratch<K> TS;
#pragma unroll
  for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
  // 1. region ids over lpar (label order), root flags, smallest labels
  u32 R = 0, nodd = 0;
  int root = -1;
  for (u32 l = 0; l < nl; ++l) {
    const u32 p = S.lpar(l) & TS::LOW;
    const u32 is_root = p == l;
    const u32 rp = S.lpar(p);
    if (is_root) {
      if (R >= K::RMAX) {
        err |= TC_ERR_OVERFLOW;
        return;
      }
      if (K::D % 2 == 0 && tc_odd(S, l)) {
        ++nodd;
        root = (int)R;
      }
      *S.half(K::OFF_RLAB, R) = (u16)l;
    }
    S.set_lpar(l, is_root ? R : rp);
    R += is_root;
  }
  // 2. root
  if (K::D % 2 == 0) {
    if (nodd != 1) {
      err |= TC_ERR_INTERNAL;
      return;
    }
  } else {
    for (u32 i = 0; i < nb; ++i) {
      const u32 e = S.word(K::OFF_BPAIR, i);
      const u32 ra = S.lpar(e & 0xFFFFu), rb = S.lpar(e >> 16);
      if (ra != rb) continue;
      if (root >= 0 && root != (int)ra) {
        err |= TC_ERR_INTERNAL;
        return;
      }
      root = (int)ra;
    }
    if (root < 0) {
      err |= TC_ERR_INTERNAL;
      return;
    }
  }
  // 3. the tree hanging from region 0 (parent(r) < r), then re-rooted
  *S.byte(K::OFF_WPAR, 0) = (u8)NONE8;
  for (u32 r = 1; r < R; ++r) {
    const u32 c = S.cand(*S.half(K::OFF_RLAB, r)) & TS::LOW;
    if (c == TS::NONE) {
      err |= TC_ERR_INTERNAL;
      return;
    }
    const u32 p = S.lpar(c);
    if (p >= r) {
      err |= TC_ERR_INTERNAL;
      return;
    }
    *S.byte(K::OFF_WPAR, r) = (u8)p;
  }
  tc_wide_tree_code(S, R, root, err, code);
}

// ------------------------------------------------ table-driven sweep ----
//
// The triangulation tables of host.cpp (32-bit words, vertices in the sweep
// order of T^diamond; a vertex's label lives in a label slot, reused once no
// later vertex reads it, so the sweep touches only the slots live at once):
//   vdesc[V]  bits 0-7 lattice index k(v), bit 8 Eq. 2 parity constant c(v)
//             (sign(v) = sigma_k ^ c), bits 9-15 fan length m, bits 16-25
//             v's label slot, bit 26 "vext[v] is not empty"; v's fan
//             entries follow those of v - 1
//   fan[NF]   bits 0-9 label slot of the earlier neighbour u, bits 10-17
//             k(u), bit 18 c(u), bit 19 "u and the previous entry span a
//             triangle with v"
//   vext[V]   bits 0-9 the label slot of the antipodal partner x < v of v,
//             bits 10-19 and 20-29 those of the other end b < v of up to two
//             boundary edges kept for root detection (1023: none), bit 30
//             "apply the pending joins before v" (a static schedule from the
//             most joins each vertex can push, the same in every instance)
#define TC_TAB_NONE 1023u

// Sweep vertices [v0, v1) (Alg. 1, lines 3-4): every vertex takes the label
// of its first same-sign earlier neighbour, or a fresh label; joins (several
// same-sign runs in a vertex's fan, antipodal pairs) are appended to the
// join list (applied where the tables' schedule says); crossed boundary edges are
// kept for the root of odd degree.  SIG provides bit(k); labels of the
// vertices are stored in the scratch's [lab] region with the vertex's sign in
// the top bit (labels need at most 15 of 16 / 7 of 8 bits), so a fan entry
// reads its neighbour's label and sign in one load.
// Byte offset of label slot i from a thread's word 0 (slots interleaved by
// word across `threads` threads, epw labels of lbytes bytes per word).
__device__ __forceinline__ u32 tc_slot_offset(u32 i, u32 epw, u32 lbytes, u32 threads) {
  return (i / epw) * threads * 4u + (i % epw) * lbytes;
}

// Rewrite staged fan entries (nf of them) for OFF sweeps: bits 0..18 (label
// slot, k(u), c(u), which the sweep does not read) become the byte offset of
// the neighbour's label slot; the link bit (19) stays.  Called by the
// threads [t, t + stride) of a block right after staging, before a barrier.
__device__ __forceinline__ void tc_fan_to_offsets(u32 *fan, u32 nf, u32 epw, u32 lbytes,
                                                  u32 threads, u32 t, u32 stride) {
  for (u32 i = t; i < nf; i += stride) {
    const u32 f = fan[i];
    fan[i] = (f & ~0x7FFFFu) | tc_slot_offset(f & 1023u, epw, lbytes, threads);
  }
}

// lw: word 0 of this thread's label slots, word i at lw[i * THREADS] (by
// default the scratch's [lab] region; a kernel may keep them in shared
// memory while the rest of the scratch is in global memory).  OFF: the fan
// entries carry byte offsets of their slots (tc_fan_to_offsets), so a fan
// entry finds its neighbour's label with one mask and one add.
template <class K, bool OFF = false, class SIG>
__device__ __forceinline__ void tc_sweep_table(const SIG &sig, const u32 *__restrict__ vdesc,
                                               const u32 *__restrict__ fan,
                                               const u32 *__restrict__ vext, u32 v0, u32 v1,
                                               const TcScratch<K> &S, u32 *lw, u32 &nl, u32 &nb,
                                               u32 &np) {
  typedef TcScratch<K> TS;
  auto slot = [&](u32 i) -> typename TS::lab_t * {
    return reinterpret_cast<typename TS::lab_t *>(lw + (i / TS::EPW) * K::THREADS) + (i % TS::EPW);
  };
  // the label slot a fan entry names
  auto fslot = [&](u32 f) -> typename TS::lab_t * {
    if constexpr (OFF)
      return reinterpret_cast<typename TS::lab_t *>(reinterpret_cast<u8 *>(lw) + (f & 0x7FFFFu));
    else
      return slot(f & 1023u);
  };
  u32 fs = 0;  // the first fan entry of v: fans are stored in sweep order
  for (u32 v = 0; v < v0; ++v) fs += (vdesc[v] >> 9) & 127u;
  for (u32 v = v0; v < v1; ++v) {
    const u32 desc = vdesc[v];
    const u32 sv = sig.bit(desc & 255u) ^ ((desc >> 8) & 1u);
    const u32 m = (desc >> 9) & 127u;
    const bool ext = (desc >> 26) & 1u;  // warp-uniform: most vertices are interior
    const u32 x = ext ? vext[v] : TC_TAB_NONE | (TC_TAB_NONE << 10) | (TC_TAB_NONE << 20);
    if (ext && ((x >> 30) & 1u)) {  // the schedule's flush: the same vertex in every lane
      tc_unions(S, np);
      np = 0;
    }
    constexpr u32 SB = 8u * K::LBYTES - 1u;  // the sign bit of a [lab] entry
    u32 lv = 0, any = 0, prev = 0;
    // one fan entry: its label and sign from the entry's label slot
    auto entry = [&](u32 f, u32 raw) {
      const u32 lu = raw & TS::LOW;
      const u32 e = (raw >> SB) ^ sv ^ 1u;
      const u32 st = e & ~(((f >> 19) & 1u) & prev) & 1u;  // e starts a run of the fan
      // a run after the first: join its label with the vertex's label
      // (a predicated store: no branch, and no write when nothing joins)
      if (st & any) S.word(K::OFF_PEND, np) = lv | (lu << 16);
      np += st & any;
      lv = any ? lv : (st ? lu : lv);
      any |= st;
      prev = e;
    };
    // from d = 12 (scratch-latency-bound) the first four entries' labels are
    // loaded before any is used, so the loads overlap (m is the same in every
    // lane); at lower degrees the extra registers cost more than that gains
    constexpr u32 PRE = K::D >= 12 ? 4u : 0u;
    u32 fpre[PRE > 0 ? PRE : 1], rpre[PRE > 0 ? PRE : 1];
#pragma unroll
    for (u32 i = 0; i < PRE; ++i)
      if (i < m) {
        fpre[i] = fan[fs + i];
        rpre[i] = *fslot(fpre[i]);
      }
#pragma unroll
    for (u32 i = 0; i < PRE; ++i)
      if (i < m) entry(fpre[i], rpre[i]);
    for (u32 i = PRE; i < m; ++i) {
      const u32 f = fan[fs + i];
      entry(f, *fslot(f));
    }
    if (!any) {  // a fresh label; its cand is the label of the first fan entry
      const u32 l0 = m == 0 ? TS::NONE
                            : ((PRE > 0 ? rpre[0] : (u32)*fslot(fan[fs])) & TS::LOW);
      lv = nl;
      tc_newlab(S, nl, l0);
      ++nl;
    }
    *slot((desc >> 16) & 1023u) = (typename TS::lab_t)(lv | (sv << SB));
    fs += m;
    if (!ext) continue;
    if ((x & 1023u) != TC_TAB_NONE) {  // the antipodal partner, reached earlier
      S.word(K::OFF_PEND, np) =
          ((u32)*slot(x & 1023u) & TS::LOW) | (lv << 16) | 0x80000000u;
      ++np;
    }
    if (K::D % 2) {  // crossed boundary edges, for the pseudoline's region
#pragma unroll
      for (u32 sh = 10; sh <= 20; sh += 10) {
        const u32 b = (x >> sh) & 1023u;
        if (b == TC_TAB_NONE) continue;
        const u32 rb = *slot(b);
        if ((rb >> SB) != sv) {
          tc_bpair(S, nb, rb & TS::LOW, lv);
          ++nb;
        }
      }
    }
  }
}

// The same with the label slots in the scratch's [lab] region.
template <class K, class SIG>
__device__ __forceinline__ void tc_sweep_table(const SIG &sig, const u32 *__restrict__ vdesc,
                                               const u32 *__restrict__ fan,
                                               const u32 *__restrict__ vext, u32 v0, u32 v1,
                                               const TcScratch<K> &S, u32 &nl, u32 &nb, u32 &np) {
  tc_sweep_table<K, false>(sig, vdesc, fan, vext, v0, v1, S, S.w + K::OFF_LAB * K::THREADS, nl,
                           nb, np);
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

// Multi-word keys (d >= 10).  A slot's count word carries two flags: BUSY
// while the inserting thread writes the key, READY once it is published
// (keys: slots x CW words, zero = empty).
#define TC_SLOT_BUSY (1ull << 62)
#define TC_SLOT_READY (1ull << 63)

template <u32 CW>
__device__ __forceinline__ u64 tc_key_hash(const u64 *key) {
  u64 h = key[0];
#pragma unroll
  for (u32 w = 1; w < CW; ++w) h = (h ^ key[w]) * 0x9E3779B97F4A7C15ull + w;
  return h;
}

template <u32 CW>
__device__ void tc_global_add_wide(u64 *gkeys, unsigned long long *gcnt, u64 gslots, u32 *gerr,
                                   const u64 *key, unsigned long long cnt) {
  const u64 mask = gslots - 1;
  u64 s = tc_hash_slot(tc_key_hash<CW>(key), mask);
  for (u64 probe = 0; probe < gslots; ++probe) {
    unsigned long long *cp = gcnt + s;
    unsigned long long c = *reinterpret_cast<volatile unsigned long long *>(cp);
    if (c == 0) {
      c = atomicCAS(cp, 0ull, (unsigned long long)TC_SLOT_BUSY);
      if (c == 0) {
#pragma unroll
        for (u32 w = 0; w < CW; ++w) gkeys[s * CW + w] = key[w];
        __threadfence();
        atomicAdd(cp, (unsigned long long)(TC_SLOT_READY - TC_SLOT_BUSY) + cnt);
        return;
      }
    }
    for (u32 it = 0; !(c & TC_SLOT_READY) && it < (1u << 20); ++it) {  // bounded wait
      __nanosleep(64);
      c = *reinterpret_cast<volatile unsigned long long *>(cp);
    }
    if (!(c & TC_SLOT_READY)) {
      atomicOr(gerr, TC_ERR_TIMEOUT);
      return;
    }
    __threadfence();
    bool eq = true;
#pragma unroll
    for (u32 w = 0; w < CW; ++w)
      eq &= *reinterpret_cast<volatile u64 *>(gkeys + s * CW + w) == key[w];
    if (eq) {
      atomicAdd(cp, cnt);
      return;
    }
    s = (s + 1) & mask;
  }
  atomicOr(gerr, TC_ERR_OVERFLOW);
}

// Warp-aggregated insert of multi-word keys (all 32 lanes call it; an
// all-zero key means "nothing to add").
template <u32 CW>
__device__ __forceinline__ void tc_hist_add_wide(const u64 *key, u64 *gkeys, unsigned long long *gcnt,
                                                 u64 gslots, u32 *gerr) {
  const u32 lane = threadIdx.x & 31u;
  unsigned peers = 0xffffffffu;
  bool nz = false;
#pragma unroll
  for (u32 w = 0; w < CW; ++w) {
    peers &= __match_any_sync(0xffffffffu, key[w]);
    nz |= key[w] != 0;
  }
  if (nz && lane == (u32)(__ffs(peers) - 1))
    tc_global_add_wide<CW>(gkeys, gcnt, gslots, gerr, key, (unsigned long long)__popc(peers));
}

// ---------------------------------------------------------- sign vectors ----

// A sign vector of W words (bit k of word k / 64 is sigma at lattice index k).
template <u32 W>
struct TcSig {
  u64 w[W];
  __device__ __forceinline__ u32 bit(u32 k) const {
    u64 x = w[0];
#pragma unroll
    for (u32 i = 1; i < W; ++i) x = (k >> 6) == i ? w[i] : x;
    return (u32)(x >> (k & 63u)) & 1u;
  }
};

// Mask of the top word of a sign vector of np points.
__device__ __forceinline__ u64 tc_top_mask(u32 np, u32 W) {
  const u32 r = np - 64 * (W - 1);
  return r >= 64 ? ~0ull : ((1ull << r) - 1);
}

// Enumeration masks (ts_enumerate flags): k, k << 1, k with zero bits
// inserted at positions 0, 1 and d + 1, or splitmix64(k) cut to |A| bits.
// x with a zero bit inserted at position p (higher bits move up one).
__device__ __forceinline__ u64 tc_ins0(u64 x, u32 p) {
  return ((x >> p) << (p + 1)) | (x & ((1ull << p) - 1));
}

// The orbit sweep's high part of block u: zeros inserted at the pivots p2 <
// p1 (bits 8-15 and 16-23 of flags hold p1 and p2, set by the host).
__device__ __forceinline__ u64 tc_orbit_high(u64 u, u32 flags) {
  return tc_ins0(tc_ins0(u, (flags >> 16) & 0xFFu), (flags >> 8) & 0xFFu);
}

__device__ __forceinline__ u64 tc_enum_mask(u64 k, u32 flags, u32 d) {
  if (flags & 4u) {
    const u32 np = (d + 1) * (d + 2) / 2;
    return tc_splitmix64(k) & (np >= 64 ? ~0ull : ((1ull << np) - 1));
  }
  if (flags & 1u) return k << 1;
  if (flags & 2u) return ((k & ((1ull << (d - 1)) - 1)) << 2) | ((k >> (d - 1)) << (d + 2));
  if (flags & 8u)  // orbit sweep: every middle-row pattern, high part from the block index
    return (tc_orbit_high(k >> (d + 1), flags) << (d + 2)) | (k & ((1ull << (d + 1)) - 1));
  return k;
}

// Enumeration sign vectors of W words: as tc_enum_mask, with the bits that
// leave the first word carried into the second; splitmix64 fills word w of
// counter k with splitmix64(k * W + w).
template <u32 W>
__device__ __forceinline__ TcSig<W> tc_enum_sig(u64 k, u32 flags, u32 d) {
  TcSig<W> s;
  const u32 np = (d + 1) * (d + 2) / 2;
  if (flags & 4u) {
#pragma unroll
    for (u32 w = 0; w < W; ++w) s.w[w] = tc_splitmix64(k * W + w);
    s.w[W - 1] &= tc_top_mask(np, W);
    return s;
  }
  u64 lo = k, hi = 0;
  if (flags & 1u) {
    lo = k << 1;
    hi = k >> 63;
  } else if (flags & 2u) {
    const u64 h = k >> (d - 1);
    lo = ((k & ((1ull << (d - 1)) - 1)) << 2) | (h << (d + 2));
    hi = h >> (62 - d);
  } else if (flags & 8u) {  // one sign word only (d <= 9)
    lo = tc_enum_mask(k, flags, d);
  }
  s.w[0] = lo;
#pragma unroll
  for (u32 w = 1; w < W; ++w) s.w[w] = w == 1 ? hi : 0ull;
  return s;
}
