// tc_warp_sweep.cuh -- Algorithm 1 for one sign vector by a whole warp (the
// warp-per-instance tile, TS_KERNEL_WARP).
//
// The 32 lanes of a warp work on one instance at a time, with its state in
// the warp's part of shared memory:
//   1. the signs of all diamond vertices (bit k(v) of sigma xor the Eq. 2
//      constant c(v)), one bit each;
//   2. the same-sign components of T^diamond (Alg. 1, line 3): a lock-free
//      union-find over the edges, spread over the lanes, that always hooks
//      the larger root under the smaller (so every component's root is its
//      smallest vertex in sweep order);
//   3. the regions (Alg. 1, line 4): the 2d antipodal pairs join the
//      components with orientation parity 1 (one lane; an inconsistent join
//      marks the odd cycle of the non-orientable region, proof of Thm. 2);
//   4. regions numbered in the order of their smallest vertex; the region
//      tree from each region's smallest vertex s and s's first earlier
//      neighbour, which has the other sign and lies in a region with a
//      smaller number (the same argument as the label sweep's back end);
//   5. the root region (the odd cycle for even d, the pseudoline's region
//      for odd d) and the canonical code of the rooted tree (one lane, the
//      wide back end's tree code).
// Every step is a phase that each lane runs for its share, followed by a
// warp synchronisation; no phase needs another lane's registers, so a host
// build (TC_WARP_EMULATE) runs the same code for lanes 0 .. 31 in turn.
#pragma once

#include "tc_layout.h"
#include "tc_runtime.cuh"

// Traits of one warp's instance: the scratch layout (32-bit words,
// contiguous: one instance per warp) and the offsets the wide back end's
// tree code reads (THREADS = 1: no interleaving).
template <int D_>
struct TcWarpK {
  static constexpr TcLayout L = tc_layout(D_, true, 32);
  static constexpr u32 D = D_, V = L.V, NPOINTS = L.np, W = L.sw, CW = L.cw, RMAX = L.rmax,
                       WARENA = L.warena_words, THREADS = 1, LBYTES = L.lbytes,
                       VW = (L.V + 31) / 32, WB = (L.rmax + 3) / 4;
  // the tree code's region arrays (relative to OFF_TREE)
  static constexpr u32 OFF_WPAR = 0, OFF_WFC = WB, OFF_WNS = 2 * WB, OFF_WENT = 3 * WB,
                       OFF_WARENA = 3 * WB + (L.rmax / 2 + 2 + 1) / 2,
                       OFF_WTEMP = OFF_WARENA + L.warena_words,
                       TREE = OFF_WTEMP + L.warena_words, OFF_LPAR = 0, OFF_CAND = 0;
  // one warp's words (an even number, so that the u64 codes of every warp
  // are 8-byte aligned): pcode[32] (u64) | plen[32] and pdep[32] (bytes) |
  // par[V] and lnk[V] (u16) | sgn[VW] | odd[VW] | roots[VW] | rootv[RMAX] |
  // err | root | depth | tree[TREE]
  static constexpr u32 VH = (V + 1) / 2;
  static constexpr u32 OFF_PCODE = 0, OFF_PLEN = 64, OFF_PDEP = 72, OFF_PAR = 80,
                       OFF_LNK = OFF_PAR + VH, OFF_SGN = OFF_LNK + VH, OFF_ODD = OFF_SGN + VW,
                       OFF_ROOTS = OFF_ODD + VW, OFF_ROOTV = OFF_ROOTS + VW,
                       OFF_ERR = OFF_ROOTV + RMAX, OFF_ROOT = OFF_ERR + 1, OFF_DEPTH = OFF_ROOT + 1,
                       OFF_TREE = OFF_DEPTH + 1, WORDS = (OFF_TREE + TREE + 1) & ~1u;
};

// A phase of the warp: each lane runs f(lane) for its share, then the warp
// synchronises (its shared-memory writes are then visible to every lane).
#ifdef TC_WARP_EMULATE
// host build: the lanes run one after another, in reverse order when
// tc_emu_reverse is set (no phase may depend on the order)
static bool tc_emu_reverse = false;
template <class F>
inline void tc_lanes(F f) {
  for (u32 l = 0; l < 32; ++l) f(tc_emu_reverse ? 31u - l : l);
}
inline u32 tc_lane_cas(u16 *p, u32 cmp, u32 val) {
  const u32 o = *p;
  if (o == cmp) *p = (u16)val;
  return o;
}
inline void tc_lane_or(u32 *p, u32 v) { *p |= v; }
inline void tc_warp_sync() {}
inline bool tc_warp_any(bool b) { return b; }  // each lane loops until its own work is done
inline void tc_lane_max(u32 *p, u32 v) { *p = *p > v ? *p : v; }
// a per-lane value that lives across phases (one per lane on the host)
template <class T>
struct TcLaneVar {
  T v[32];
  T &operator()(u32 lane) { return v[lane]; }
};
// bit `lane` of *w (zeroed before) from every lane's b
inline void tc_lane_bits(u32 *w, u32 lane, bool b) {
  if (b) *w |= 1u << lane;
}
#else
template <class F>
__device__ __forceinline__ void tc_lanes(F f) {
  f(threadIdx.x & 31u);
  __syncwarp();
}
__device__ __forceinline__ u32 tc_lane_cas(u16 *p, u32 cmp, u32 val) {
  return atomicCAS(reinterpret_cast<unsigned short *>(p), (unsigned short)cmp, (unsigned short)val);
}
__device__ __forceinline__ void tc_lane_or(u32 *p, u32 v) { atomicOr(p, v); }
// Reconvergence point inside a phase (all lanes run the same number of steps).
__device__ __forceinline__ void tc_warp_sync() { __syncwarp(); }
// Loop condition of a lock-step loop: true while any lane has work left.
__device__ __forceinline__ bool tc_warp_any(bool b) { return __any_sync(0xffffffffu, b) != 0; }
__device__ __forceinline__ void tc_lane_max(u32 *p, u32 v) { atomicMax(p, v); }
template <class T>
struct TcLaneVar {
  T v;
  __device__ __forceinline__ T &operator()(u32) { return v; }
};
// Bit `lane` of *w from every lane's b (one ballot; every lane calls it).
__device__ __forceinline__ void tc_lane_bits(u32 *w, u32 lane, bool b) {
  const u32 m = __ballot_sync(0xffffffffu, b);
  if (lane == 0) *w = m;
}
#endif

// The real scheme of sig (all lanes pass the same sign vector) by the warp;
// tables: wv[V], wedge[E], wanti[nanti], wbedge[nbedge] (format at
// WarpLayout in engine.h, staged in shared memory); ws: the warp's
// TcWarpK<D>::WORDS words of shared memory.  Lane 0 receives the code in
// code[0 .. CW-1] (zero on failure) and returns the error bits.
template <int D_, class SIG>
__device__ __forceinline__ u32 tc_warp_classify(const SIG &sig, const u32 *__restrict__ wv,
                                                const u32 *__restrict__ wedge, u32 E,
                                                const u32 *__restrict__ wanti, u32 nanti,
                                                const u32 *__restrict__ wbedge, u32 nbedge,
                                                u32 *ws, u64 *code) {
  typedef TcWarpK<D_> K;
  u16 *par = reinterpret_cast<u16 *>(ws + K::OFF_PAR), *lnk = reinterpret_cast<u16 *>(ws + K::OFF_LNK);
  u32 *sgn = ws + K::OFF_SGN,
      *odd = ws + K::OFF_ODD, *roots = ws + K::OFF_ROOTS, *rootv = ws + K::OFF_ROOTV,
      *errw = ws + K::OFF_ERR;
  volatile u16 *vpar = par, *vlnk = lnk;
  auto sign = [&](u32 v) { return (sgn[v >> 5] >> (v & 31u)) & 1u; };
  // root of a, halving the path on the way (a parent link only ever moves to
  // an ancestor, and only roots are hooked, so concurrent lanes agree)
  auto find = [&](u32 a) {
    for (;;) {
      const u32 p = vpar[a];
      if (p == a) return a;
      const u32 g = vpar[p];
      if (g == p) return p;
      vpar[a] = (u16)g;
      a = g;
    }
  };
  // 1. signs of the diamond vertices (lane l holds vertices 32 i + l, bit l
  //    of word i), every vertex its own component
  tc_lanes([&](u32 lane) {
    for (u32 c = lane; c < K::VW; c += 32) {
      sgn[c] = 0;
      odd[c] = 0;
      roots[c] = 0;
    }
    if (lane == 0) *errw = 0;
  });
  tc_lanes([&](u32 lane) {
    for (u32 i = 0; i < K::VW; ++i) {
      const u32 v = 32 * i + lane;
      bool s = false;
      if (v < K::V) {
        const u32 x = wv[v];
        par[v] = (u16)v;
        lnk[v] = (u16)(v << 1);
        s = (sig.bit(x & 255u) ^ ((x >> 8) & 1u)) != 0;
      }
      tc_lane_bits(sgn + i, lane, s);
    }
  });
  // 2. same-sign components, 32 vertices per step in sweep order (Alg. 1,
  //    line 3, as the label sweep takes it): the runs of v's fan entries
  //    with v's sign (a run ends at an entry of the other sign or where two
  //    entries do not span a triangle with v) are each connected already;
  //    v's parent is the root of its first run's first entry, and each later
  //    run is a join of v with its first entry, done lock-free: a hook links
  //    the larger root under the smaller and fails only when another lane
  //    hooked that root first (then both ends are found again)
  TcLaneVar<u64> starts;
  TcLaneVar<u32> fan0;
  for (u32 i = 0; i < K::VW; ++i) {
    tc_lanes([&](u32 lane) {
      const u32 v = 32 * i + lane;
      u64 st = 0;
      if (v < K::V) {
        const u32 x = wv[v], n = (x >> 9) & 127u, f0 = x >> 16, sv = sign(v);
        u32 prev = 0;
        for (u32 j = 0; j < n; ++j) {
          const u32 e = wedge[f0 + j];
          const u32 same = sign(e & 0x3FFu) == sv;
          if (same && !(prev && ((e >> 15) & 1u))) st |= 1ull << j;
          prev = same;
        }
        if (st) {
          vpar[v] = (u16)find(wedge[f0 + __ffsll(st) - 1] & 0x3FFu);
          st &= st - 1;
        }
        fan0(lane) = f0;
      }
      starts(lane) = st;
    });
    tc_lanes([&](u32 lane) {
      const u32 v = 32 * i + lane;
      u64 &st = starts(lane);
      while (tc_warp_any(st != 0)) {
        if (st == 0) continue;
        const u32 j = __ffsll(st) - 1;
        st &= st - 1;
        u32 a = v, b = wedge[fan0(lane) + j] & 0x3FFu;
        for (u32 it = 0;; ++it) {
          a = find(a);
          b = find(b);
          if (a == b) break;
          const u32 hi = a > b ? a : b, lo = a > b ? b : a;
          if (tc_lane_cas(par + hi, hi, lo) == hi) break;
          if (it >= 4 * K::V) {  // more failed hooks than hooks there are: an internal error
            tc_lane_or(errw, TC_ERR_INTERNAL);
            break;
          }
        }
      }
    });
  }
  // 3. every vertex points at its component's root (its smallest vertex);
  //    parents are smaller, so those of earlier steps point at roots already
  tc_lanes([&](u32 lane) {
    for (u32 i = 0; i < K::VW; ++i) {
      const u32 v = 32 * i + lane;
      if (v < K::V) {
        u32 a = vpar[v];
        while (vpar[a] != a) a = vpar[a];
        vpar[v] = (u16)a;
      }
      tc_warp_sync();
    }
  });
  // 4. the antipodal pairs join components with parity 1 into regions, one
  //    pair per lane, lock-free as in step 2 on the links lnk = parent << 1 |
  //    parity (links of non-roots never change, so a path's parity is fixed
  //    while its root stays a root); a join inside one region with odd parity
  //    marks an odd cycle at the region's root of the moment (even d only;
  //    step 5 carries the marks to the final roots)
  tc_lanes([&](u32 lane) {
    u32 bad = 0;
    for (u32 i = lane; i < nanti; i += 32) {
      const u32 ab = wanti[i];
      const u32 x = par[ab & 0xFFFFu], y = par[ab >> 16];
      for (u32 it = 0;; ++it) {
        u32 a = x, b = y, pa = 0, pb = 0;
        for (u32 l = vlnk[a]; (l >> 1) != a; l = vlnk[a]) {
          pa ^= l & 1u;
          a = l >> 1;
        }
        for (u32 l = vlnk[b]; (l >> 1) != b; l = vlnk[b]) {
          pb ^= l & 1u;
          b = l >> 1;
        }
        const u32 q = (pa ^ pb ^ 1u) & 1u;
        if (a == b) {
          if (K::D % 2 == 0 && q) tc_lane_or(odd + (a >> 5), 1u << (a & 31u));
          break;
        }
        const u32 hi = a > b ? a : b, lo = a > b ? b : a;
        if (tc_lane_cas(lnk + hi, hi << 1, (lo << 1) | q) == hi << 1) break;
        if (it >= 4 * K::V) {
          bad = 1;
          break;
        }
      }
    }
    if (bad) tc_lane_or(errw, TC_ERR_INTERNAL);
  });
  // 5. every vertex points at its region's smallest vertex; those are marked
  tc_lanes([&](u32 lane) {
    for (u32 i = 0; i < K::VW; ++i) {
      const u32 v = 32 * i + lane;
      bool r = false;
      if (v < K::V) {
        u32 a = par[v];
        while ((lnk[a] >> 1) != a) a = lnk[a] >> 1;
        par[v] = (u16)a;
        r = a == v;
        if (K::D % 2 == 0 && a != v && ((odd[i] >> lane) & 1u))
          tc_lane_or(odd + (a >> 5), 1u << (a & 31u));
      }
      tc_lane_bits(roots + i, lane, r);
    }
  });
  // 6. region numbers in the order of the regions' smallest vertices: lane l
  //    holds vertices 32 i + l, so bit l of root word i, and counts the roots
  //    before it; lnk of a region's smallest vertex becomes its number
  u32 R = 0;
  tc_lanes([&](u32 lane) {
    u32 pre = 0;
    for (u32 i = 0; i < K::VW; ++i) {
      const u32 m = roots[i];
      if ((m >> lane) & 1u) {
        const u32 r = pre + __popc(m & ((1u << lane) - 1u));
        if (r < K::RMAX) {
          rootv[r] = 32 * i + lane;
          lnk[32 * i + lane] = (u16)r;
        }
      }
      pre += __popc(m);
    }
    R = pre;  // the same in every lane
  });
  const TcScratch<K> S{ws + K::OFF_TREE};
  if (R > K::RMAX) {
    tc_lanes([&](u32 lane) {
      if (lane == 0) *errw |= TC_ERR_OVERFLOW;
    });
  } else {
    // 7. the tree hanging from region 0: the parent of region r >= 1 is the
    //    region of the first earlier neighbour of r's smallest vertex (it has
    //    the other sign, and its region has a smaller vertex, so a smaller
    //    number; the edge between them crosses one oval)
    tc_lanes([&](u32 lane) {
      u32 bad = 0;
      for (u32 r = lane + 1; r < R; r += 32) {
        const u32 x = wv[rootv[r]];
        const u32 p = (x >> 9) & 127u ? lnk[par[wedge[x >> 16] & 0x3FFu]] : r;
        if (p >= r) bad = 1;
        else *S.byte(K::OFF_WPAR, r) = (u8)p;
      }
      if (bad) tc_lane_or(errw, TC_ERR_INTERNAL);
    });
  }
  // 8. the root region (one lane); for at most 32 regions the tree is then
  //    re-rooted there (the path from the root to region 0 reversed)
  constexpr u32 NONE8 = 0xFFu;
  u32 *pl = ws + K::OFF_ROOT;
  tc_lanes([&](u32 lane) {
    if (lane != 0) return;
    int root = -1;
    if (*errw == 0) {
      if constexpr (K::D % 2 == 0) {
        // the region with an odd cycle of antipodal crossings (non-orientable)
        u32 cnt = 0;
        for (u32 i = 0; i < K::VW; ++i) {
          const u32 m = odd[i] & roots[i];
          if (m && root < 0) root = (int)lnk[32 * i + __ffs(m) - 1];
          cnt += __popc(m);
        }
        if (cnt != 1) root = -1;
      } else {
        // the region on both sides of a crossed boundary edge (the pseudoline)
        for (u32 i = 0; i < nbedge; ++i) {
          const u32 e = wbedge[i], a = e & 0xFFFFu, b = e >> 16;
          if (sign(a) == sign(b) || par[a] != par[b]) continue;
          const int r = (int)lnk[par[a]];
          if (root >= 0 && root != r) {
            root = -2;
            break;
          }
          root = r;
        }
      }
      if (root < 0) *errw |= TC_ERR_INTERNAL;
    }
    pl[0] = root < 0 ? 0u : (u32)root;
    pl[1] = 0;
    if (root >= 0 && R <= 32) {
      *S.byte(K::OFF_WPAR, 0) = (u8)NONE8;
      for (u32 x = (u32)root, prev = NONE8, it = 0; it < R; ++it) {
        const u32 nx = *S.byte(K::OFF_WPAR, x);
        *S.byte(K::OFF_WPAR, x) = (u8)prev;
        if (x == 0) break;
        prev = x;
        x = nx;
      }
    }
  });
  u32 err = *errw;
  const u32 root = pl[0];
  u64 *pcode = reinterpret_cast<u64 *>(ws + K::OFF_PCODE);
  u8 *plen = reinterpret_cast<u8 *>(ws + K::OFF_PLEN), *pdep = reinterpret_cast<u8 *>(ws + K::OFF_PDEP);
  if (err || R > 32) {
    // errors, and trees of more than 32 regions: the wide back end's tree code
    tc_lanes([&](u32 lane) {
      if (lane != 0) return;
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
      if (!err) tc_wide_tree_code<K>(S, R, (int)root, err, code);
    });
    return err;
  }
  // 9. the canonical code level by level, one lane per region: every
  //    region's code is '1', its children's codes in descending order, '0'
  //    (the root's without the enclosing pair), MSB first in one word
  tc_lanes([&](u32 lane) {
    if (lane >= R) return;
    u32 dep = 0;
    for (u32 x = lane; *S.byte(K::OFF_WPAR, x) != NONE8 && dep < R; x = *S.byte(K::OFF_WPAR, x)) ++dep;
    pdep[lane] = (u8)dep;
    tc_lane_max(pl + 1, dep);
  });
  auto node_code = [&](u32 r) {
    u32 kids = 0, nleaf = 0;
    for (u32 c = 0; c < R; ++c) {
      if (*S.byte(K::OFF_WPAR, c) != r) continue;
      if (plen[c] == 2) ++nleaf;
      else kids |= 1u << c;
    }
    const bool top = r == root;
    u64 acc = top ? 0ull : 1ull << 63;
    u32 q = top ? 0u : 1u;
    while (kids) {
      u32 best = __ffs(kids) - 1;
      for (u32 m = kids & (kids - 1); m; m &= m - 1) {
        const u32 c = __ffs(m) - 1;
        if (pcode[c] > pcode[best]) best = c;
      }
      kids &= ~(1u << best);
      acc |= pcode[best] >> q;
      q += plen[best];
    }
    if (nleaf) acc |= (0xAAAAAAAAAAAAAAAAull & ~(~0ull >> (2 * nleaf))) >> q;
    q += 2 * nleaf + (top ? 0u : 1u);
    pcode[r] = acc;
    plen[r] = (u8)q;
  };
  for (u32 lev = pl[1]; lev >= 1; --lev)
    tc_lanes([&](u32 lane) {
      if (lane < R && pdep[lane] == lev) node_code(lane);
    });
  tc_lanes([&](u32 lane) {
    if (lane != 0) return;
    node_code(root);
    const u32 q = plen[root];
#pragma unroll
    for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
    if (q != 2 * (R - 1)) {
      err |= TC_ERR_INTERNAL;
      return;
    }
    code[0] = (1ull << q) | (q ? pcode[root] >> (64 - q) : 0ull);
  });
  return err;
}
