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
  // one warp's words: par[V] | lnk[V] | sgn[VW] | odd[VW] | roots[VW] |
  // rootv[RMAX] | err | tree[TREE]
  static constexpr u32 OFF_PAR = 0, OFF_LNK = V, OFF_SGN = 2 * V, OFF_ODD = OFF_SGN + VW,
                       OFF_ROOTS = OFF_ODD + VW, OFF_ROOTV = OFF_ROOTS + VW,
                       OFF_ERR = OFF_ROOTV + RMAX, OFF_TREE = OFF_ERR + 1,
                       WORDS = OFF_TREE + TREE;
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
inline u32 tc_lane_cas(u32 *p, u32 cmp, u32 val) {
  const u32 o = *p;
  if (o == cmp) *p = val;
  return o;
}
inline void tc_lane_or(u32 *p, u32 v) { *p |= v; }
#else
template <class F>
__device__ __forceinline__ void tc_lanes(F f) {
  f(threadIdx.x & 31u);
  __syncwarp();
}
__device__ __forceinline__ u32 tc_lane_cas(u32 *p, u32 cmp, u32 val) { return atomicCAS(p, cmp, val); }
__device__ __forceinline__ void tc_lane_or(u32 *p, u32 v) { atomicOr(p, v); }
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
  u32 *par = ws + K::OFF_PAR, *lnk = ws + K::OFF_LNK, *sgn = ws + K::OFF_SGN,
      *odd = ws + K::OFF_ODD, *roots = ws + K::OFF_ROOTS, *rootv = ws + K::OFF_ROOTV,
      *errw = ws + K::OFF_ERR;
  volatile u32 *vpar = par;
  auto sign = [&](u32 v) { return (sgn[v >> 5] >> (v & 31u)) & 1u; };
  // 1. signs of the diamond vertices, every vertex its own component
  tc_lanes([&](u32 lane) {
    for (u32 c = lane; c < K::VW; c += 32) {
      sgn[c] = 0;
      odd[c] = 0;
      roots[c] = 0;
    }
    if (lane == 0) *errw = 0;
  });
  tc_lanes([&](u32 lane) {
    for (u32 v = lane; v < K::V; v += 32) {
      const u32 x = wv[v];
      par[v] = v;
      lnk[v] = v << 1;
      if (sig.bit(x & 255u) ^ ((x >> 8) & 1u)) tc_lane_or(sgn + (v >> 5), 1u << (v & 31u));
    }
  });
  // 2. same-sign components: the lanes take the edges in turn; a hook links
  //    the larger root under the smaller and fails only when another lane
  //    hooked that root first (then both ends are found again)
  tc_lanes([&](u32 lane) {
    u32 bad = 0;
    for (u32 e = lane; e < E; e += 32) {
      const u32 uv = wedge[e];
      u32 a = uv & 0xFFFFu, b = uv >> 16;
      if (sign(a) != sign(b)) continue;
      for (u32 it = 0;; ++it) {
        while (vpar[a] != a) a = vpar[a];  // parents only decrease: this ends
        while (vpar[b] != b) b = vpar[b];
        if (a == b) break;
        const u32 hi = a > b ? a : b, lo = a > b ? b : a;
        if (tc_lane_cas(par + hi, hi, lo) == hi) break;
        if (it >= 4 * K::V) {  // more failed hooks than hooks there are: an internal error
          bad = 1;
          break;
        }
      }
    }
    if (bad) tc_lane_or(errw, TC_ERR_INTERNAL);
  });
  // 3. every vertex points at its component's root (its smallest vertex)
  tc_lanes([&](u32 lane) {
    for (u32 v = lane; v < K::V; v += 32) {
      u32 a = v;
      while (vpar[a] != a) a = vpar[a];
      par[v] = a;
    }
  });
  // 4. the antipodal pairs join components with parity 1 into regions (one
  //    lane); an inconsistent join marks an odd cycle (read for even d only)
  tc_lanes([&](u32 lane) {
    if (lane != 0) return;
    for (u32 i = 0; i < nanti; ++i) {
      const u32 ab = wanti[i];
      u32 a = par[ab & 0xFFFFu], b = par[ab >> 16], pa = 0, pb = 0;
      while ((lnk[a] >> 1) != a) {
        pa ^= lnk[a] & 1u;
        a = lnk[a] >> 1;
      }
      while ((lnk[b] >> 1) != b) {
        pb ^= lnk[b] & 1u;
        b = lnk[b] >> 1;
      }
      const u32 q = (pa ^ pb ^ 1u) & 1u;
      if (a == b) {
        if (K::D % 2 == 0 && q) odd[a >> 5] |= 1u << (a & 31u);
        continue;
      }
      const u32 hi = a > b ? a : b, lo = a > b ? b : a;
      lnk[hi] = (lo << 1) | q;
      if (K::D % 2 == 0 && ((odd[hi >> 5] >> (hi & 31u)) & 1u)) odd[lo >> 5] |= 1u << (lo & 31u);
    }
  });
  // 5. every vertex points at its region's smallest vertex; those are marked
  tc_lanes([&](u32 lane) {
    for (u32 v = lane; v < K::V; v += 32) {
      u32 a = par[v];
      while ((lnk[a] >> 1) != a) a = lnk[a] >> 1;
      par[v] = a;
      if (a == v) tc_lane_or(roots + (v >> 5), 1u << (v & 31u));
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
          lnk[32 * i + lane] = r;
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
        const u32 u = (wv[rootv[r]] >> 9) & 1023u;
        const u32 p = u < K::V ? lnk[par[u]] : r;
        if (p >= r) bad = 1;
        else *S.byte(K::OFF_WPAR, r) = (u8)p;
      }
      if (bad) tc_lane_or(errw, TC_ERR_INTERNAL);
    });
  }
  // 8.-9. the root region and the code of the rooted tree (one lane)
  u32 err = 0;
  tc_lanes([&](u32 lane) {
    if (lane != 0) return;
    err = *errw;
    if (err) {
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
      return;
    }
    int root = -1;
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
    if (root < 0) {
      err |= TC_ERR_INTERNAL;
#pragma unroll
      for (u32 w = 0; w < K::CW; ++w) code[w] = 0;
      return;
    }
    tc_wide_tree_code<K>(S, R, root, err, code);
  });
  return err;
}
