// tc_table_sweep.cuh -- Algorithm 1 for one sign vector, driven by the
// triangulation tables of host.cpp (TS_KERNEL_TABLE; the query, sweep and
// batch kernels of kernels.cu and batch.cu all call tc_table_classify).
//
// Table format (32-bit words, vertex ids are positions in the sweep order):
//   vdesc[V]  bits 0-7 lattice index k(v), bit 8 Eq. 2 parity constant c(v)
//             (sign(v) = sigma_k ^ c), bits 9-15 fan length m, bits 16-31
//             first fan entry
//   fan[NF]   bits 0-9 earlier neighbour u, bits 10-17 k(u), bit 18 c(u),
//             bit 19 "u and the previous entry span a triangle with v"
//   vext[V]   bits 0-9 the antipodal partner x < v of v, bits 10-19 and
//             20-29 the other end b < v of up to two boundary edges kept for
//             root detection (1023: none)
//
// The sweep gives every vertex the label of its first same-sign earlier
// neighbour, or a fresh label; joins (several same-sign runs in a vertex's
// fan, antipodal pairs) are appended without branching and applied after the
// sweep (Alg. 1, lines 3-4); the back end does lines 5-11.
#pragma once

#include "tc_layout.h"
#include "tc_runtime.cuh"

constexpr u32 TC_TAB_NONE = 1023u;

// Traits of a table-driven kernel of degree D_ (scratch with one label per
// vertex, since the sweep is not unrolled): block size MAXT if FIXED, else
// the largest multiple of 32 up to MAXT of which two blocks fit an SM.
template <int D_, int MAXT, bool FIXED>
struct TcTableK {
  static constexpr TcLayout L = tc_layout(D_, true, MAXT);
  static constexpr u32 D = D_, V = L.V, NPOINTS = L.np, W = L.sw, CW = L.cw, WIDE = L.wide,
                       RMAX = L.rmax, NB = L.nb, THREADS = FIXED ? MAXT : L.threads,
                       HASH = L.hash, LBYTES = L.lbytes, CODE64 = L.code64, PCAP = L.pcap,
                       WODD = L.wodd, WORDS = L.words, OFF_LPAR = L.off_lpar,
                       OFF_CAND = L.off_cand, OFF_LAB = L.off_lab, OFF_BPAIR = L.off_bpair,
                       OFF_PEND = L.off_pend, OFF_ADJ = L.off_adj, OFF_RLAB = L.off_rlab,
                       OFF_TPAR = L.off_tpar, OFF_ORDER = L.off_order, OFF_CLEN = L.off_clen,
                       OFF_ODD = L.off_odd, OFF_CODE = L.off_code, OFF_WPAR = L.off_wpar,
                       OFF_WFC = L.off_wfc, OFF_WNS = L.off_wns, OFF_WENT = L.off_went,
                       OFF_WARENA = L.off_warena, OFF_WTEMP = L.off_wtemp,
                       WARENA = L.warena_words;
  static_assert(L.ok, "scratch layout");
};

template <class K>
struct TcCodeOut {
  u64 w[K::CW];
};

template <class K>
__device__ __forceinline__ TcCodeOut<K> tc_table_classify(const TcSig<K::W> &sig,
                                                          const u32 *__restrict__ tab, u32 off_fan,
                                                          u32 off_vext, const TcScratch<K> &S,
                                                          u32 &err) {
  typedef TcScratch<K> TS;
  const u32 *vdesc = tab;
  const u32 *fan = tab + off_fan;
  const u32 *vext = tab + off_vext;
  u32 nl = 0, nb = 0, np = 0;
  tc_clear_odd(S);
  for (u32 v = 0; v < K::V; ++v) {
    const u32 desc = vdesc[v];
    const u32 sv = sig.bit(desc & 255u) ^ ((desc >> 8) & 1u);
    const u32 m = (desc >> 9) & 127u, fs = desc >> 16;
    if (np + m + 1 > K::PCAP) {  // at most m - 1 run joins and one antipodal join at v
      tc_unions(S, np);
      np = 0;
    }
    u32 lv = 0, l0 = TS::NONE, any = 0, prev = 0;
    for (u32 i = 0; i < m; ++i) {
      const u32 f = fan[fs + i];
      const u32 lu = *S.lab(K::OFF_LAB, f & 1023u);
      const u32 e = sig.bit((f >> 10) & 255u) ^ ((f >> 18) & 1u) ^ sv ^ 1u;
      const u32 st = e & ~(((f >> 19) & 1u) & prev) & 1u;  // e starts a run of the fan
      l0 = i == 0 ? lu : l0;
      // a run after the first: join its label with the vertex's label
      // (a predicated store: no branch, and no write when nothing joins)
      if (st & any) S.word(K::OFF_PEND, np) = lv | (lu << 16);
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
    *S.lab(K::OFF_LAB, v) = (typename TS::lab_t)lv;
    const u32 x = vext[v];
    if ((x & 1023u) != TC_TAB_NONE) {  // the antipodal partner, reached earlier
      S.word(K::OFF_PEND, np) = (u32)*S.lab(K::OFF_LAB, x & 1023u) | (lv << 16) | 0x80000000u;
      ++np;
    }
    if (K::D % 2) {  // crossed boundary edges, for the pseudoline's region
#pragma unroll
      for (u32 sh = 10; sh <= 20; sh += 10) {
        const u32 b = (x >> sh) & 1023u;
        if (b == TC_TAB_NONE) continue;
        const u32 db = vdesc[b];
        if ((sig.bit(db & 255u) ^ ((db >> 8) & 1u)) != sv) {
          tc_bpair(S, nb, *S.lab(K::OFF_LAB, b), lv);
          ++nb;
        }
      }
    }
  }
  tc_unions(S, np);
  TcCodeOut<K> out;
  if constexpr (K::WIDE) {
    tc_backend_wide(S, nl, nb, err, out.w);
  } else {
    out.w[0] = tc_backend(S, nl, nb, err);
  }
  return out;
}

// Load one sign vector of W words (bits at or above |A| dropped).
template <class K>
__device__ __forceinline__ TcSig<K::W> tc_load_sig(const u64 *__restrict__ signs, u64 i) {
  TcSig<K::W> s;
#pragma unroll
  for (u32 w = 0; w < K::W; ++w) s.w[w] = signs[i * K::W + w];
  s.w[K::W - 1] &= tc_top_mask(K::NPOINTS, K::W);
  return s;
}
