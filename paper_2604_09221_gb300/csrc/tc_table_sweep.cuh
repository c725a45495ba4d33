// tc_table_sweep.cuh -- Algorithm 1 for one sign vector, driven by the
// triangulation tables of host.cpp (TS_KERNEL_TABLE; the query, sweep and
// batch kernels of kernels.cu and batch.cu all call tc_table_classify).
//
// The sweep itself (and the table format) is tc_sweep_table of
// tc_runtime.cuh; the back end picks the narrow or the wide form.
#pragma once

#include "tc_layout.h"
#include "tc_runtime.cuh"

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

// lw: the label slots (tc_sweep_table), null for the scratch's [lab] region;
// OFF: the tables' fan entries carry slot offsets (tc_fan_to_offsets).
template <class K, bool OFF = false>
__device__ __forceinline__ TcCodeOut<K> tc_table_classify(const TcSig<K::W> &sig,
                                                          const u32 *__restrict__ tab, u32 off_fan,
                                                          u32 off_vext, const TcScratch<K> &S,
                                                          u32 &err, u32 *lw = nullptr) {
  u32 nl = 0, nb = 0, np = 0;
  tc_clear_odd(S);
  tc_sweep_table<K, OFF>(sig, tab, tab + off_fan, tab + off_vext, 0, K::V, S,
                         lw ? lw : S.w + K::OFF_LAB * K::THREADS, nl, nb, np);
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
