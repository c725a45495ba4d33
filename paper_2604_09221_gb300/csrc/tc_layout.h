// tc_layout.h -- per-thread scratch layout of the label-sweep kernels, shared
// by the host (jit.cpp, which writes it into generated sources) and by the
// table-driven kernels (kernels.cu, batch.cu, which evaluate it at compile
// time).
//
// Scratch is counted in 32-bit words; word i of thread t of a block lives at
// [i * threads + t], so any per-thread access pattern is free of bank
// conflicts.  Regions:
//   [lpar | cand]  one entry per label (at most one label per vertex)
//   [lab]          one label per vertex (table-driven sweep only: the
//                  specialised sweep keeps vertex labels in registers)
//   [bpair]        crossed boundary edges (odd d), for root detection
//   [pend]         pending joins; later the region children masks and four
//                  per-region byte arrays (smallest label, parent, path,
//                  code length) of the narrow back end, or the regions'
//                  smallest labels (u16) of the wide one
//   [odd]          one odd-cycle bit per label
// Narrow back end (at most 32 regions, d <= 9): the AHU codes reuse [lpar]
// once the region tree is built.  Wide back end (d >= 10, up to 107 regions
// and 213-bit codes): parent, first-child and next-sibling bytes per region,
// the stack of live code offsets and two bit arenas, all over [lab] (free
// once the sweep has ended).
#pragma once

struct TcLayout {
  int d, V, np, sw, cw, wide, lbytes, epw, wlab, nb, rmax, code64, wcode, pcap, wodd, snapw;
  int off_lpar, off_cand, off_lab, off_bpair, off_pend, off_adj, off_rlab, off_tpar, off_order,
      off_clen, off_odd, off_code, words, threads, hash;
  // wide back end: region bytes, code-offset stack (u16), arena and build area
  int off_wpar, off_wfc, off_wns, off_went, off_warena, off_wtemp, warena_words, wide_words;
  bool ok;
};

constexpr int tc_max(int a, int b) { return a > b ? a : b; }

// Longest fan (earlier neighbours of one vertex of T^diamond) the join list
// can take: a vertex pushes at most one join per run of its fan plus one
// antipodal join, and the list is flushed when a fan might not fit.
constexpr int tc_pcap(int d) { return d <= 9 ? 2 * d + 24 : 4 * d + 16; }

// max_threads: upper bound of the block size (a multiple of 32); the block
// size is the largest multiple of 32 not above it of which two blocks fit in
// the 227 KB of shared memory of an SM (with the block's hash table).
constexpr TcLayout tc_layout(int d, bool vertex_labels, int max_threads) {
  TcLayout L{};
  L.d = d;
  L.V = 2 * d * d + 2 * d + 1;
  L.np = (d + 1) * (d + 2) / 2;
  L.sw = (L.np + 63) / 64;
  const int M = (d - 1) * (d - 2) / 2 + 1, nmax = (d % 2 == 0) ? M : M - 1;
  L.cw = (2 * nmax + 1 + 63) / 64;
  L.lbytes = L.V <= 126 ? 1 : 2;  // label ids and the "none" value fit 7 / 15 bits
  L.epw = 4 / L.lbytes;
  L.wlab = (L.V + L.epw - 1) / L.epw;
  L.nb = (d % 2) ? 2 * d : 0;
  L.rmax = nmax + 1;
  L.wide = L.rmax > 32 ? 1 : 0;
  L.code64 = 2 * nmax > 30 ? 1 : 0;
  L.wcode = L.wide ? 0 : L.rmax * (L.code64 ? 2 : 1);
  const int wb = (L.rmax + 3) / 4;
  L.pcap = tc_pcap(d);
  L.wodd = (L.V + 31) / 32;
  L.snapw = (32 + L.epw - 1) / L.epw;
  L.off_lpar = 0;
  L.off_cand = L.wlab;
  L.off_lab = 2 * L.wlab;
  L.off_bpair = L.off_lab + (vertex_labels ? L.wlab : 0);
  L.off_pend = L.off_bpair + L.nb;
  L.off_adj = L.off_pend;
  L.off_rlab = L.off_adj + (L.wide ? 0 : L.rmax);
  L.off_tpar = L.off_rlab + wb;
  L.off_order = L.off_tpar + wb;
  L.off_clen = L.off_order + wb;
  const int narrow_pend = L.rmax + 4 * wb, wide_pend = (L.rmax + 1) / 2;
  L.off_odd = L.off_pend + tc_max(L.pcap, L.wide ? wide_pend : narrow_pend);
  L.off_code = 0;
  // wide back end: live codes total at most 2 * (rmax - 1) bits
  L.warena_words = (2 * L.rmax + 63) / 32 + 3;
  L.off_wpar = L.off_lab;
  L.off_wfc = L.off_wpar + wb;
  L.off_wns = L.off_wfc + wb;
  L.off_went = L.off_wns + wb;
  L.off_warena = L.off_went + (L.rmax / 2 + 2 + 1) / 2;
  L.off_wtemp = L.off_warena + L.warena_words;
  L.wide_words = L.off_wtemp + L.warena_words - L.off_lab;
  L.words = L.off_odd + L.wodd;
  L.hash = L.cw > 1 ? 0 : (d <= 7 ? 256 : 1024);
  // the table-driven kernels also hold the staged tables (<= 17 KB) per block
  const int budget = (vertex_labels ? (d <= 9 ? 216 : 192) : 224) * 1024;
  L.threads = max_threads;
  while (L.threads > 32 && 2 * (L.words * 4 * L.threads + L.hash * 16 + 16) > budget)
    L.threads -= 32;
  const bool wide_fits = !L.wide || (vertex_labels && L.wide_words <= L.wlab);
  L.ok = L.wcode <= L.wlab && wide_fits && d >= 1 && d <= 16 && L.cw <= 4 && L.sw <= 3;
  return L;
}

// Pivots of the orbit sweep (TS_ENUM_ORBITS, Sec. 3 symmetry).  The four
// elements of (Z/2)^3 that keep sigma(0, 1) (sigma -> sigma + a + b i + c j
// with a + c = 0 mod 2) change the high part of a mask (bits d+2 .. |A|-1:
// every lattice point with j >= 1 but (0, 1), bit b = k(i, j) - d - 2) by
// the span of A (points with i odd) and B (points with j even).  With A and
// B in echelon form (top bits p1 > p2), every coset h + span{A, B} holds
// exactly one high part whose bits p1 and p2 are zero.  Needs 2 <= d <= 9
// (A and B independent; one sign word); returns false otherwise.
constexpr bool tc_orbit_pivots(int d, int *p1, int *p2) {
  if (d < 2 || d > 9) return false;
  unsigned long long a = 0, b = 0;
  for (int j = 1; j <= d; ++j)
    for (int i = 0; i + j <= d; ++i) {
      if (i == 0 && j == 1) continue;
      const int k = j * (d + 1) - j * (j - 1) / 2 + i, bit = k - d - 2;
      if (i % 2 == 1) a |= 1ull << bit;
      if (j % 2 == 0) b |= 1ull << bit;
    }
  auto top = [](unsigned long long x) {
    int t = -1;
    for (int q = 0; q < 64; ++q)
      if ((x >> q) & 1ull) t = q;
    return t;
  };
  if (top(b) > top(a)) {
    const unsigned long long x = a;
    a = b;
    b = x;
  }
  if (top(b) == top(a)) b ^= a;
  *p1 = top(a);
  *p2 = top(b);
  return *p1 > *p2 && *p2 >= 0;
}
