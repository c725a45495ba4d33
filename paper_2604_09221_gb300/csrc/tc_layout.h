// tc_layout.h -- per-thread scratch layout of the label-sweep kernels, shared
// by the host (jit.cpp, which writes it into generated sources) and by the
// table-driven kernels (kernels.cu, which evaluate it at compile time).
//
// Scratch is counted in 32-bit words; word i of thread t of a block lives at
// [i * threads + t] in shared memory, so any per-thread access pattern is
// free of bank conflicts.  Regions:
//   [lpar | cand]  one entry per label (at most one label per vertex)
//   [lab]          one label per vertex (table-driven sweep only: the
//                  specialised sweep keeps vertex labels in registers)
//   [bpair]        crossed boundary edges (odd d), for root detection
//   [pend]         pending joins; later the region children masks and four
//                  per-region byte arrays (smallest label, parent, path,
//                  code length)
//   [odd]          one odd-cycle bit per label
// The AHU codes reuse [lpar] once the region tree is built.
#pragma once

struct TcLayout {
  int d, V, lbytes, epw, wlab, nb, rmax, code64, wcode, pcap, wodd, snapw;
  int off_lpar, off_cand, off_lab, off_bpair, off_pend, off_adj, off_rlab, off_tpar, off_order,
      off_clen, off_odd, off_code, words, threads, hash;
  bool ok;
};

constexpr int tc_max(int a, int b) { return a > b ? a : b; }

// max_threads: upper bound of the block size (a multiple of 32); the block
// size is the largest multiple of 32 not above it of which two blocks fit in
// the 227 KB of shared memory of an SM (with the block's hash table).
constexpr TcLayout tc_layout(int d, bool vertex_labels, int max_threads) {
  TcLayout L{};
  L.d = d;
  L.V = 2 * d * d + 2 * d + 1;
  const int M = (d - 1) * (d - 2) / 2 + 1, nmax = (d % 2 == 0) ? M : M - 1;
  L.lbytes = L.V <= 126 ? 1 : 2;  // label ids and the "none" value fit 7 / 15 bits
  L.epw = 4 / L.lbytes;
  L.wlab = (L.V + L.epw - 1) / L.epw;
  L.nb = (d % 2) ? 2 * d : 0;
  L.rmax = nmax + 1;
  L.code64 = 2 * nmax > 30 ? 1 : 0;
  L.wcode = L.rmax * (L.code64 ? 2 : 1);
  const int wb = (L.rmax + 3) / 4;
  L.pcap = 2 * d + 24;
  L.wodd = (L.V + 31) / 32;
  L.snapw = (32 + L.epw - 1) / L.epw;
  L.off_lpar = 0;
  L.off_cand = L.wlab;
  L.off_lab = 2 * L.wlab;
  L.off_bpair = L.off_lab + (vertex_labels ? L.wlab : 0);
  L.off_pend = L.off_bpair + L.nb;
  L.off_adj = L.off_pend;
  L.off_rlab = L.off_adj + L.rmax;
  L.off_tpar = L.off_rlab + wb;
  L.off_order = L.off_tpar + wb;
  L.off_clen = L.off_order + wb;
  L.off_odd = L.off_pend + tc_max(L.pcap, L.rmax + 4 * wb);
  L.off_code = 0;
  L.words = L.off_odd + L.wodd;
  L.hash = d <= 7 ? 256 : 1024;
  // the table-driven kernels also hold the staged tables (<= 4 KB) per block
  const int budget = (vertex_labels ? 216 : 224) * 1024;
  L.threads = max_threads;
  while (L.threads > 32 && 2 * (L.words * 4 * L.threads + L.hash * 16 + 16) > budget)
    L.threads -= 32;
  L.ok = L.wcode <= L.wlab && d >= 1 && d <= 9;
  return L;
}
