// Test infrastructure: the table-driven sweep (tc_table_sweep.cuh, both back
// ends) or the warp-per-instance sweep (tc_warp_sweep.cuh, its 32 lanes run
// one after another, forward for even instances and in reverse for odd ones)
// compiled for the host, fed the tables that host.cpp builds, one instance
// at a time, against the oracle.  Random sign vectors of a seeded counter
// stream, then eight special ones (constant, Harnack's distribution,
// parities).  Usage: run_table_sweep <d> <edges file> <n> [warp]; exit 0
// when all codes agree.
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <vector>
static inline int __popc(unsigned x) { return __builtin_popcount(x); }
static inline int __popcll(unsigned long long x) { return __builtin_popcountll(x); }
static inline int __ffs(unsigned x) { return __builtin_ffs(x); }
static inline int __ffsll(unsigned long long x) { return __builtin_ffsll(x); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
struct HostDim { unsigned x; } threadIdx{0};
static inline unsigned long long atomicCAS(unsigned long long *p, unsigned long long c, unsigned long long v) { auto o = *p; if (o == c) *p = v; return o; }
static inline unsigned long long atomicAdd(unsigned long long *p, unsigned long long v) { auto o = *p; *p += v; return o; }
static inline unsigned atomicOr(unsigned *p, unsigned v) { auto o = *p; *p |= v; return o; }
static inline unsigned __match_any_sync(unsigned, unsigned long long) { return 1u; }
static inline void __nanosleep(unsigned) {}
static inline void __threadfence() {}
#include "host.cpp"
#undef __noinline__
#define __noinline__
#include "tc_table_sweep.cuh"
#define TC_WARP_EMULATE
#include "tc_warp_sweep.cuh"
extern "C" {
#include "tcurve_oracle.h"
}
// the device launches host.cpp refers to are not used here
namespace tcurve {
cudaError_t jit_prepare(ts_tri *) { return cudaErrorNotSupported; }
cudaError_t launch_real_schemes_jit(ts_tri *, const uint64_t *, uint64_t, uint64_t *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_real_schemes(const ts_tri *, const uint64_t *, uint64_t, uint64_t *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_splitmix_masks(int, uint64_t, uint64_t, uint64_t *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_hist_clear(ts_hist *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_hist_compact(ts_hist *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_selftest_wait(unsigned long long, uint32_t *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_enumerate_jit(ts_tri *, uint64_t, uint64_t, uint32_t, ts_hist *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_enumerate(const ts_tri *, uint64_t, uint64_t, uint32_t, ts_hist *, cudaStream_t, bool) { return cudaErrorNotSupported; }
cudaError_t launch_real_schemes_warp(const ts_tri *, const uint64_t *, uint64_t, uint64_t *, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_enumerate_warp(const ts_tri *, uint64_t, uint64_t, uint32_t, ts_hist *, cudaStream_t) { return cudaErrorNotSupported; }
void jit_release(ts_tri *) {}
std::string jit_source(const Diamond &, bool, int) { return ""; }
std::string jit_compile_cubin(const std::string &, std::string *, const std::vector<std::string> &) {
  return "";
}
std::string jit_jobs_link(const std::vector<const Diamond *> &, std::string *) { return ""; }
void jit_config(int, int, int, bool *, int *) {}
}  // namespace tcurve

template <int D>
struct HostK : TcTableK<D, 32, true> {
  static constexpr u32 THREADS = 1;  // one instance: contiguous scratch
};

static uint64_t mix64(uint64_t x) {  // splitmix64 finaliser, for the inputs only
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <int D>
int run(const char *edge_file, int n, bool warp) {
  typedef HostK<D> K;
  typedef TcWarpK<D> WK;
  std::vector<int32_t> e;
  {
    std::ifstream f(edge_file);
    int a;
    while (f >> a) e.push_back(a);
  }
  const int ne = (int)e.size() / 4;
  std::vector<std::array<Pt, 3>> tris;
  ts_tri t;
  if (!triangles_of(D, e.data(), ne, tris) || !build_diamond(D, tris, t.dia) || !pack_tables(t.dia, &t))
    return 2;
  std::vector<int32_t> otri(6 * D * D);
  if (orc_triangles_from_edges(D, ne, e.data(), otri.data(), D * D) != D * D) return 2;
  std::vector<u32> scratch(K::WORDS > WK::WORDS ? K::WORDS : WK::WORDS, 0xA5A5A5A5u);
  const TcScratch<K> S{scratch.data()};
  std::vector<u32> slots((t.lay.nslots + TcScratch<K>::EPW - 1) / TcScratch<K>::EPW, 0x5A5A5A5Au);
  std::vector<u32> offtab(t.host_tables);
  tc_fan_to_offsets(offtab.data() + t.lay.off_fan, t.lay.NF, TcScratch<K>::EPW, K::LBYTES,
                    K::THREADS, 0, 1);
  const u32 *wt = t.host_wtables.data();
  const int cw = orc_code_words(D);
  int bad = 0;
  for (int i = 0; i < n + 8; ++i) {
    TcSig<K::W> sg;
    for (u32 w = 0; w < K::W; ++w) sg.w[w] = mix64(1000003ull * D + (uint64_t)i * K::W + w);
    if (i >= n) {  // special sign vectors
      for (u32 w = 0; w < K::W; ++w) sg.w[w] = 0;
      for (int j = 0; j <= D; ++j)
        for (int ii = 0; ii + j <= D; ++ii) {
          const int k = j * (D + 1) - j * (j - 1) / 2 + ii;
          bool b = false;
          switch (i - n) {
            case 1: b = true; break;
            case 2: b = ii % 2 == 0 && j % 2 == 0; break;  // Harnack's distribution
            case 3: b = ii % 2 == 1 && j % 2 == 1; break;
            case 4: b = (ii + j) % 2 == 0; break;
            case 5: b = ii % 2 == 0; break;
            case 6: b = k % 2 == 0; break;
            case 7: b = (ii % 2 == 0) != (j % 2 == 0); break;
            default: break;
          }
          if (b) sg.w[k >> 6] |= 1ull << (k & 63);
        }
    }
    sg.w[K::W - 1] &= tc_top_mask(K::NPOINTS, K::W);
    u32 err = 0;
    TcCodeOut<K> got;
    if (warp) {
      tc_emu_reverse = i % 2 == 1;
      err = tc_warp_classify<D>(sg, wt + t.wlay.off_v, wt + t.wlay.off_e, t.wlay.E,
                                wt + t.wlay.off_anti, t.wlay.nanti, wt + t.wlay.off_bedge,
                                t.wlay.nbedge, scratch.data(), got.w);
    } else {
      // odd instances keep the label slots apart from the scratch, as the
      // kernels with global scratch do (slots in shared memory); the slot
      // buffer holds exactly the words the table's slots need.  Every fourth
      // instance also reads the tables with the fan entries rewritten to
      // their slots' byte offsets, as those kernels stage them.
      if (i % 4 == 3)
        got = tc_table_classify<K, true>(sg, offtab.data(), t.lay.off_fan, t.lay.off_vext, S, err,
                                         slots.data());
      else
        got = tc_table_classify<K>(sg, t.host_tables.data(), t.lay.off_fan, t.lay.off_vext, S, err,
                                   i % 2 ? slots.data() : nullptr);
    }
    uint64_t want[4] = {0, 0, 0, 0};
    const int rc = orc_real_scheme(D, otri.data(), (const uint64_t *)sg.w, want, cw, nullptr);
    bool same = rc == 0 && !err;
    for (int w = 0; w < cw; ++w) same &= got.w[w] == want[w];
    if (!same) {
      if (bad < 3) printf("instance %d differs (err %u, oracle status %d)\n", i, err, rc);
      ++bad;
    }
  }
  printf("d=%d %s instances=%d differing=%d\n", D, warp ? "warp" : "table", n + 8, bad);
  return bad != 0;
}

int main(int argc, char **argv) {
  const int d = atoi(argv[1]), n = atoi(argv[3]);
  const bool warp = argc > 4 && std::string(argv[4]) == "warp";
  switch (d) {
    case 1: return run<1>(argv[2], n, warp);
    case 2: return run<2>(argv[2], n, warp);
    case 3: return run<3>(argv[2], n, warp);
    case 4: return run<4>(argv[2], n, warp);
    case 5: return run<5>(argv[2], n, warp);
    case 6: return run<6>(argv[2], n, warp);
    case 7: return run<7>(argv[2], n, warp);
    case 8: return run<8>(argv[2], n, warp);
    case 9: return run<9>(argv[2], n, warp);
    case 10: return run<10>(argv[2], n, warp);
    case 11: return run<11>(argv[2], n, warp);
    case 12: return run<12>(argv[2], n, warp);
    case 13: return run<13>(argv[2], n, warp);
    case 14: return run<14>(argv[2], n, warp);
    case 15: return run<15>(argv[2], n, warp);
    case 16: return run<16>(argv[2], n, warp);
  }
  return 2;
}
