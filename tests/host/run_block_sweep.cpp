// Test infrastructure: run the block sweep of a generated specialised source
// (included as GEN) on the host, one lane at a time, for whole warps, and
// compare each warp's histogram with the oracle's over the same masks.
// Usage: run_block_sweep <edges file> <warps> [plain|flip|reduced|orbits|classify];
// the mask map of a warp is (h << oshift) | (t << ishift), t < 2^ib, as in
// the sweeps without flags, with TS_ENUM_FLIP (bit 0 fixed) and with
// TS_ENUM_REDUCED (bits 0, 1 and d + 1 fixed), and blocks of TS_ENUM_ORBITS
// (h the block's orbit high part, bit d + 1 fixed).  "classify" runs the per-mask
// classifier tc_classify (query kernel, per-mask sweeps) on 64 x <warps>
// random masks and the constant ones instead.  Exit status 0 when all match.
#include "device_shims.h"
#include "tc_layout.h"
#include GEN
extern "C" {
#include "tcurve_oracle.h"
}
#include <fstream>
#include <map>
#include <string>
#include <vector>

int main(int argc, char **argv) {
  const int d = TcK::D;
  std::vector<int32_t> e;
  {
    std::ifstream f(argv[1]);
    int a;
    while (f >> a) e.push_back(a);
  }
  const int nh = argc > 2 ? atoi(argv[2]) : 8;
  const std::string mode = argc > 3 ? argv[3] : "plain";
  std::vector<int32_t> otri(6 * d * d);
  if (orc_triangles_from_edges(d, (int)e.size() / 4, e.data(), otri.data(), d * d) != d * d) return 2;
  if (mode == "classify") {
    const unsigned npts = (d + 1) * (d + 2) / 2;
    const u64 valid = npts >= 64 ? ~0ull : (1ull << npts) - 1;
    std::vector<unsigned> scr1((size_t)TcK::WORDS * TcK::THREADS + 64, 0xA5A5A5A5u);
    unsigned long long st = 99991;
    int bad = 0, n = 64 * nh + 2;
    for (int i = 0; i < n; ++i) {
      st = st * 6364136223846793005ull + 1442695040888963407ull;
      const u64 m = i == 0 ? 0 : (i == 1 ? valid : (st ^ (st >> 29)) & valid);
      threadIdx.x = (unsigned)(i & 31);
      u32 err = 0;
      const TcS S{scr1.data() + threadIdx.x};
      const u64 got = tc_classify(m, S, err);
      uint64_t want = 0;
      const uint64_t mw = m;
      if (orc_real_scheme(d, otri.data(), &mw, &want, 1, nullptr) != 0) return 3;
      if (got != want || err) {
        if (bad < 3) printf("mask %llx: %llx, oracle %llx (err %u)\n", (unsigned long long)m,
                            (unsigned long long)got, (unsigned long long)want, err);
        ++bad;
      }
    }
    printf("d=%d map=classify masks=%d differing=%d\n", d, n, bad);
    return bad != 0;
  }
  unsigned ib = d + 1, oshift = d + 1, ishift = 0, oflags = 0;
  if (mode == "flip") { ib = d; ishift = 1; }
  else if (mode == "reduced") { ib = d - 1; ishift = 2; oshift = d + 2; }
  else if (mode == "orbits") {  // blocks of orbit high parts (TS_ENUM_ORBITS)
    int p1 = 0, p2 = 0;
    if (!tc_orbit_pivots(d, &p1, &p2)) return 2;
    oshift = d + 2;
    oflags = 8u | ((unsigned)p1 << 8) | ((unsigned)p2 << 16);
  } else if (mode != "plain") return 2;
  if (ib < 5) return 2;  // fewer middle-row patterns than lanes: no block sweep
  const unsigned ireps = (1u << ib) / 32u;
  std::vector<unsigned> scr((size_t)TcK::WORDS * TcK::THREADS + 64, 0xA5A5A5A5u);
  const unsigned npts = (d + 1) * (d + 2) / 2;
  const unsigned long long hmax = 1ull << (npts - oshift - (oflags ? 2 : 0));
  unsigned long long state = 12345;
  int bad = 0;
  for (int t = 0; t < nh; ++t) {
    state = state * 6364136223846793005ull + 1442695040888963407ull;
    const unsigned long long hb = t == 0 ? 0 : (t == 1 ? hmax - 1 : (state >> 11) % hmax);
    const unsigned long long h = oflags ? tc_orbit_high(hb, oflags) : hb;  // as the kernel maps it
    std::vector<u64> hkeys(TcK::HASH, 0), gkeys(1 << 12, 0);
    std::vector<unsigned long long> hcnt(TcK::HASH, 0), gcnt(1 << 12, 0);
    u32 gerr = 0, err = 0;
    unsigned long long failed = 0;
    for (unsigned lane = 0; lane < 32; ++lane) {
      threadIdx.x = lane;
      const TcS S{scr.data() + lane};
      tc_sweep_amortised(h << oshift, ishift, ireps, S, err, hkeys.data(), hcnt.data(), gkeys.data(),
                         gcnt.data(), gkeys.size(), &gerr, failed);
    }
    std::map<u64, unsigned long long> got, want;
    for (size_t s = 0; s < hkeys.size(); ++s)
      if (hkeys[s]) got[hkeys[s]] += hcnt[s];
    for (size_t s = 0; s < gkeys.size(); ++s)
      if (gkeys[s]) got[gkeys[s]] += gcnt[s];
    for (unsigned long long tt = 0; tt < (1ull << ib); ++tt) {
      const uint64_t m = (h << oshift) | (tt << ishift);
      uint64_t code = 0;
      if (orc_real_scheme(d, otri.data(), &m, &code, 1, nullptr) != 0) return 3;
      want[code] += 1;
    }
    if (got != want || err || gerr || failed) {
      ++bad;
      printf("warp h=%llu differs (%zu codes, oracle %zu; err %u %u, failed %llu)\n", h, got.size(),
             want.size(), err, gerr, failed);
    }
  }
#ifdef TC_TEST_COUNT_SNAP
  // lanes whose half-diamonds left more than 32 labels (the snapshot path),
  // and lanes with an odd-cycle flag set when the snapshot was taken
  printf("snapshot_lanes=%ld odd_lanes=%ld ", tc_test_snap_lanes, tc_test_odd_lanes);
#endif
  printf("d=%d map=%s warps=%d differing=%d\n", d, mode.c_str(), nh, bad);
  return bad != 0;
}
