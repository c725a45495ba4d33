// Test infrastructure: the histogram inserts of tc_runtime.cuh run on the
// host, one call at a time (device_shims.h), against a std::map:
//  - tc_global_add (one-word codes): open addressing with linear probing;
//  - tc_hist_add (block-private table of HASH slots), which spills into the
//    device table when it is full;
//  - tc_global_add_wide and tc_hist_add_wide (codes of 2 to 4 words), whose
//    count word carries the BUSY / READY flags.
// Every key must land in exactly one slot with the summed count, every used
// slot of a multi-word table must end READY and not BUSY, and a table with
// fewer slots than keys must report TC_ERR_OVERFLOW.  Keys are drawn from a
// small pool so that they repeat, and small tables so that probes collide.
// Exit status 0 when every check holds.
#include "device_shims.h"
#include "tc_runtime.cuh"

#include <array>
#include <map>
#include <vector>

static u64 rng_state = 88172645463325252ull;
static u64 next_rand() {  // xorshift64, for the keys only
  rng_state ^= rng_state << 13;
  rng_state ^= rng_state >> 7;
  rng_state ^= rng_state << 17;
  return rng_state;
}

static int failures = 0;
#define CHECK(cond, what)                                              \
  do {                                                                 \
    if (!(cond)) {                                                     \
      printf("FAILED %s (%s:%d)\n", what, __FILE__, __LINE__);         \
      ++failures;                                                      \
    }                                                                  \
  } while (0)

// A pool of n distinct nonzero keys of CW words: some equal in word 0, some
// with word 0 zero.
template <u32 CW>
static std::vector<std::array<u64, CW>> key_pool(int n) {
  std::map<std::array<u64, CW>, int> seen;
  std::vector<std::array<u64, CW>> pool;
  while ((int)pool.size() < n) {
    std::array<u64, CW> k{};
    const int kind = (int)(next_rand() % 3);
    for (u32 w = 0; w < CW; ++w) k[w] = next_rand();
    if (kind == 1 && !pool.empty()) k[0] = pool[0][0];    // shares word 0 with the first key
    if (kind == 2 && CW > 1) k[0] = 0;                      // only upper words set
    bool nz = false;
    for (u32 w = 0; w < CW; ++w) nz |= k[w] != 0;
    if (!nz || seen.count(k)) continue;
    seen[k] = 1;
    pool.push_back(k);
  }
  return pool;
}

static void one_word(u64 slots, int distinct, int inserts, bool expect_overflow) {
  std::vector<u64> keys(slots, 0);
  std::vector<unsigned long long> cnt(slots, 0);
  u32 err = 0;
  auto pool = key_pool<1>(distinct);
  std::map<u64, unsigned long long> want, got;
  for (int i = 0; i < inserts; ++i) {
    const u64 k = pool[next_rand() % pool.size()][0];
    const unsigned long long c = 1 + next_rand() % 7;
    tc_global_add(keys.data(), cnt.data(), slots, &err, k, c);
    want[k] += c;
  }
  if (expect_overflow) {
    CHECK(err & TC_ERR_OVERFLOW, "one-word table overflow reported");
    return;
  }
  CHECK(err == 0, "one-word insert without error");
  for (u64 s = 0; s < slots; ++s)
    if (keys[s]) {
      CHECK(!got.count(keys[s]), "one-word key in one slot");
      got[keys[s]] = cnt[s];
    } else {
      CHECK(cnt[s] == 0, "empty one-word slot has no count");
    }
  CHECK(got == want, "one-word counts");
}

static void block_table_spills(int distinct, int inserts) {
  constexpr u32 HASH = 16;
  std::vector<u64> hkeys(HASH, 0), gkeys(256, 0);
  std::vector<unsigned long long> hcnt(HASH, 0), gcnt(256, 0);
  u32 gerr = 0;
  auto pool = key_pool<1>(distinct);
  std::map<u64, unsigned long long> want, got;
  for (int i = 0; i < inserts; ++i) {
    threadIdx.x = (unsigned)(i & 31);  // any lane: it inserts alone
    const u64 k = i % 11 == 0 ? 0 : pool[next_rand() % pool.size()][0];   // 0: nothing to add
    tc_hist_add<HASH>(k, hkeys.data(), hcnt.data(), gkeys.data(), gcnt.data(), gkeys.size(), &gerr);
    if (k) want[k] += 1;
  }
  CHECK(gerr == 0, "block table spill without error");
  for (u32 s = 0; s < HASH; ++s)
    if (hkeys[s]) got[hkeys[s]] += hcnt[s];
  for (size_t s = 0; s < gkeys.size(); ++s)
    if (gkeys[s]) got[gkeys[s]] += gcnt[s];
  CHECK(got == want, "block table + device table counts");
  if (distinct > (int)HASH) {
    int in_global = 0;
    for (u64 k : gkeys) in_global += k != 0;
    CHECK(in_global >= distinct - (int)HASH, "full block table spills into the device table");
  }
}

template <u32 CW>
static void multi_word(u64 slots, int distinct, int inserts, bool expect_overflow, bool warp_api) {
  std::vector<u64> keys(slots * CW, 0);
  std::vector<unsigned long long> cnt(slots, 0);
  u32 err = 0;
  auto pool = key_pool<CW>(distinct);
  std::map<std::array<u64, CW>, unsigned long long> want, got;
  for (int i = 0; i < inserts; ++i) {
    std::array<u64, CW> k = pool[next_rand() % pool.size()];
    unsigned long long c = 1;
    if (warp_api) {
      threadIdx.x = (unsigned)(i & 31);
      if (i % 13 == 0) k = std::array<u64, CW>{};   // all-zero key: nothing to add
      tc_hist_add_wide<CW>(k.data(), keys.data(), cnt.data(), slots, &err);
    } else {
      c = 1 + next_rand() % 5;
      tc_global_add_wide<CW>(keys.data(), cnt.data(), slots, &err, k.data(), c);
    }
    bool nz = false;
    for (u32 w = 0; w < CW; ++w) nz |= k[w] != 0;
    if (nz) want[k] += c;
  }
  if (expect_overflow) {
    CHECK(err & TC_ERR_OVERFLOW, "multi-word table overflow reported");
    return;
  }
  CHECK(err == 0, "multi-word insert without error");
  for (u64 s = 0; s < slots; ++s) {
    std::array<u64, CW> k;
    bool nz = false;
    for (u32 w = 0; w < CW; ++w) nz |= (k[w] = keys[s * CW + w]) != 0;
    if (!nz) {
      CHECK(cnt[s] == 0, "empty multi-word slot has no count or flag");
      continue;
    }
    CHECK(cnt[s] & TC_SLOT_READY, "used slot published READY");
    CHECK(!(cnt[s] & TC_SLOT_BUSY), "used slot not left BUSY");
    CHECK(!got.count(k), "multi-word key in one slot");
    got[k] = cnt[s] & (TC_SLOT_BUSY - 1);
  }
  CHECK(got == want, "multi-word counts");
}

int main() {
  one_word(16, 5, 400, false);
  one_word(16, 16, 2000, false);     // every slot used
  one_word(64, 40, 5000, false);
  one_word(16, 17, 400, true);
  block_table_spills(10, 600);
  block_table_spills(40, 3000);      // more codes than the block table holds
  multi_word<2>(16, 9, 500, false, false);
  multi_word<2>(32, 32, 3000, false, false);
  multi_word<3>(64, 50, 4000, false, false);
  multi_word<4>(128, 100, 8000, false, false);
  multi_word<4>(16, 17, 500, true, false);
  multi_word<2>(64, 30, 2000, false, true);
  multi_word<4>(64, 30, 2000, false, true);
  printf("hash insert checks: %d failed\n", failures);
  return failures != 0;
}
