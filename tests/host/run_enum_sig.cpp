// Test infrastructure: the sweep's mask maps (tc_enum_sig of tc_runtime.cuh,
// with the orbit sweep's pivots from tc_layout.h) run on the host.  Reads lines "d flags k" from standard input and prints
// the W sign words of mask m(k) for each, in hexadecimal, W = ceil(|A| / 64).
#include "device_shims.h"
#include "tc_layout.h"
#include "tc_runtime.cuh"

template <u32 W>
static void print_sig(u64 k, u32 flags, u32 d) {
  const TcSig<W> s = tc_enum_sig<W>(k, flags, d);
  for (u32 w = 0; w < W; ++w) printf("%s%llx", w ? " " : "", (unsigned long long)s.w[w]);
  printf("\n");
}

int main() {
  unsigned d, flags;
  unsigned long long k;
  while (scanf("%u %u %llu", &d, &flags, &k) == 3) {
    const u32 W = ((d + 1) * (d + 2) / 2 + 63) / 64;
    if (flags & 8u) {  // the orbit sweep: the pivots ride in the flags, as ts_enumerate puts them
      int p1 = 0, p2 = 0;
      if (!tc_orbit_pivots((int)d, &p1, &p2)) return 2;
      flags |= ((unsigned)p1 << 8) | ((unsigned)p2 << 16);
    }
    if (W == 1) print_sig<1>(k, flags, d);
    else if (W == 2) print_sig<2>(k, flags, d);
    else print_sig<3>(k, flags, d);
  }
  return 0;
}
