// jit_kernels.cuh -- kernels of the triangulation-specialised sources.
//
// A generated source is: the traits struct TcK (degree, block size, scratch
// layout of tc_layout.h), tc_runtime.cuh, the generated sweep functions
// tc_classify (one mask) and tc_sweep_amortised (a block of masks that share
// their high bits), then this file.

// Per-thread scratch: in shared memory, or (TcK::GSCR) in the launch's
// global buffer, one slab of WORDS x THREADS words per block.
__device__ __forceinline__ TcScratch<TcK> tc_scratch(u32 *smem, u32 *gscr) {
  return TcScratch<TcK>{(TcK::GSCR ? gscr + (u64)blockIdx.x * TcK::WORDS * TcK::THREADS : smem) +
                        threadIdx.x};
}

// Shared words in front of the block's hash table (the scratch, unless global).
#define TC_SMEM_SCRATCH (TcK::GSCR ? 0u : TcK::WORDS * TcK::THREADS)

// Codes of n sign vectors (one word each), grid-stride.
// Register budgets: the block sweep is compiled for MINB resident blocks per
// SM; the per-mask kernels, which keep more live state per thread, for at
// most 4 (global scratch) or MINB (shared scratch).
#define TC_MINB_MASK (TcK::GSCR && TcK::MINB > 4u ? 4u : TcK::MINB)

extern "C" __global__ void __launch_bounds__(TcK::THREADS, TC_MINB_MASK)
    tc_real_schemes(const u64 *__restrict__ signs, u64 n, u64 *__restrict__ codes, u32 *err_word,
                    u32 *gscr) {
  extern __shared__ __align__(16) u32 tc_smem[];
  const TcScratch<TcK> S = tc_scratch(tc_smem, gscr);
  const u64 valid = TcK::NPOINTS >= 64 ? ~0ull : ((1ull << (TcK::NPOINTS & 63)) - 1);
  u32 err = 0;
  for (u64 i = (u64)blockIdx.x * TcK::THREADS + threadIdx.x; i < n;
       i += (u64)gridDim.x * TcK::THREADS)
    codes[i] = tc_classify(signs[i] & valid, S, err);
  if (err) atomicOr(err_word, err);
}

#define TC_CHUNK (TcK::THREADS * 16)

// Sweep of masks m(lo + i), i < total, in chunks pulled from a work counter.
extern "C" __global__ void __launch_bounds__(TcK::THREADS, TC_MINB_MASK)
    tc_enumerate(u64 lo, u64 total, u32 flags, u64 *gkeys, unsigned long long *gcnt, u64 gslots,
                 u32 *gerr, unsigned long long *gfailed, unsigned long long *work, u32 *gscr) {
  extern __shared__ __align__(16) u32 tc_smem[];
  u64 *hkeys = reinterpret_cast<u64 *>(tc_smem + TC_SMEM_SCRATCH);
  unsigned long long *hcnt = reinterpret_cast<unsigned long long *>(hkeys + TcK::HASH);
  unsigned long long *chunk = hcnt + TcK::HASH;
  const TcScratch<TcK> S = tc_scratch(tc_smem, gscr);
  for (u32 s = threadIdx.x; s < TcK::HASH; s += TcK::THREADS) {
    hkeys[s] = 0;
    hcnt[s] = 0;
  }
  __syncthreads();
  u32 err = 0;
  unsigned long long failed = 0;
  for (;;) {
    if (threadIdx.x == 0) *chunk = atomicAdd(work, (unsigned long long)TC_CHUNK);
    __syncthreads();
    const u64 base = *chunk;
    __syncthreads();
    if (base >= total) break;
    for (u32 j = 0; j < TC_CHUNK; j += TcK::THREADS) {
      const u64 idx = base + j + threadIdx.x;
      u64 key = 0;
      if (idx < total) {
        key = tc_classify(tc_enum_mask(lo + idx, flags, TcK::D), S, err);
        failed += key == 0;
      }
      tc_hist_add<TcK::HASH>(key, hkeys, hcnt, gkeys, gcnt, gslots, gerr);
    }
  }
  __syncthreads();
  for (u32 s = threadIdx.x; s < TcK::HASH; s += TcK::THREADS)
    if (hkeys[s]) tc_global_add(gkeys, gcnt, gslots, gerr, hkeys[s], hcnt[s]);
  if (err) atomicOr(gerr, err);
  if (failed) atomicAdd(gfailed, failed);
}

// Exhaustive sweep of whole middle-row blocks: masks (h << oshift) |
// (t << ishift) for h in [hi0, hi0 + n_hi) (with TS_ENUM_ORBITS in flags,
// h = the block's high part, tc_orbit_high) and every t < 32 * ireps.  Each
// warp takes one h at a time; the two half-diamonds depend on h only and are
// swept once, then every lane classifies ireps middle-row patterns
// (tc_sweep_amortised).
extern "C" __global__ void __launch_bounds__(TcK::THREADS, TcK::MINB)
    tc_enumerate_blocks(u64 hi0, u64 n_hi, u32 oshift, u32 ishift, u32 ireps, u32 flags,
                        u64 *gkeys, unsigned long long *gcnt, u64 gslots, u32 *gerr,
                        unsigned long long *gfailed, unsigned long long *work, u32 *gscr) {
  extern __shared__ __align__(16) u32 tc_smem[];
  u64 *hkeys = reinterpret_cast<u64 *>(tc_smem + TC_SMEM_SCRATCH);
  unsigned long long *hcnt = reinterpret_cast<unsigned long long *>(hkeys + TcK::HASH);
  const TcScratch<TcK> S = tc_scratch(tc_smem, gscr);
  for (u32 s = threadIdx.x; s < TcK::HASH; s += TcK::THREADS) {
    hkeys[s] = 0;
    hcnt[s] = 0;
  }
  __syncthreads();
  const u32 lane = threadIdx.x & 31u;
  u32 err = 0;
  unsigned long long failed = 0;
  for (;;) {
    unsigned long long h = 0;
    if (lane == 0) h = atomicAdd(work, 1ull);
    h = __shfl_sync(0xffffffffu, h, 0);
    if (h >= n_hi) break;
    // the orbit sweep's blocks: block index -> high part with the pivots zero
    const u64 hh = (flags & 8u) ? tc_orbit_high(hi0 + h, flags) : hi0 + h;
    tc_sweep_amortised(hh << oshift, ishift, ireps, S, err, hkeys, hcnt, gkeys, gcnt, gslots, gerr,
                       failed);
  }
  __syncthreads();
  for (u32 s = threadIdx.x; s < TcK::HASH; s += TcK::THREADS)
    if (hkeys[s]) tc_global_add(gkeys, gcnt, gslots, gerr, hkeys[s], hcnt[s]);
  if (err) atomicOr(gerr, err);
  if (failed) atomicAdd(gfailed, failed);
}
