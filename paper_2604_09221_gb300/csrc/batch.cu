// batch.cu -- many triangulations of mixed degree in one graph launch.
//
// A batch is a list of jobs (triangulation, number of sign vectors, splitmix64
// stream of the sign vectors, optional code output).  For each degree present
// the batch runs ONE persistent kernel over all jobs of that degree: blocks
// pull (job, chunk) work items from a counter, re-stage a job's tables into
// shared memory with cp.async.bulk when the job changes, generate the sign
// vectors on the device, classify them with the table-driven sweep
// (Algorithm 1) and add the codes to the job's own device hash histogram
// (warp-aggregated atomics).  The per-degree kernels run on forked streams
// inside one CUDA graph that is captured on the first run and replayed after;
// each degree has its own tile shape (threads per block, instances per work
// item, scratch in shared or global memory), which ts_batch_set_tile
// changes (the autotuner's knob).
//
// A degree group with many sign vectors (or whose triangulations ask for
// TS_KERNEL_SPECIALIZED) runs specialised code instead: its persistent
// kernel tcj_jobs (jit.cpp) calls, per job, the straight-line sweep generated
// for that job's triangulation; all of the batch's objects are compiled in
// parallel at creation and linked per degree.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "engine.h"
#include "tc_layout.h"
#include "tc_table_sweep.cuh"

namespace tcurve {
namespace {

constexpr long kWaitIters = 1L << 22;

// Largest table of degree d: 2V + |E(T^diamond)| words, V = 2d^2 + 2d + 1 and
// |E(T^diamond)| = 6d^2 + 2d, padded to 16 bytes.
constexpr size_t max_table_bytes(int d) {
  return (size_t)(((10 * d * d + 6 * d + 2) + 3) & ~3) * 4;
}

// Degree-D_ kernel with T_ threads per block; per-thread scratch in shared
// memory, or (G_) in global memory, L1/L2-resident.
template <int D_, int T_, bool G_>
struct JobK : TcTableK<D_, T_, true> {
  static constexpr bool fits = JobK::L.ok && (max_table_bytes(D_) + 127) / 128 * 128 + 128 +
                                                     (G_ ? 0 : (size_t)JobK::WORDS * 4 * T_) <=
                                                 227 * 1024;
};

struct DevJob {
  const u32 *tab;
  u64 n;              // sign vectors
  u64 base;           // splitmix64 counter base of the sign vectors
  u64 *codes;         // per-instance codes, code_words each (or null)
  u64 *hkeys;         // job histogram (open addressing, code_words per key, 0 = empty)
  unsigned long long *hcnt;
  u64 hslots;
  u64 chunk0;         // first work item of the job
  u32 fn, pad;        // specialised groups: index of the job's function in the module
};
static_assert(sizeof(DevJob) == 72, "the job table layout of the generated batch kernels");

// Degree groups of at least this many sign vectors run specialised code
// (TS_KERNEL_AUTO): the compile at creation (about a second per
// triangulation, in parallel) pays for itself.
constexpr uint64_t kJitGroupMin = 1ull << 22;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

template <int D, int T, bool G>
__global__ void __launch_bounds__(T)
    jobs_kernel(const DevJob *__restrict__ jobs, u32 njobs, u64 total_items, u32 chunk,
                u32 table_words, u32 off_fan, u32 off_vext, unsigned long long *work, u32 *err_word,
                unsigned long long *failed_word, u32 *gscratch) {
  typedef JobK<D, T, G> K;
  extern __shared__ __align__(128) uint8_t smem[];
  u32 *tab = reinterpret_cast<u32 *>(smem);
  const size_t toff = ((size_t)table_words * 4 + 127) / 128 * 128;
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem + toff);
  unsigned long long *slot = reinterpret_cast<unsigned long long *>(smem + toff + 64);
  const TcScratch<K> S{(G ? gscratch + (size_t)blockIdx.x * K::WORDS * T
                         : reinterpret_cast<u32 *>(smem + toff + 128)) +
                        threadIdx.x};
  // global scratch: the label slots of the sweep in shared memory
  u32 *const ls = G ? reinterpret_cast<u32 *>(smem + toff + 128) + threadIdx.x : nullptr;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1u));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const u32 lane = threadIdx.x & 31u;
  u32 cur = 0xFFFFFFFFu, phase = 0, err = 0;
  unsigned long long failed = 0;
  for (;;) {
    if (threadIdx.x == 0) *slot = atomicAdd(work, 1ull);
    __syncthreads();
    const u64 c = *slot;
    __syncthreads();  // also: every thread is done with the previous job's tables
    if (c >= total_items) break;
    u32 lo = 0, hi = njobs;  // the job holding item c: last j with chunk0 <= c
    while (hi - lo > 1) {
      const u32 mid = (lo + hi) / 2;
      if (jobs[mid].chunk0 <= c) lo = mid; else hi = mid;
    }
    const u32 j = lo;
    if (j != cur) {  // stage the job's tables (cp.async.bulk, bounded wait)
      if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                     "r"(table_words * 4u) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                "r"(smem_u32(tab)), "l"(jobs[j].tab), "r"(table_words * 4u), "r"(smem_u32(bar))
            : "memory");
      }
      bool ok = false;
      for (long it = 0; it < kWaitIters && !ok; ++it) {
        uint32_t r;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}"
            : "=r"(r) : "r"(smem_u32(bar)), "r"(phase) : "memory");
        ok = r != 0;
      }
      if (__syncthreads_or(!ok)) {
        if (threadIdx.x == 0) atomicOr(err_word, kErrTimeout);
        for (long it = 0; it < kWaitIters && !ok; ++it) {
          uint32_t r;
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
              " selp.u32 %0, 1, 0, p;\n}"
              : "=r"(r) : "r"(smem_u32(bar)), "r"(phase) : "memory");
          ok = r != 0;
        }
        return;
      }
      phase ^= 1u;
      cur = j;
      if (G) {  // label slots in shared memory, found by the fan entries' offsets
        tc_fan_to_offsets(tab + off_fan, off_vext - off_fan, TcScratch<K>::EPW, K::LBYTES, T,
                          threadIdx.x, T);
        __syncthreads();
      }
    }
    const DevJob J = jobs[j];
    const u64 first = (c - J.chunk0) * (u64)chunk;
    for (u32 k = 0; k < chunk; k += T) {
      const u64 idx = first + k + threadIdx.x;
      TcCodeOut<K> key{};
      if (idx < J.n) {
        // the sign vector of counter base + idx, as ts_splitmix_masks writes it
        TcSig<K::W> sg;
#pragma unroll
        for (u32 w = 0; w < K::W; ++w) sg.w[w] = tc_splitmix64((J.base + idx) * K::W + w);
        sg.w[K::W - 1] &= tc_top_mask(K::NPOINTS, K::W);
        key = tc_table_classify<K, G>(sg, tab, off_fan, off_vext, S, err, ls);
        u64 any = 0;
#pragma unroll
        for (u32 w = 0; w < K::CW; ++w) {
          any |= key.w[w];
          if (J.codes) J.codes[idx * K::CW + w] = key.w[w];
        }
        failed += any == 0;
      }
      if constexpr (K::CW == 1) {
        const unsigned peers = __match_any_sync(0xffffffffu, key.w[0]);
        if (key.w[0] != 0 && lane == (u32)(__ffs(peers) - 1))
          tc_global_add(J.hkeys, J.hcnt, J.hslots, err_word, key.w[0],
                        (unsigned long long)__popc(peers));
      } else {
        tc_hist_add_wide<K::CW>(key.w, J.hkeys, J.hcnt, J.hslots, err_word);
      }
    }
  }
  if (err) atomicOr(err_word, err);
  if (failed) atomicAdd(failed_word, failed);
}

// (degree, threads, scratch) -> kernel; only instantiations whose block fits.
typedef void (*JobsFn)(const DevJob *, u32, u64, u32, u32, u32, u32, unsigned long long *, u32 *,
                       unsigned long long *, u32 *);

template <int D, int T, bool G>
JobsFn jobs_fn() {
  if constexpr (JobK<D, T, G>::fits) return jobs_kernel<D, T, G>;
  else return nullptr;
}

template <int D, bool G>
JobsFn jobs_fn_tg(int t) {
  switch (t) {
    case 32: return jobs_fn<D, 32, G>();
    case 64: return jobs_fn<D, 64, G>();
    case 96: return jobs_fn<D, 96, G>();
    case 128: return jobs_fn<D, 128, G>();
    case 192: return jobs_fn<D, 192, G>();
    case 256: return jobs_fn<D, 256, G>();
    default: return nullptr;
  }
}

template <int D>
JobsFn jobs_fn_t(int t, bool g) {
  return g ? jobs_fn_tg<D, true>(t) : jobs_fn_tg<D, false>(t);
}

JobsFn jobs_fn_dt(int d, int t, bool g) {
  switch (d) {
    case 1: return jobs_fn_t<1>(t, g);
    case 2: return jobs_fn_t<2>(t, g);
    case 3: return jobs_fn_t<3>(t, g);
    case 4: return jobs_fn_t<4>(t, g);
    case 5: return jobs_fn_t<5>(t, g);
    case 6: return jobs_fn_t<6>(t, g);
    case 7: return jobs_fn_t<7>(t, g);
    case 8: return jobs_fn_t<8>(t, g);
    case 9: return jobs_fn_t<9>(t, g);
    case 10: return jobs_fn_t<10>(t, g);
    case 11: return jobs_fn_t<11>(t, g);
    case 12: return jobs_fn_t<12>(t, g);
    case 13: return jobs_fn_t<13>(t, g);
    case 14: return jobs_fn_t<14>(t, g);
    case 15: return jobs_fn_t<15>(t, g);
    case 16: return jobs_fn_t<16>(t, g);
    default: return nullptr;
  }
}

// ls_words: label-slot words per thread (global scratch: kept in shared memory)
size_t jobs_smem(int d, int t, uint32_t table_words, uint32_t ls_words, bool g) {
  const TcLayout L = tc_layout(d, true, t);
  return ((size_t)table_words * 4 + 127) / 128 * 128 + 128 +
         (g ? (size_t)ls_words * 4 * t : (size_t)L.words * 4 * t);
}

size_t scratch_words(int d, int t) { return (size_t)tc_layout(d, true, t).words * t; }

ts_status cuda_st(cudaError_t e) {
  if (e == cudaSuccess) return TS_OK;
  return e == cudaErrorMemoryAllocation ? TS_ENOMEM : TS_ECUDA;
}

}  // namespace
}  // namespace tcurve

using namespace tcurve;

struct ts_batch {
  struct Group {  // all jobs of one degree
    int d = 0, threads = 64, chunk = 1024;
    bool global = false;        // per-thread scratch in global memory
    std::shared_ptr<JitJobsModule> jit;  // specialised kernel (null: table-driven)
    std::string jit_log;        // why the specialised kernel could not be built
    JobsFn fn = nullptr;        // the kernel of this tile, its launch shape
    size_t smem = 0;
    unsigned grid = 1;
    u32 *scratch = nullptr;     // global scratch (grid x threads x words)
    size_t scratch_bytes = 0;
    uint32_t table_words = 0, off_fan = 0, off_vext = 0;
    uint32_t ls_words = 0;      // label-slot words per thread (largest of the group's tables)
    std::vector<int> jobs;      // indices into the batch's job list
    DevJob *d_jobs = nullptr;   // device job table (sorted as `jobs`)
    uint64_t items = 0;
    unsigned long long *d_work = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    int fwarp = 0;              // fused launch: warp (1) or thread (0) per instance
    int fchunk = kFusedThreads * 8;  // fused launch: sign vectors per work item
  };
  std::vector<DevJob> jobs;  // host copies (chunk0 per group)
  std::vector<int> degree, cws;       // degree and code words of every job
  std::vector<size_t> kofs;           // first key word of every job's histogram
  std::vector<size_t> cofs;           // first count of every job's histogram
  std::vector<uint64_t> jslots;       // slots of every job's histogram
  size_t key_words = 0, count_words = 0;
  std::vector<Group> groups;
  uint64_t *d_keys = nullptr;  // per job: slots x code_words
  unsigned long long *d_counts = nullptr;
  uint32_t *d_err = nullptr;
  unsigned long long *d_failed = nullptr;
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  int device = 0;
  std::vector<ts_tri *> tris;  // triangulation of every job
  std::vector<const uint64_t *> signs;  // caller sign vectors of every job (null: splitmix64)
  bool serial = false;         // degree groups one after the other (else concurrent streams)
  // fused launch (ts_batch_set_fused): one persistent kernel over all jobs
  bool fused = false;
  FusedJob *d_fjobs = nullptr;  // jobs sorted by degree
  uint64_t fitems = 0;
  int ftier = -1;
  unsigned fgrid = 1;
  size_t fsmem = 0;
  uint32_t ftoff = 0, fls = 0, fws = 0;
  uint32_t *fscratch = nullptr;
  size_t fscratch_bytes = 0;
  unsigned long long *d_fwork = nullptr;
};

namespace {

cudaError_t upload_group(ts_batch *b, ts_batch::Group &g) {
  std::vector<DevJob> dj;
  uint64_t items = 0;
  for (int j : g.jobs) {
    DevJob x = b->jobs[j];
    x.chunk0 = items;
    items += (x.n + g.chunk - 1) / g.chunk;
    dj.push_back(x);
  }
  g.items = items;
  if (!g.d_jobs) {
    cudaError_t e = cudaMalloc(&g.d_jobs, sizeof(DevJob) * dj.size());
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpy(g.d_jobs, dj.data(), sizeof(DevJob) * dj.size(), cudaMemcpyHostToDevice);
}

// Kernel, shared memory, persistent grid and global scratch of the group's
// tile (host work only: done at creation and on a tile change, never while a
// stream is being captured).
cudaError_t prepare_group(ts_batch::Group &g) {
  int per_sm = 0, sms = 0, dev = 0;
  cudaError_t e = cudaSuccess;
  if (g.jit) {  // specialised: 128-thread blocks, global scratch, grid from its occupancy
    g.fn = nullptr;
    g.smem = 0;
    per_sm = jit_jobs_blocks_per_sm(*g.jit);
  } else {
    g.fn = jobs_fn_dt(g.d, g.threads, g.global);
    if (!g.fn) return cudaErrorInvalidConfiguration;
    g.smem = jobs_smem(g.d, g.threads, g.table_words, g.ls_words, g.global);
    e = cudaFuncSetAttribute((const void *)g.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)g.smem);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)g.fn, g.threads, g.smem);
    if (e != cudaSuccess) return e;
  }
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t cap = (uint64_t)per_sm * sms;
  g.grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(cap, g.items));
  if (g.global) {
    const size_t need = g.jit ? (size_t)g.grid * jit_jobs_slab_bytes(*g.jit)
                              : (size_t)g.grid * scratch_words(g.d, g.threads) * 4;
    if (need > g.scratch_bytes) {
      if (g.scratch) cudaFree(g.scratch);
      g.scratch = nullptr;
      g.scratch_bytes = 0;
      e = cudaMalloc(&g.scratch, need);
      if (e != cudaSuccess) return e;
      g.scratch_bytes = need;
    }
  }
  return cudaSuccess;
}

cudaError_t launch_group(ts_batch *b, ts_batch::Group &g, cudaStream_t st) {
  if (!g.fn && !g.jit) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaMemsetAsync(g.d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  if (g.jit)
    return jit_jobs_launch(*g.jit, g.grid, g.d_jobs, (uint32_t)g.jobs.size(), g.items,
                           (uint32_t)g.chunk, g.d_work, b->d_err, b->d_failed, g.scratch, st);
  g.fn<<<g.grid, g.threads, g.smem, st>>>(g.d_jobs, (u32)g.jobs.size(), g.items, (u32)g.chunk,
                                          g.table_words, g.off_fan, g.off_vext, g.d_work, b->d_err,
                                          b->d_failed, g.scratch);
  return cudaGetLastError();
}

// Job table, kernel tier, shared memory, persistent grid and global scratch
// of the fused launch (host work only, never while a stream is captured):
// the jobs in degree order, each with its degree's tile; the tier of the
// largest degree, or the warp tier when a degree has a warp tile.
cudaError_t prepare_fused(ts_batch *b) {
  std::vector<const ts_batch::Group *> gs;
  for (const auto &g : b->groups) gs.push_back(&g);
  std::sort(gs.begin(), gs.end(), [](const ts_batch::Group *x, const ts_batch::Group *y) {
    return x->d < y->d;
  });
  std::vector<FusedJob> fj;
  uint64_t items = 0;
  uint32_t maxtab = 0, wsw = 0, lsw = 0;
  int dmax = 0;
  bool anywarp = false;
  for (const ts_batch::Group *g : gs) {
    for (int j : g->jobs) {
      const DevJob &dj = b->jobs[j];
      const ts_tri *t = b->tris[j];
      FusedJob x{};
      x.n = dj.n;
      x.base = dj.base;
      x.codes = dj.codes;
      x.hkeys = dj.hkeys;
      x.hcnt = dj.hcnt;
      x.hslots = dj.hslots;
      x.item0 = items;
      x.signs = reinterpret_cast<const unsigned long long *>(b->signs[j]);
      x.d = (uint32_t)g->d;
      x.chunk = (uint32_t)g->fchunk;
      x.warp = (uint32_t)g->fwarp;
      if (x.warp) {
        x.tab = t->d_wtables;
        x.tab_words = t->wlay.words;
        x.wl = t->wlay;
        wsw = std::max(wsw, fused_warp_words(g->d));
        anywarp = true;
      } else {
        x.tab = t->d_tables;
        x.tab_words = t->lay.words;
        x.off_fan = t->lay.off_fan;
        x.off_vext = t->lay.off_vext;
        const uint32_t epw = tc_layout(g->d, true, kFusedThreads).epw;
        lsw = std::max(lsw, (t->lay.nslots + epw - 1) / epw);
      }
      maxtab = std::max(maxtab, x.tab_words);
      items += (x.n + x.chunk - 1) / x.chunk;
      dmax = std::max(dmax, g->d);
      fj.push_back(x);
    }
  }
  const int tier = anywarp ? kFusedWarpTier : fused_tier(dmax);
  if (tier < 0 || fj.empty()) return cudaErrorInvalidConfiguration;
  const uint32_t toff = (maxtab * 4 + 127) / 128 * 128;
  const size_t smem = (size_t)toff + 128 + (size_t)kFusedThreads * lsw * 4 +
                      (anywarp ? (size_t)4 * wsw * 4 : 0);
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  int per_sm = 0, sms = 0, dev = 0;
  cudaError_t e = fused_occupancy(tier, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const uint64_t cap = (uint64_t)per_sm * sms;
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(cap, items));
  const size_t need = (size_t)grid * kFusedThreads * fused_slab_words(tier) * 4;
  if (need > b->fscratch_bytes) {
    if (b->fscratch) cudaFree(b->fscratch);
    b->fscratch = nullptr;
    b->fscratch_bytes = 0;
    e = cudaMalloc(&b->fscratch, need);
    if (e != cudaSuccess) return e;
    b->fscratch_bytes = need;
  }
  if (!b->d_fjobs) {
    e = cudaMalloc(&b->d_fjobs, sizeof(FusedJob) * fj.size());
    if (e != cudaSuccess) return e;
  }
  if (!b->d_fwork) {
    e = cudaMalloc(&b->d_fwork, sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
  }
  e = cudaMemcpy(b->d_fjobs, fj.data(), sizeof(FusedJob) * fj.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  b->fitems = items;
  b->ftier = tier;
  b->fgrid = grid;
  b->fsmem = smem;
  b->ftoff = toff;
  b->fls = lsw;
  b->fws = wsw;
  return cudaSuccess;
}

// The whole batch as stream work on `st`: clear, then either the fused
// launch or fork, one kernel per degree, join.
cudaError_t enqueue(ts_batch *b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_keys, 0, b->key_words * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counts, 0, b->count_words * 8, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, 4, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_failed, 0, 8, st);
  if (b->fused) {  // one persistent kernel for every job of every degree
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_fwork, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess)
      e = fused_launch(b->ftier, b->fgrid, b->fsmem, b->ftoff, b->fls, b->fws, b->d_fjobs,
                       (uint32_t)b->jobs.size(), b->fitems, b->d_fwork, b->d_err, b->d_failed,
                       b->fscratch, st);
    return e;
  }
  if (b->serial) {  // one degree after the other, each persistent kernel on the whole GPU
    for (auto &g : b->groups)
      if (e == cudaSuccess) e = launch_group(b, g, st);
    return e;
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->fork, st);
  for (auto &g : b->groups) {
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g.stream, b->fork, 0);
    if (e == cudaSuccess) e = launch_group(b, g, g.stream);
    if (e == cudaSuccess) e = cudaEventRecord(g.done, g.stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, g.done, 0);
  }
  return e;
}

// Table-driven tile of a group at creation: global scratch from d = 7 with
// 128-thread blocks, shared scratch below (64-thread blocks from d = 8).
void table_defaults(ts_batch::Group &g) {
  g.jit.reset();
  g.global = g.d >= kGlobalScratchFrom;
  g.threads = g.global ? 128 : (g.d >= 8 ? 64 : 128);
  while (g.threads > 32 && !jobs_fn_dt(g.d, g.threads, g.global)) g.threads -= 32;
  g.chunk = g.threads * 8;
}

// TS_KERNEL_AUTO at creation: specialised code for groups of at least
// kJitGroupMin sign vectors up to degree kMaxBatchSpecialized, or when a
// triangulation of the group asks for it; never when one asks for tables.
bool wants_specialised(const ts_batch *b, const ts_batch::Group &g) {
  bool table = false, forced = false;
  uint64_t total = 0;
  for (int j : g.jobs) {
    table |= b->tris[j]->kernel == TS_KERNEL_TABLE;
    forced |= b->tris[j]->kernel == TS_KERNEL_SPECIALIZED;
    total += b->jobs[j].n;
  }
  return !table && (forced || (total >= kJitGroupMin && g.d <= kMaxBatchSpecialized));
}

// Build the specialised modules of the groups `gids` at once (one parallel
// compile): every job gets the index of its triangulation's function (one
// per distinct ts_tri of the group).  A group whose module cannot be built
// gets the table-driven tile and the log.  Returns false if any failed.
bool make_specialised(ts_batch *b, const std::vector<int> &gids) {
  if (gids.empty()) return true;
  std::vector<std::vector<const Diamond *>> want;
  std::vector<int> min_blocks;
  for (int gi : gids) {
    auto &g = b->groups[gi];
    std::map<const ts_tri *, uint32_t> fn;
    std::vector<const Diamond *> dias;
    int occ = 0;  // a register budget asked for with ts_set_occupancy
    for (int j : g.jobs) {
      occ = std::max(occ, b->tris[j]->occupancy);
      auto it = fn.find(b->tris[j]);
      if (it == fn.end()) {
        it = fn.emplace(b->tris[j], (uint32_t)dias.size()).first;
        dias.push_back(&b->tris[j]->dia);
      }
      b->jobs[j].fn = it->second;
    }
    want.push_back(dias);
    min_blocks.push_back(occ);
  }
  std::vector<std::shared_ptr<JitJobsModule>> mods;
  std::vector<std::string> logs;
  jit_jobs_build(want, min_blocks, &mods, &logs);
  bool all = true;
  for (size_t k = 0; k < gids.size(); ++k) {
    auto &g = b->groups[gids[k]];
    if (k < mods.size() && mods[k]) {
      g.jit = mods[k];
      g.jit_log.clear();
      g.global = true;
      g.threads = jit_jobs_threads();
      g.chunk = g.threads * 16;
    } else {
      table_defaults(g);
      g.jit_log = k < logs.size() && !logs[k].empty() ? logs[k] : "specialised batch kernel unavailable";
      all = false;
    }
  }
  return all;
}

}  // namespace

extern "C" {

ts_status ts_batch_create(int njobs, ts_tri *const *tris, const uint64_t *counts,
                          const uint64_t *bases, uint64_t *const *code_outputs,
                          uint64_t hist_capacity, ts_batch **out) {
  if (!out || njobs < 1 || !tris || !counts || !bases || hist_capacity == 0 ||
      hist_capacity > (1u << 20))
    return TS_EINVAL;
  *out = nullptr;
  ts_batch *b = new (std::nothrow) ts_batch();
  if (!b) return TS_ENOMEM;
  cudaError_t e = cudaGetDevice(&b->device);
  for (int j = 0; j < njobs; ++j) {
    if (!tris[j] || counts[j] > (1ull << 62)) {  // counts: room for the work-item arithmetic
      ts_batch_free(b);
      return TS_EINVAL;
    }
    // a job of n sign vectors has at most n distinct schemes
    const uint64_t cap = std::min<uint64_t>(hist_capacity, std::max<uint64_t>(counts[j], 1));
    uint64_t s = 16;
    while (s < 2 * cap) s <<= 1;
    b->jslots.push_back(s);
    b->kofs.push_back(b->key_words);
    b->cofs.push_back(b->count_words);
    b->cws.push_back(tris[j]->cw);
    b->key_words += s * tris[j]->cw;
    b->count_words += s;
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->d_keys, b->key_words * 8);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counts, b->count_words * 8);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_err, 4);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_failed, 8);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  std::map<int, int> gi;
  for (int j = 0; j < njobs && e == cudaSuccess; ++j) {
    const ts_tri *t = tris[j];
    if (t->device != b->device) {
      ts_batch_free(b);
      return TS_EINVAL;
    }
    DevJob x{};
    x.tab = t->d_tables;
    x.n = counts[j];
    x.base = bases[j];
    x.codes = code_outputs ? reinterpret_cast<u64 *>(code_outputs[j]) : nullptr;
    x.hkeys = reinterpret_cast<u64 *>(b->d_keys + b->kofs[j]);
    x.hcnt = b->d_counts + b->cofs[j];
    x.hslots = b->jslots[j];
    b->jobs.push_back(x);
    b->degree.push_back(t->d);
    b->tris.push_back(tris[j]);
    b->signs.push_back(nullptr);
    if (!gi.count(t->d)) {
      gi[t->d] = (int)b->groups.size();
      ts_batch::Group g;
      g.d = t->d;
      g.table_words = t->lay.words;
      g.off_fan = t->lay.off_fan;
      g.off_vext = t->lay.off_vext;
      table_defaults(g);
      b->groups.push_back(g);
    }
    auto &grp = b->groups[gi[t->d]];
    grp.jobs.push_back(j);
    grp.table_words = std::max(grp.table_words, t->lay.words);
    const uint32_t epw = (uint32_t)tc_layout(t->d, true, 32).epw;
    grp.ls_words = std::max(grp.ls_words, (t->lay.nslots + epw - 1) / epw);
  }
  if (e == cudaSuccess) {
    std::vector<int> spec;
    for (size_t gi = 0; gi < b->groups.size(); ++gi)
      if (wants_specialised(b, b->groups[gi])) spec.push_back((int)gi);
    make_specialised(b, spec);
  }
  for (auto &g : b->groups) {
    if (e == cudaSuccess) e = cudaMalloc(&g.d_work, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = upload_group(b, g);
    if (e == cudaSuccess) e = prepare_group(g);
  }
  if (e != cudaSuccess) {
    ts_batch_free(b);
    return cuda_st(e);
  }
  *out = b;
  return TS_OK;
}

void ts_batch_free(ts_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto &g : b->groups) {
    if (g.d_jobs) cudaFree(g.d_jobs);
    if (g.d_work) cudaFree(g.d_work);
    if (g.scratch) cudaFree(g.scratch);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.done) cudaEventDestroy(g.done);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->d_fjobs) cudaFree(b->d_fjobs);
  if (b->fscratch) cudaFree(b->fscratch);
  if (b->d_fwork) cudaFree(b->d_fwork);
  if (b->d_keys) cudaFree(b->d_keys);
  if (b->d_counts) cudaFree(b->d_counts);
  if (b->d_err) cudaFree(b->d_err);
  if (b->d_failed) cudaFree(b->d_failed);
  delete b;
}

ts_status ts_batch_set_tile(ts_batch *b, int d, int threads, int chunk, int scratch) {
  if (!b || threads < 32 || threads % 32 || chunk < threads || chunk % threads ||
      scratch < TS_SCRATCH_AUTO || scratch > TS_SCRATCH_GLOBAL)
    return TS_EINVAL;
  for (auto &g : b->groups) {
    if (g.d != d) continue;
    bool global = scratch == TS_SCRATCH_AUTO ? d >= kGlobalScratchFrom : scratch == TS_SCRATCH_GLOBAL;
    if (g.jit) {  // specialised: the block size and global scratch are fixed at compile time
      if (threads != jit_jobs_threads() || scratch == TS_SCRATCH_SHARED) return TS_EINVAL;
      global = true;
    } else if (!jobs_fn_dt(d, threads, global)) {
      return TS_EINVAL;  // block does not fit shared memory
    }
    // runs already launched (graph launches included) read the job table and
    // the scratch that this call rewrites or frees: let them finish first
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_st(e);
    g.threads = threads;
    g.chunk = chunk;
    g.global = global;
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    e = upload_group(b, g);
    if (e == cudaSuccess) e = prepare_group(g);
    return cuda_st(e);
  }
  return TS_EINVAL;
}

ts_status ts_batch_set_kernel(ts_batch *b, int d, int kind) {
  if (!b || kind < TS_KERNEL_AUTO || kind > TS_KERNEL_SPECIALIZED) return TS_EINVAL;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    auto &g = b->groups[gi];
    if (g.d != d) continue;
    // runs already launched read the job table and scratch rewritten here
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_st(e);
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    bool ok = true;
    const bool spec = kind == TS_KERNEL_SPECIALIZED || (kind == TS_KERNEL_AUTO && wants_specialised(b, g));
    if (!spec) table_defaults(g);
    else if (!g.jit) ok = make_specialised(b, {(int)gi});
    e = upload_group(b, g);
    if (e == cudaSuccess) e = prepare_group(g);
    if (e != cudaSuccess) return cuda_st(e);
    return ok ? TS_OK : TS_ECUDA;
  }
  return TS_EINVAL;
}

ts_status ts_batch_set_serial(ts_batch *b, int serial) {
  if (!b || serial < 0 || serial > 1) return TS_EINVAL;
  if (b->serial != (serial != 0) && b->exec) {
    cudaError_t e = cudaDeviceSynchronize();  // a graph launched before may still run
    if (e != cudaSuccess) return cuda_st(e);
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->serial = serial != 0;
  return TS_OK;
}

ts_status ts_batch_set_fused(ts_batch *b, int fused) {
  if (!b || fused < 0 || fused > 1) return TS_EINVAL;
  if (b->fused == (fused != 0)) return TS_OK;
  cudaError_t e = cudaDeviceSynchronize();  // a run launched before may still read the tables
  if (e != cudaSuccess) return cuda_st(e);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (fused) {
    e = prepare_fused(b);
    if (e != cudaSuccess) return cuda_st(e);
  }
  b->fused = fused != 0;
  return TS_OK;
}

ts_status ts_batch_set_fused_tile(ts_batch *b, int d, int kind, int chunk) {
  if (!b || chunk < kFusedThreads || chunk % kFusedThreads || chunk > (1 << 24) ||
      (kind != TS_KERNEL_AUTO && kind != TS_KERNEL_TABLE && kind != TS_KERNEL_WARP) ||
      (kind == TS_KERNEL_WARP && d < kFusedWarpFrom))
    return TS_EINVAL;
  for (auto &g : b->groups) {
    if (g.d != d) continue;
    cudaError_t e = cudaDeviceSynchronize();  // runs already launched read the job table
    if (e != cudaSuccess) return cuda_st(e);
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
    const int ow = g.fwarp, oc = g.fchunk;
    g.fwarp = kind == TS_KERNEL_WARP ? 1 : 0;
    g.fchunk = chunk;
    if (b->fused) {
      e = prepare_fused(b);
      if (e != cudaSuccess) {  // keep the previous, prepared tile
        g.fwarp = ow;
        g.fchunk = oc;
        const cudaError_t e2 = prepare_fused(b);
        return e2 != cudaSuccess ? cuda_st(e2) : TS_EINVAL;
      }
    }
    return TS_OK;
  }
  return TS_EINVAL;
}

ts_status ts_batch_set_signs(ts_batch *b, int job, const uint64_t *signs) {
  if (!b || job < 0 || job >= (int)b->jobs.size()) return TS_EINVAL;
  if (b->signs[job] == signs) return TS_OK;
  cudaError_t e = cudaDeviceSynchronize();  // a run launched before may still read the job table
  if (e != cudaSuccess) return cuda_st(e);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  b->signs[job] = signs;
  if (b->fused) {
    e = prepare_fused(b);
    if (e != cudaSuccess) return cuda_st(e);
  }
  return TS_OK;
}

ts_status ts_batch_run(ts_batch *b, int use_graph, void *stream) {
  if (!b) return TS_EINVAL;
  if (!b->fused)  // the degree-group kernels draw their sign vectors: caller inputs need the fused launch
    for (const uint64_t *p : b->signs)
      if (p) return TS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (!use_graph) return cuda_st(enqueue(b, st));
  if (!b->exec) {
    cudaStream_t cap = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    cudaGraph_t graph = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t e2 = enqueue(b, cap);
      e = cudaStreamEndCapture(cap, &graph);
      if (e2 != cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (e != cudaSuccess) return cuda_st(e);
  }
  return cuda_st(cudaGraphLaunch(b->exec, st));
}

ts_status ts_batch_info(const ts_batch *b, int d, ts_batch_group_info *info, char *log,
                        size_t len) {
  if (!b || !info) return TS_EINVAL;
  for (const auto &g : b->groups) {
    if (g.d != d) continue;
    ts_batch_group_info x{};
    if (b->fused) {  // the degree's tile in the one fused launch
      x.kernel = g.fwarp ? TS_KERNEL_WARP : TS_KERNEL_TABLE;
      x.threads = kFusedThreads;
      x.chunk = g.fchunk;
      x.scratch = g.fwarp ? TS_SCRATCH_SHARED : TS_SCRATCH_GLOBAL;
      x.grid = (int)b->fgrid;
      fused_attrs(b->ftier, &x.registers, &x.local_bytes);
      fused_occupancy(b->ftier, b->fsmem, &x.blocks_per_sm);
      *info = x;
      if (log && len) log[0] = 0;
      return TS_OK;
    }
    x.kernel = g.jit ? TS_KERNEL_SPECIALIZED : TS_KERNEL_TABLE;
    x.threads = g.threads;
    x.chunk = g.chunk;
    x.scratch = g.global ? TS_SCRATCH_GLOBAL : TS_SCRATCH_SHARED;
    x.grid = (int)g.grid;
    if (g.jit) {
      jit_jobs_attrs(*g.jit, &x.registers, &x.local_bytes);
      x.blocks_per_sm = jit_jobs_blocks_per_sm(*g.jit);
    } else if (g.fn) {
      cudaFuncAttributes fa{};
      if (cudaFuncGetAttributes(&fa, (const void *)g.fn) == cudaSuccess) {
        x.registers = fa.numRegs;
        x.local_bytes = (int)fa.localSizeBytes;
      }
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&x.blocks_per_sm, (const void *)g.fn, g.threads,
                                                    g.smem);
    }
    *info = x;
    if (log && len) {
      const size_t n = std::min(len - 1, g.jit_log.size());
      std::memcpy(log, g.jit_log.data(), n);
      log[n] = 0;
    }
    return TS_OK;
  }
  return TS_EINVAL;
}

ts_status ts_batch_read(ts_batch *b, int job, uint64_t *codes, uint64_t *counts, uint64_t cap,
                        uint64_t *n_out, uint64_t *n_failed, void *stream) {
  if (!b || !n_out || job < 0 || job >= (int)b->jobs.size() || (cap && (!codes || !counts)))
    return TS_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  const int cw = b->cws[job];
  const uint64_t hs = b->jslots[job];
  std::vector<uint64_t> k(hs * cw);
  std::vector<unsigned long long> c(hs);
  uint32_t err = 0;
  unsigned long long failed = 0;
  if (e == cudaSuccess)
    e = cudaMemcpy(k.data(), b->d_keys + b->kofs[job], k.size() * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess)
    e = cudaMemcpy(c.data(), b->d_counts + b->cofs[job], hs * 8,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&err, b->d_err, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&failed, b->d_failed, 8, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_st(e);
  std::vector<uint64_t> idx;
  for (uint64_t s = 0; s < hs; ++s) {
    bool nz = false;
    for (int w = 0; w < cw; ++w) nz |= k[s * cw + w] != 0;
    if (nz) idx.push_back(s);
  }
  std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t x) {
    for (int w = cw - 1; w >= 0; --w)
      if (k[a * cw + w] != k[x * cw + w]) return k[a * cw + w] < k[x * cw + w];
    return false;
  });
  *n_out = idx.size();
  if (n_failed) *n_failed = failed;
  for (uint64_t i = 0; i < idx.size() && i < cap; ++i) {
    for (int w = 0; w < cw; ++w) codes[i * cw + w] = k[idx[i] * cw + w];
    counts[i] = c[idx[i]] & kCountMask;
  }
  if (idx.size() > cap) return TS_EOVERFLOW;
  if (err & kErrTimeout) return TS_ETIMEOUT;
  if (err & kErrOverflow) return TS_EOVERFLOW;
  if (err & kErrInternal) return TS_EINTERNAL;
  return TS_OK;
}

}  // extern "C"
