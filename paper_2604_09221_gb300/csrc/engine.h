// engine.h -- internal interface between the host library (host.cpp) and the
// CUDA kernels (kernels.cu).  Not part of the public ABI (include/tcurve.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tcurve.h"

namespace tcurve {

constexpr int kMaxDegree = 16;     // |A| <= 153: three sign words, four code words
constexpr int kMaxSpecialized = 9;  // triangulation-specialised kernels: one sign word
constexpr int kGlobalScratchFrom = 7;  // TS_SCRATCH_AUTO: table kernels use global scratch from here
constexpr int kMaxBatchSpecialized = 6;  // TS_KERNEL_AUTO: largest degree of specialised batch groups

// Count words of multi-word histograms carry two flags in their top bits
// (slot being written / key published); the count is the rest.
constexpr uint64_t kCountMask = (1ull << 62) - 1;

// Triangulation tables (32-bit words, format in tc_table_sweep.cuh): vdesc[V],
// fan[NF], vext[V] at the offsets below, vertex ids in the sweep order of
// T^diamond (host.cpp).
struct TableLayout {
  uint32_t V, NF;
  uint32_t off_vdesc, off_fan, off_vext;
  uint32_t words;   // padded to a multiple of 4 (16-byte TMA granule)
  uint32_t nslots;  // label slots the sweep uses (lab_slots)
};

// Tables of the warp-per-instance kernels (32-bit words, vertex ids in the
// sweep order of T^diamond): wv[V] = k(v) (8 bits) | c(v) << 8 | the length
// of v's fan (earlier neighbours) << 9 (7 bits) | the position of its first
// entry in wedge << 16; wedge[E] = u | link << 15 | v << 16 for the fan
// entries u of every vertex v in angular order (link: u, the entry before it
// and v span a triangle); wanti[2d] and wbedge[2d] = a | b << 16 for the
// antipodal pairs and one boundary edge of each antipodal pair of boundary
// edges.
struct WarpLayout {
  uint32_t V, E, nanti, nbedge;
  uint32_t off_v, off_e, off_anti, off_bedge;
  uint32_t words;  // padded to a multiple of 4
};
// Device error word bits.
enum : uint32_t {
  kErrInternal = 1u,   // invariant violated (root, tree, scratch)
  kErrOverflow = 2u,   // scheme beyond code width / hash table full
  kErrTimeout = 4u,    // bounded wait gave up
};

// The reflected triangulation T^diamond (Alg. 1, line 1) in sweep order:
// vertices sorted by (y, x); fan[v] = earlier neighbours of v in angular
// order, link[v][n] = 1 if fan[v][n-1], fan[v][n] and v span a triangle;
// k = lattice index and c = Eq. 2 parity constant of each vertex; anti =
// antipodal boundary pairs (v < w); bedge = one boundary edge of each
// antipodal pair of boundary edges.
struct Diamond {
  int d = 0, V = 0;
  std::vector<int> x, y, k, c;
  std::vector<std::vector<int>> fan, link;
  std::vector<std::pair<int, int>> anti, bedge;
};

struct JitModule;  // compiled specialised kernels (jit.cpp)

// Tables of the table-driven sweep (host.cpp; format in tc_runtime.cuh).
bool pack_diamond_tables(const Diamond &D, std::vector<uint32_t> &tables, TableLayout &lay);
// Tables of the warp-per-instance kernels (host.cpp; format at WarpLayout).
bool pack_warp_tables(const Diamond &D, std::vector<uint32_t> &tables, WarpLayout &lay);
// Label slot of every vertex in the table-driven sweep (a slot is reused once
// its vertex has no later reader) and, in *nslots, how many slots are used.
std::vector<int> lab_slots(const Diamond &D, int *nslots);

// Most joins vertex v can push in a sweep: one per run of same-sign fan
// entries after the first (a run starts at entry i when it has the vertex's
// sign and entry i-1 has not, or the two are not linked), plus its antipodal
// join.
int vertex_pushes(const Diamond &D, int v);
// Static flush schedule of the join list for vertices [v0, v1): flush[v] = 1
// where the joins pushed since the last flush might not leave room for v's.
std::vector<char> flush_schedule(const Diamond &D, int v0, int v1, int pcap);

}  // namespace tcurve

struct ts_tri {
  int d = 0, np = 0, V = 0, sw = 0, cw = 0, nmax = 0;
  int device = 0;
  tcurve::TableLayout lay{};
  std::vector<uint32_t> host_tables;
  uint32_t *d_tables = nullptr;  // lay.words words, 16-byte aligned
  tcurve::WarpLayout wlay{};
  std::vector<uint32_t> host_wtables;
  uint32_t *d_wtables = nullptr;  // wlay.words words (warp-per-instance kernels)
  uint32_t *d_err = nullptr;     // device error word (scratch, owned here)
  tcurve::Diamond dia;
  int kernel = 0;                // TS_KERNEL_*
  int scratch = 0;               // TS_SCRATCH_* (both kernel families)
  int occupancy = 0;             // target blocks per SM of the specialised kernels (0: default)
  std::mutex jit_mu;
  std::shared_ptr<tcurve::JitModule> jit;
  std::string jit_log;
};

struct ts_hist {
  int cw = 0;
  uint64_t slots = 0;                 // power of two
  uint64_t *d_keys = nullptr;         // slots * cw words, 0 = empty
  unsigned long long *d_counts = nullptr;
  uint32_t *d_err = nullptr;          // device error word
  unsigned long long *d_failed = nullptr;
  unsigned long long *d_work = nullptr;  // work counter of the persistent sweep
  // compaction buffers of ts_hist_read: the occupied slots, packed
  uint64_t *d_ckeys = nullptr;        // slots * cw words
  unsigned long long *d_ccnt = nullptr;  // slots counts
  unsigned long long *d_cn = nullptr;    // number of packed entries
  int device = 0;
};

namespace tcurve {
cudaError_t launch_real_schemes(const ts_tri *tri, const uint64_t *signs, uint64_t n,
                                uint64_t *codes, cudaStream_t stream);
// allow_global = false keeps the scratch in shared memory (no allocation).
cudaError_t launch_enumerate(const ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                             ts_hist *hist, cudaStream_t stream, bool allow_global = true);
// Warp-per-instance kernels (warp_kernels.cu, TS_KERNEL_WARP): the whole
// scratch in shared memory, so they allocate nothing either.
cudaError_t launch_real_schemes_warp(const ts_tri *tri, const uint64_t *signs, uint64_t n,
                                     uint64_t *codes, cudaStream_t stream);
cudaError_t launch_enumerate_warp(const ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                                  ts_hist *hist, cudaStream_t stream);
cudaError_t launch_hist_clear(ts_hist *hist, cudaStream_t stream);
cudaError_t launch_selftest_wait(unsigned long long iters, uint32_t *err, cudaStream_t stream);
// Pack the occupied slots of the table into d_ckeys / d_ccnt (count flags
// removed) and their number into d_cn.
cudaError_t launch_hist_compact(ts_hist *hist, cudaStream_t stream);
cudaError_t launch_splitmix_masks(int d, uint64_t base, uint64_t n, uint64_t *out,
                                  cudaStream_t stream);

// Stream-ordered device allocation for per-launch global scratch (the
// device's default pool keeps freed memory); free with cudaFreeAsync.
cudaError_t scratch_alloc(void **p, size_t bytes, cudaStream_t stream);

// Specialised kernels (jit.cpp).  global: per-thread scratch in global memory
// (128-thread blocks); min_blocks: blocks per SM the register budget is set for.
std::string jit_source(const Diamond &D, bool global = false, int min_blocks = 2);
// Configuration for a degree and the TS_SCRATCH_* / occupancy settings.
void jit_config(int d, int scratch, int occupancy, bool *global, int *min_blocks);
// Compile the generated source with NVRTC for sm_103a; returns the cubin (or
// an empty string and the log in *log).
std::string jit_compile_cubin(const std::string &src, std::string *log,
                              const std::vector<std::string> &extra = {});
cudaError_t jit_prepare(ts_tri *tri);  // compile + load once (thread-safe)
cudaError_t launch_real_schemes_jit(ts_tri *tri, const uint64_t *signs, uint64_t n,
                                    uint64_t *codes, cudaStream_t stream);
cudaError_t launch_enumerate_jit(ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                                 ts_hist *hist, cudaStream_t stream);
void jit_release(ts_tri *tri);

// Specialised kernels of batches (jit.cpp): per degree, one relocatable
// object per distinct triangulation (its per-mask sweep as straight-line
// code, exported as tcj_<i>) and one persistent kernel tcj_jobs that calls
// them, compiled in parallel and linked with nvJitLink.
struct JitJobsModule;
std::string jit_job_source(const Diamond &D, int idx, int min_blocks);
std::string jit_jobs_kernel_source(int d, int nfn, int min_blocks);
// Compile and link without a device (the linked cubin, or empty and the log).
std::string jit_jobs_link(const std::vector<const Diamond *> &tris, std::string *log);
// Build the modules of several degree groups (each group: the diamonds of
// its distinct triangulations, function i = group[i]; min_blocks[g]: the
// resident 128-thread blocks per SM its register budget is set for, 0 for
// the default) on the current device; a group whose module cannot be built
// gets null and a log.
cudaError_t jit_jobs_build(const std::vector<std::vector<const Diamond *>> &groups,
                           const std::vector<int> &min_blocks,
                           std::vector<std::shared_ptr<JitJobsModule>> *mods,
                           std::vector<std::string> *logs);
int jit_jobs_threads();
void jit_jobs_attrs(const JitJobsModule &m, int *regs, int *local_bytes);
int jit_jobs_blocks_per_sm(const JitJobsModule &m);
size_t jit_jobs_slab_bytes(const JitJobsModule &m);  // global scratch per block
cudaError_t jit_jobs_launch(const JitJobsModule &m, unsigned grid, const void *jobs, uint32_t njobs,
                            uint64_t items, uint32_t chunk, unsigned long long *work, uint32_t *err,
                            unsigned long long *failed, uint32_t *scratch, cudaStream_t st);

// Fused batch kernel (fused.cu): one persistent launch over the jobs of all
// degrees of a batch, each degree with its own tile (one thread or one warp
// per sign vector, sign vectors per work item).
constexpr int kFusedThreads = 128;  // threads per block (4 warps)
constexpr int kFusedTiers = 4;      // register tiers: degrees up to 6, 9, 11, 16
constexpr int kFusedWarpTier = 4;   // the tier-3 kernel with warp-per-instance bodies
constexpr int kFusedWarpFrom = 7;   // warp-per-instance bodies from this degree
struct FusedJob {
  const uint32_t *tab;   // tables staged for the job: table-driven or warp layout (tile)
  uint64_t n, base;      // sign vectors, splitmix64 counter base
  unsigned long long *codes;  // per-instance codes or null
  unsigned long long *hkeys;  // the job's histogram
  unsigned long long *hcnt;
  uint64_t hslots;
  uint64_t item0;        // first work item of the job
  uint32_t d, chunk;     // degree; sign vectors per work item (a multiple of kFusedThreads)
  uint32_t warp;         // 1: warp per instance (warp tables), 0: thread per instance
  uint32_t tab_words;    // words staged (a multiple of 4)
  uint32_t off_fan, off_vext;  // table-driven layout
  WarpLayout wl;               // warp layout
  uint32_t pad;
  const unsigned long long *signs;  // the caller's sign vectors (n x words), or null: splitmix64
};
int fused_tier(int dmax);          // tier of a batch whose largest degree is dmax (-1: none)
int fused_tier_degree(int tier);   // largest degree of a tier
uint32_t fused_slab_words(int tier);  // global scratch words per thread of a tier's kernel
uint32_t fused_warp_words(int d);     // shared words of one warp of a degree-d warp tile
cudaError_t fused_occupancy(int tier, size_t smem, int *blocks_per_sm);
cudaError_t fused_attrs(int tier, int *regs, int *local_bytes);
// smem = toff (the tables, 128-byte aligned) + 128 + kFusedThreads x
// ls_words words (label slots of the thread tiles) + 4 x ws_stride words
// (warp tiles); scratch: grid x kFusedThreads x fused_slab_words(tier) words.
cudaError_t fused_launch(int tier, unsigned grid, size_t smem, uint32_t toff, uint32_t ls_words,
                         uint32_t ws_stride, const FusedJob *jobs, uint32_t njobs, uint64_t items,
                         unsigned long long *work, uint32_t *err, unsigned long long *failed,
                         uint32_t *scratch, cudaStream_t st);
}  // namespace tcurve
