/* tcurve.h -- C ABI of the GB300 T-curve real-scheme engine (libtcurve.so).
 *
 * The engine computes, for a unimodular triangulation T of d*Delta_2 and a
 * batch of sign distributions sigma: A -> F_2, the real scheme (isotopy type
 * in RP^2) of the patchworked curve C(T, sigma) with Algorithm 1 of
 * "Fast Isotopy Computation for T-Curves" (Sec. 2), on the GPU.
 *
 * Conventions (the paper fixes none of them):
 *  - Lattice point set A = {(i,j) : i,j >= 0, i+j <= d} (Eq. 1); lattice
 *    index k(i,j) = j*(d+1) - j*(j-1)/2 + i.
 *  - A sign vector is ts_sign_words(tri) little-endian uint64 words; bit k
 *    (word k/64, bit k%64) is sigma at lattice index k.  Bit 1 means a
 *    negative coefficient: the coefficient of x^i y^j is (-1)^sigma(i,j)
 *    (Thm. 1).  Bits at positions >= |A| are ignored: every kernel clears
 *    them when it loads a sign vector.
 *  - A scheme code is ts_code_words(tri) little-endian uint64 words holding
 *    the integer (1 << nbits) | bits, where bits is the canonical encoding of
 *    the nesting tree of the ovals: enc(oval) = '1' . (encodings of the ovals
 *    directly inside it, in descending lexicographic order) . '0', and bits =
 *    the encodings of the outermost ovals in descending order (MSB first);
 *    nbits = 2 * #ovals.  The pseudoline of odd degree is implied by d.
 *    Code 0 is never a valid scheme; it marks an instance that failed.
 *  - Pointers documented as "device" must be CUDA device (or managed)
 *    memory; "host" pointers are ordinary host memory.  Streams are passed
 *    as void* holding a cudaStream_t (NULL = the legacy default stream).
 *  - The caller owns every buffer it passes; the engine owns ts_tri and
 *    ts_hist objects.  A ts_tri is immutable after loading and may be shared
 *    by concurrent launches; a ts_hist must not be written by two
 *    overlapping launches unless both are ts_enumerate calls (they merge by
 *    atomics).
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns TS_ECUDA.
 */
#ifndef TCURVE_H
#define TCURVE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ts_tri ts_tri;   /* a loaded triangulation (host + device tables) */
typedef struct ts_hist ts_hist; /* a device hash histogram: scheme code -> count  */

typedef enum ts_status {
  TS_OK = 0,
  TS_EINVAL = 1,       /* bad argument (range, null pointer, unknown flag) */
  TS_ENOTTRI = 2,      /* edges are not a unimodular triangulation of d*Delta_2 */
  TS_ENOMEM = 3,       /* host or device allocation failed */
  TS_ECUDA = 4,        /* CUDA error or no usable device */
  TS_EOVERFLOW = 5,    /* histogram or output capacity exceeded */
  TS_ETIMEOUT = 6,     /* a bounded device wait gave up */
  TS_EINTERNAL = 7,    /* an instance violated an invariant (no unique root,
                          region graph not a tree, scratch overflow) */
  TS_EUNSUPPORTED = 8  /* degree outside the range this build supports */
} ts_status;

/* Flags of ts_enumerate. */
#define TS_ENUM_FLIP 1u    /* mask = k << 1: one representative per global sign flip */
#define TS_ENUM_REDUCED 2u /* zeros inserted at bits 0, 1, d+1 (sigma(0,0) = sigma(1,0) =
                              sigma(0,1) = 0): one representative per (Z/2)^3 class (Sec. 3) */
#define TS_ENUM_SPLITMIX 4u /* word w of the mask = splitmix64(k * W + w), W sign words,
                               bits >= |A| cleared (one word: splitmix64(k)): a sampled,
                               reproducible stream of sign vectors (the stream of
                               ts_splitmix_masks and ts_batch_create); no bound on hi */
#define TS_ENUM_ORBITS 8u  /* one representative per (Z/2)^3 class (Sec. 3), other than
                              TS_ENUM_REDUCED's: sigma(0,1) = 0, all d+1 middle-row bits
                              free, the high part (bits d+2..|A|-1) the one of its coset
                              under the class group with two pivot bits zero:
                              m(k) = (h(k >> (d+1)) << (d+2)) | (k mod 2^(d+1)), h(u) = u
                              with zeros inserted at the pivots p2 < p1 (tc_layout.h,
                              tc_orbit_pivots).  Same histogram as TS_ENUM_REDUCED over the
                              whole range, and any range [lo, hi) keeps every middle-row
                              pattern, so chunked and sharded sweeps run whole blocks.
                              2 <= d <= 9 (TS_EUNSUPPORTED above, TS_EINVAL below) */

/* Human-readable name of a status code; never NULL. */
const char *ts_status_str(int status);

/* Largest degree this build supports (16: |A| <= 153, three sign words,
 * codes of at most four words). */
int ts_max_degree(void);

/* Load a triangulation T of d*Delta_2 given by its edge list (the input form
 * of Sec. 2).
 *   d        degree, 1 <= d <= ts_max_degree()
 *   edges_ij host, n_edges rows of 4 int32 (i1, j1, i2, j2), each a pair of
 *            lattice points of A; order and orientation are free
 *   out      receives the new object (owned by the engine; free with
 *            ts_free_triangulation)
 * Validation (TS_ENOTTRI): every end point in A, no repeated edge, exactly
 * d*d triangles (3-cliques of edges of area 1/2), every point of A used,
 * each edge on the boundary of d*Delta_2 in one triangle and every other
 * edge in two.  Regularity is not checked: Algorithm 1 does not need it
 * (proof of Thm. 2).  Builds the reflected triangulation T^diamond (Alg. 1,
 * line 1), its vertex sweep order and tables, and uploads them to the
 * current CUDA device. */
ts_status ts_load_triangulation(int d, const int32_t *edges_ij, int n_edges, ts_tri **out);
void ts_free_triangulation(ts_tri *tri);

int ts_degree(const ts_tri *tri);
int ts_num_points(const ts_tri *tri);  /* |A| = (d+1)(d+2)/2 (Eq. 1) */
int ts_sign_words(const ts_tri *tri);  /* ceil(|A| / 64)            */
/* ceil((2*nmax + 1) / 64) with nmax = M for even d and M-1 for odd d,
 * M = (d-1)(d-2)/2 + 1 Harnack's bound (Sec. 2). */
int ts_code_words(const ts_tri *tri);

/* Real schemes of n sign vectors (Algorithm 1 per instance).
 *   signs     device, n * ts_sign_words(tri) uint64, read-only
 *   out_codes device, n * ts_code_words(tri) uint64, written
 * Asynchronous on `stream`; returns TS_OK once launched.  Instances that
 * fail an invariant get code 0 and raise TS_EINTERNAL (TS_EOVERFLOW if the
 * scheme exceeds Harnack's bound) in the triangulation's error word, which
 * ts_sync reports.  Sign bits >= |A| are ignored. */
ts_status ts_real_schemes(const ts_tri *tri, const uint64_t *signs, uint64_t n,
                          uint64_t *out_codes, void *stream);

/* Kernel families (ts_set_kernel).  All compute the same codes.
 *   TS_KERNEL_TABLE: one generic kernel per degree; the triangulation's
 *     tables are staged into shared memory by a bulk copy in every block.
 *   TS_KERNEL_SPECIALIZED: a kernel generated for this triangulation (its
 *     structure compiled into the instruction stream) with NVRTC on first use;
 *     d <= 9 only (one sign word), TS_EUNSUPPORTED above.
 *   TS_KERNEL_WARP: one generic kernel per degree in which a whole warp
 *     classifies one sign vector at a time (lock-free union-find over the
 *     edges of T^diamond, region tree and code in the warp's shared memory;
 *     no global scratch).  ts_real_schemes and ts_enumerate; batches run
 *     it as the warp tile of their fused launch (ts_batch_set_fused_tile);
 *     ts_enumerate_noalloc runs the table-driven family.
 *   TS_KERNEL_AUTO (default): specialised for ts_enumerate and for batches of
 *     at least 65536 instances when d <= 9, table-driven otherwise or if the
 *     specialised kernel cannot be built. */
#define TS_KERNEL_AUTO 0
#define TS_KERNEL_TABLE 1
#define TS_KERNEL_SPECIALIZED 2
#define TS_KERNEL_WARP 3
ts_status ts_set_kernel(ts_tri *tri, int kind);

/* Where the kernels keep their per-instance scratch (labels, union-find,
 * region tree; 0.1 to 3.7 KB per instance, growing with d).
 *   TS_SCRATCH_SHARED: shared memory (few resident warps for large d).
 *   TS_SCRATCH_GLOBAL: device memory, L1/L2-resident, allocated per launch
 *     with cudaMallocAsync on the launch's stream and freed after it (the
 *     device's default memory pool is set to keep freed memory).
 *   TS_SCRATCH_AUTO (default): global from d = 7, shared below.
 * Changing it drops the specialised kernels already built for tri (they are
 * rebuilt on next use).  Results are identical. */
#define TS_SCRATCH_AUTO 0
#define TS_SCRATCH_SHARED 1
#define TS_SCRATCH_GLOBAL 2
ts_status ts_set_scratch(ts_tri *tri, int where);

/* Resident blocks per SM the specialised kernels are compiled for (their
 * register budget): 1..16, or 0 for the default (with global scratch 7, 6
 * and 4 blocks of 128 threads for d = 7, 8, 9 and 4 otherwise; 2 with shared
 * scratch).  Drops kernels already built for tri.  A batch's specialised
 * code (ts_batch_info) takes the largest value over its group's
 * triangulations when it is built (default: 4 blocks of 128 threads up to
 * d = 10, 3 above). */
ts_status ts_set_occupancy(ts_tri *tri, int blocks_per_sm);

/* Build the specialised kernels now (NVRTC compile and module load on the
 * current device; about a second).  Call it before capturing launches of
 * this triangulation in a CUDA graph, since the first specialised launch
 * otherwise compiles.  Returns TS_ECUDA if compilation or loading fails
 * (ts_specialized_log then holds the compiler log), TS_EUNSUPPORTED for
 * d > 9. */
ts_status ts_prepare(ts_tri *tri);
ts_status ts_specialized_log(const ts_tri *tri, char *buf, size_t len);

/* Host-only helper (no device needed): validate the edge list and write the
 * generated specialised CUDA source into buf (compile = 0), or compile it
 * with NVRTC for sm_103a and write the compiler log (compile = 1; returns
 * TS_ECUDA if it does not compile).  *needed receives the full length + 1.
 * The source is that of the default configuration (TS_SCRATCH_AUTO, default
 * occupancy).  TS_EUNSUPPORTED for d > 9. */
ts_status ts_specialized_source(int d, const int32_t *edges_ij, int n_edges, int compile, char *buf,
                                size_t len, size_t *needed);

/* Same computation with host buffers: copies signs to the device, runs,
 * copies codes back and synchronises (allocates device memory per call).
 * Returns the error status of the run. */
ts_status ts_real_schemes_host(const ts_tri *tri, const uint64_t *signs_host, uint64_t n,
                               uint64_t *codes_host);

/* Wait for `stream`, then return and clear the triangulation's device error
 * word (TS_OK if no instance failed since the last call). */
ts_status ts_sync(const ts_tri *tri, void *stream);

/* Input generation: the sign vectors of counters base .. base+n-1 of degree
 * d: word w of vector i is splitmix64((base + i) * W + w), W sign words, with
 * the bits >= |A| cleared (one word: splitmix64(base + i)).  out: device,
 * n * W uint64; asynchronous.  The same sign vectors as TS_ENUM_SPLITMIX
 * sweeps and batches use. */
ts_status ts_splitmix_masks(int d, uint64_t base, uint64_t n, uint64_t *out, void *stream);

/* Device hash histogram of scheme codes with room for `capacity` distinct
 * codes of `code_words` words each (rounded up to a power of two, x2). */
ts_status ts_hist_create(uint64_t capacity, int code_words, ts_hist **out);
void ts_hist_free(ts_hist *hist);
/* Reset counts and error state (asynchronous on stream). */
ts_status ts_hist_clear(ts_hist *hist, void *stream);

/* Exhaustive sweep (Sec. 3, an exhaustive check of the sign distributions of
 * one or a few triangulations): adds the scheme of every mask m(k), k in
 * [lo, hi), to `hist`, which must have ts_code_words(tri) words per code.
 * m(k) = k by default; k << 1 with TS_ENUM_FLIP; k with zero bits inserted at
 * positions 0, 1 and d+1 with TS_ENUM_REDUCED (bits carried past bit 63 go
 * to the second sign word); the splitmix64 stream with TS_ENUM_SPLITMIX; the
 * orbit representatives of TS_ENUM_ORBITS (at most one flag).
 * Except with TS_ENUM_SPLITMIX, m(hi-1) < 2^|A| (a bound only for d <= 9
 * and, with TS_ENUM_REDUCED, d = 10).  Persistent launches on `stream`
 * (whole blocks of middle-row patterns, and a ragged head and tail mask by
 * mask); asynchronous.  With TS_ENUM_FLIP the specialised kernels take a
 * block of masks and the block of their complements (every bit flipped)
 * together, evaluating the complements of half of them instead: the global
 * sign flip keeps the curve, so the histogram is the one of the masks m(k).
 * Failed instances are counted, not inserted, and set the histogram's
 * error word. */
ts_status ts_enumerate(const ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                       ts_hist *hist, void *stream);

/* Copy the histogram to the host, sorted by code (little-endian word
 * order, most significant word first in the comparison).  Synchronises
 * `stream`.
 *   codes   host, cap * code_words uint64 (may be NULL when cap == 0)
 *   counts  host, cap uint64
 *   n_out   receives the number of distinct codes
 *   n_failed (may be NULL) receives the number of failed instances
 * Returns TS_EOVERFLOW if n_out > cap (nothing beyond cap is written) or if
 * the device table overflowed; otherwise the histogram's error status. */
ts_status ts_hist_read(ts_hist *hist, uint64_t *codes, uint64_t *counts, uint64_t cap,
                       uint64_t *n_out, uint64_t *n_failed, void *stream);

/* ---- Batches of mixed-degree triangulations (one graph launch) ----
 *
 * A batch holds njobs jobs; job j classifies counts[j] sign vectors of tris[j]
 * (any supported degree), vector i being the splitmix64 sign vector of
 * counter bases[j] + i (ts_splitmix_masks; splitmix64 as published by Steele,
 * Lea and Flood: z = x + 0x9E3779B97F4A7C15; z = (z ^ z >> 30) *
 * 0xBF58476D1CE4E5B9; z = (z ^ z >> 27) * 0x94D049BB133111EB; z ^ z >> 31),
 * and adds each code to the job's own device histogram (room for
 * min(hist_capacity, counts[j]) distinct codes, hist_capacity <= 2^20); if code_outputs is
 * not NULL and code_outputs[j] is not NULL (device, counts[j] *
 * ts_code_words(tris[j]) uint64), it also stores every code there.  By
 * default, for each degree present one persistent kernel serves all jobs of
 * that degree, staging a job's tables into shared memory when it moves to
 * that job, and the per-degree kernels run concurrently
 * (ts_batch_set_serial orders them; ts_batch_set_fused runs every job in
 * one kernel).  counts[j] <= 2^62 (TS_EINVAL above).  The triangulations
 * must stay loaded while the batch exists.  Allocates device memory at
 * creation and when a tile or launch plan changes (ts_batch_set_tile,
 * ts_batch_set_kernel, ts_batch_set_fused, ts_batch_set_fused_tile,
 * ts_batch_set_signs), never in ts_batch_run. */
typedef struct ts_batch ts_batch;
ts_status ts_batch_create(int njobs, ts_tri *const *tris, const uint64_t *counts,
                          const uint64_t *bases, uint64_t *const *code_outputs,
                          uint64_t hist_capacity, ts_batch **out);
void ts_batch_free(ts_batch *batch);
/* Tile of the degree-d kernel: threads per block (multiple of 32, at most 256;
 * with shared scratch the block's scratch must fit shared memory), sign
 * vectors per work item (a multiple of threads) and scratch placement
 * (TS_SCRATCH_*; global scratch is allocated here, grid x threads x
 * scratch words).  Returns TS_EINVAL for tiles that do not fit, and for a
 * specialised group (ts_batch_info) any block size but 128 or shared
 * scratch: its code is compiled for 128-thread blocks and global scratch.
 * Waits for
 * all work on the device first (runs already launched use the tile's tables
 * and scratch); the next ts_batch_run with use_graph captures a new graph. */
ts_status ts_batch_set_tile(ts_batch *batch, int d, int threads, int chunk, int scratch);
/* How ts_batch_run orders the degree groups' persistent kernels: serial = 0
 * (default) forks them onto streams of their own, so they run concurrently;
 * serial = 1 runs them one after the other on the run's stream, each
 * filling the whole GPU.  Takes effect at the next run (a new graph is
 * captured).  TS_EINVAL for other values. */
ts_status ts_batch_set_serial(ts_batch *batch, int serial);
/* One persistent launch for the whole batch (an engine facility against the
 * kernel-dispatch overhead that Sec. 3 names as a cost at scale): with
 * fused = 1, ts_batch_run launches a single kernel that pulls the work items
 * of every job of every degree from one counter (jobs in degree order, so
 * the degrees follow one another without a gap), stages a job's tables with
 * cp.async.bulk when it moves to another triangulation, and runs each job
 * with its degree's fused tile (ts_batch_set_fused_tile).  The kernel is
 * compiled per range of degrees with the register budget of that range's
 * table-driven sweep (degrees up to 6, 9, 11, 16: 40, 48, 64, 80
 * registers); a batch takes the range of its largest degree, or the widest
 * one when a degree has a warp tile.  Specialised groups do not apply in
 * this mode.  fused = 0 (default) returns to one persistent kernel per
 * degree group (ts_batch_set_serial).  Allocates the job table and global
 * scratch of the launch here (grid x 128 threads x scratch words), after
 * waiting for all work on the device; the next run with use_graph captures
 * a new graph.  TS_EINVAL for other values. */
ts_status ts_batch_set_fused(ts_batch *batch, int fused);
/* Tile of degree d in the fused launch: kind TS_KERNEL_TABLE or
 * TS_KERNEL_AUTO (default: one thread per sign vector, the table-driven
 * sweep, per-thread scratch in global memory) or TS_KERNEL_WARP (d >= 7:
 * the 32 lanes of a warp classify one sign vector together, the state in
 * shared memory), and chunk sign vectors per work item (a multiple of 128,
 * at most 2^24; default 1024).  May be set in either mode; in fused mode it
 * waits for all work on the device and re-plans the launch (the next run
 * with use_graph captures a new graph).  TS_EINVAL for other values, a
 * degree the batch does not hold, or a tile whose launch does not fit (the
 * previous tile is kept). */
ts_status ts_batch_set_fused_tile(ts_batch *batch, int d, int kind, int chunk);
/* Query jobs in a batch (an engine facility): job `job` classifies the
 * caller's sign vectors instead of its splitmix64 stream.
 *   signs  device, counts[job] * ts_sign_words(tris[job]) uint64, read by
 *          every run; the caller keeps it alive and unchanged while runs
 *          may read it.  NULL returns the job to its splitmix64 stream.
 * Such jobs run only in the fused launch (ts_batch_set_fused):
 * ts_batch_run returns TS_EINVAL in the per-degree group mode while a job
 * has caller sign vectors.  Waits for all work on the device first; the
 * next run with use_graph captures a new graph.  TS_EINVAL for a bad job
 * index. */
ts_status ts_batch_set_signs(ts_batch *batch, int job, const uint64_t *signs);
/* Clear the histograms and run every job, asynchronously on stream.  With
 * use_graph the work (clears, fork, per-degree kernels, join) is captured
 * into a CUDA graph on the first call (and after a tile change) and the graph
 * is launched; otherwise the same work is enqueued directly. */
ts_status ts_batch_run(ts_batch *batch, int use_graph, void *stream);
/* Kernel family, tile and launch resources of the degree-d group of a batch
 * (an engine facility).  A group runs the table-driven kernel
 * (TS_KERNEL_TABLE) or specialised code (TS_KERNEL_SPECIALIZED): every
 * distinct triangulation of the group compiled into a straight-line sweep of
 * its own (one relocatable object each, compiled with NVRTC in parallel host
 * threads) and linked with the group's persistent kernel (nvJitLink), which
 * calls each job's sweep.  A group is specialised at creation when one of its
 * triangulations was set to TS_KERNEL_SPECIALIZED, or, with TS_KERNEL_AUTO,
 * when d <= 6 and the group holds at least 2^22 sign vectors; never when
 * one of them was set to TS_KERNEL_TABLE, and not if the code cannot be
 * built (log then says why); ts_batch_set_kernel changes it later.
 * Specialised groups have 128-thread blocks and global scratch
 * (ts_batch_set_tile accepts only those; the chunk may vary).  In fused
 * mode (ts_batch_set_fused) info describes the degree's fused tile instead:
 * kernel TS_KERNEL_TABLE or TS_KERNEL_WARP, 128 threads, its chunk, scratch
 * TS_SCRATCH_GLOBAL (thread tiles) or TS_SCRATCH_SHARED (warp tiles), and
 * the registers, resident blocks and grid of the one fused kernel.
 *   info  receives kernel (TS_KERNEL_*), threads per block, chunk (sign
 *         vectors per work item), scratch (TS_SCRATCH_*), registers per
 *         thread, local_bytes (per-thread local memory: spills, call
 *         frames), blocks_per_sm (resident blocks of the launch) and grid
 *   log   (may be NULL; len bytes with the NUL) the reason a specialised
 *         group fell back to the table-driven kernel, or ""
 * TS_EINVAL if the batch has no job of degree d. */
typedef struct ts_batch_group_info {
  int kernel, threads, chunk, scratch;
  int registers, local_bytes, blocks_per_sm, grid;
} ts_batch_group_info;
ts_status ts_batch_info(const ts_batch *batch, int d, ts_batch_group_info *info, char *log,
                        size_t len);
/* Kernel family of the degree-d group: TS_KERNEL_TABLE, TS_KERNEL_SPECIALIZED
 * (builds the group's specialised code now if it has none: about a second
 * of compilation per triangulation, in parallel host threads) or
 * TS_KERNEL_AUTO (the rule at creation).  Resets the group's tile to the
 * family's default.  Waits for all work on the device first; the next
 * ts_batch_run with use_graph captures a new graph.  TS_ECUDA if the
 * specialised code cannot be built (the group then runs table-driven, and
 * ts_batch_info's log says why), TS_EINVAL without a group of degree d. */
ts_status ts_batch_set_kernel(ts_batch *batch, int d, int kind);
/* Host-only helper (no device needed): validate ntri edge lists of degree d
 * and build the specialised batch code for them as ts_batch_create would
 * (one object per triangulation and the persistent kernel, compiled with
 * NVRTC for sm_103a and linked with nvJitLink).  *linked_bytes receives the
 * size of the linked image; log (len bytes) the compiler logs of all
 * objects (their ptxas resource lines), or the failing step's log.
 * TS_ENOTTRI for a bad edge list, TS_ECUDA if compiling or linking fails. */
ts_status ts_batch_specialized_link(int d, int ntri, const int32_t *const *edges_ij,
                                    const int *n_edges, size_t *linked_bytes, char *log, size_t len);
/* Histogram of one job, sorted by code, after synchronising stream (same
 * output conventions as ts_hist_read with ts_code_words(tris[job]) words per
 * code; n_failed counts the whole batch). */
ts_status ts_batch_read(ts_batch *batch, int job, uint64_t *codes, uint64_t *counts, uint64_t cap,
                        uint64_t *n_out, uint64_t *n_failed, void *stream);

/* Exhaustive sweep that allocates nothing (the paper has no counterpart; it
 * is an engine facility).  For callers that cannot allocate device memory at
 * the time they sweep: services that reserve all device memory up front and
 * forbid later allocations, and threads that must not enter an allocator (a
 * real-time loop where an allocation could block, a thread that holds the
 * allocator's lock).  Same results as ts_enumerate followed by ts_hist_read
 * on the same range and flags, computed by the table-driven sweep kernel
 * with its hash table, counters and error word in one static device array
 * of 65 600 bytes that every GPU loading this library keeps until the
 * process exits.  The caller passes the outputs:
 *   flags          0, TS_ENUM_FLIP or TS_ENUM_REDUCED (TS_ENUM_SPLITMIX is
 *                  not accepted here: TS_EINVAL)
 *   codes, counts  device, cap uint64 each: the distinct codes (1 word each)
 *                  and their counts, unsorted
 *   cap            at most 2048 (the array's table holds 2048 codes);
 *                  larger values return TS_EINVAL
 *   n_out          device, 3 uint64: [0] distinct codes found (entries beyond
 *                  cap are dropped), [1] failed instances, [2] error bits
 *                  (nonzero: more than cap codes, a full table, or a failed
 *                  instance)
 * Requires d <= 9 (TS_EUNSUPPORTED above) and tri loaded on the current
 * device.  Asynchronous on stream.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the life of
 * the process; make that first call before any stream capture.  The kept
 * address belongs to the device's context of that time: after a
 * cudaDeviceReset of the device, do not call this entry point again in the
 * same process.  Every call reuses the same array and clears it first, so
 * calls that overlap on the GPU (different streams, or host threads without
 * ordering) race and corrupt each other's results: serialise them. */
ts_status ts_enumerate_noalloc(const ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                               uint64_t *codes, uint64_t *counts, uint64_t cap, uint64_t *n_out,
                               void *stream);

/* Self-test of the engine's bounded device waits: runs a kernel whose only
 * wait is on an mbarrier that nothing completes, polled at most iters times
 * (1 <= iters <= 2^20), and returns the status the kernel reported:
 * TS_ETIMEOUT when the wait gave up as designed (the GPU context stays
 * usable), TS_ECUDA without a device.  Synchronises stream. */
ts_status ts_selftest_wait(uint64_t iters, void *stream);

/* Measured integer-issue peak (an engine facility for the roofline of the
 * kernels above, which are integer work: no tensor-core or floating-point
 * component; the paper has no counterpart).  Runs a kernel that fills every
 * SM with 64 warps, each thread issuing independent chains of one integer
 * instruction kind for `trips` loop trips (1 <= trips <= 2^24), and times it
 * with CUDA events on stream:
 *   kind 0  lop3 (three-input logic)     kind 2  mad.lo (integer multiply-add)
 *   kind 1  add                          kind 3  lop3 and mad.lo alternating
 * *lane_ops_per_s receives the lane operations per second (thread
 * instructions of that kind per second); *ms (may be NULL) the kernel time.
 * Synchronises stream.  TS_ECUDA without a device. */
ts_status ts_int_issue_peak(int kind, uint64_t trips, double *lane_ops_per_s, double *ms,
                            void *stream);

/* Rohlin-Viro notation of a code (Sec. 2): "<0>", "<J>", "<4>", "<1<1>>",
 * "<J + 1<1> + 2>" ('+' stands for the disjoint union); writes at most len
 * bytes including the terminating NUL. */
ts_status ts_scheme_string(int d, const uint64_t *code, int code_words, char *buf, size_t len);

#ifdef __cplusplus
}
#endif
#endif
