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

constexpr int kMaxDegree = 9;  // single-word sign masks, 8-bit vertex ids

// Table layout (32-bit words, all indices are vertex positions in the sweep
// order of T^diamond, see host.cpp):
//   vdesc[V]  bits 0-5 lattice index k(v), bit 6 parity constant c(v)
//             (sign(v) = sigma_k ^ c, Eq. 2), bits 7-12 fan length m,
//             bits 16-31 first fan entry
//   fan[NF]   bits 0-7 neighbour u, bits 8-13 k(u), bit 14 c(u),
//             bit 15 "u and the previous entry span a triangle with v"
//   vext[V]   bits 0-7 the antipodal partner x < v of v (0xFF: none), bits
//             8-15 and 16-23 the other end b < v of up to two boundary edges
//             kept for root detection (0xFF: none)
struct TableLayout {
  uint32_t V, NF;
  uint32_t off_vdesc, off_fan, off_vext;
  uint32_t words;  // padded to a multiple of 4 (16-byte TMA granule)
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

}  // namespace tcurve

struct ts_tri {
  int d = 0, np = 0, V = 0, sw = 0, cw = 0, nmax = 0;
  int device = 0;
  tcurve::TableLayout lay{};
  std::vector<uint32_t> host_tables;
  uint32_t *d_tables = nullptr;  // lay.words words, 16-byte aligned
  uint32_t *d_err = nullptr;     // device error word (scratch, owned here)
  tcurve::Diamond dia;
  int kernel = 0;                // TS_KERNEL_*
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
  int device = 0;
};

namespace tcurve {
cudaError_t launch_real_schemes(const ts_tri *tri, const uint64_t *signs, uint64_t n,
                                uint64_t *codes, cudaStream_t stream);
cudaError_t launch_enumerate(const ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                             ts_hist *hist, cudaStream_t stream);
cudaError_t launch_hist_clear(ts_hist *hist, cudaStream_t stream);
cudaError_t launch_splitmix_masks(int d, uint64_t base, uint64_t n, uint64_t *out,
                                  cudaStream_t stream);

// Specialised kernels (jit.cpp).
std::string jit_source(const Diamond &D);
// Compile the generated source with NVRTC for sm_103a; returns the cubin (or
// an empty string and the log in *log).
std::string jit_compile_cubin(const std::string &src, std::string *log);
cudaError_t jit_prepare(ts_tri *tri);  // compile + load once (thread-safe)
cudaError_t launch_real_schemes_jit(ts_tri *tri, const uint64_t *signs, uint64_t n,
                                    uint64_t *codes, cudaStream_t stream);
cudaError_t launch_enumerate_jit(ts_tri *tri, uint64_t lo, uint64_t hi, uint32_t flags,
                                 ts_hist *hist, cudaStream_t stream);
void jit_release(ts_tri *tri);
}  // namespace tcurve
