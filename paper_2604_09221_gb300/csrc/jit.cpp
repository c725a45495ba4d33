// jit.cpp -- triangulation-specialised kernels.
//
// For a loaded triangulation the host writes the sweep of Algorithm 1
// (lines 1-4) as straight-line CUDA: every vertex of T^diamond in sweep
// order becomes a few integer instructions whose operands (lattice bit
// positions, Eq. 2 parity constants, fan neighbours, link bits, antipodal
// partners) are immediates, and the provisional component label of each
// vertex is a register.  The generated functions sit between the device
// runtime (tc_runtime.cuh: label union-find, region tree, AHU code, hash
// histogram) and the kernels (jit_kernels.cuh); the source is compiled with
// NVRTC for sm_103a and loaded with the driver API (entry points obtained
// from the runtime, so the library does not link libcuda or libnvrtc; NVRTC
// is opened on first use).
#include <cuda.h>
#include <dlfcn.h>
#include <nvJitLink.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstdio>
#include <map>
#include <sstream>
#include <thread>

#include "engine.h"
#include "tc_layout.h"

namespace tcurve {

namespace {

const char kRuntimeSrc[] =
#include "_tc_runtime_src.inc"
    ;
const char kKernelsSrc[] =
#include "_jit_kernels_src.inc"
    ;

constexpr int kJitThreads = 256;

typedef TcLayout Layout;

// Scratch layout of the specialised kernels: 256-thread blocks (fewer if two
// do not fit shared memory) with shared scratch, 128 with global scratch.
// The block sweep also keeps, after [odd], a snapshot of the half-diamonds'
// label parents and odd flags beyond the first SNAPW words (which stay in
// registers): [snap] = wlab + wodd words, emitted as OFF_SNAP.
Layout layout_for(const Diamond &D, bool global) {
  // one label per vertex: the block sweep's half-diamonds run table-driven
  Layout L = tc_layout(D.d, true, global ? 128 : kJitThreads);
  const int snap_words = L.wlab + L.wodd;
  L.words += snap_words;
  if (global) {
    L.threads = 128;
  } else {  // two blocks per SM, as tc_layout sizes them
    L.threads = kJitThreads;
    while (L.threads > 32 && 2 * (L.words * 4 * L.threads + L.hash * 16 + 16) > 216 * 1024)
      L.threads -= 32;
  }
  return L;
}

// First word of the [snap] region (the end of tc_layout's words).
int snap_offset(const Layout &L) { return L.words - (L.wlab + L.wodd); }

// ---- NVRTC, opened on first use ----
struct Nvrtc {
  void *h = nullptr;
  decltype(&nvrtcCreateProgram) create = nullptr;
  decltype(&nvrtcCompileProgram) compile = nullptr;
  decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
  decltype(&nvrtcGetProgramLog) log = nullptr;
  decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
  decltype(&nvrtcGetCUBIN) cubin = nullptr;
  decltype(&nvrtcDestroyProgram) destroy = nullptr;
  bool ok = false;
};

Nvrtc &nvrtc() {
  static Nvrtc n;
  static std::once_flag once;
  std::call_once(once, [] {
    const char *names[] = {"libnvrtc.so.13", "libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so.13",
                           "/usr/local/cuda/lib64/libnvrtc.so"};
    for (const char *nm : names)
      if ((n.h = dlopen(nm, RTLD_NOW | RTLD_GLOBAL))) break;
    if (!n.h) return;
    n.create = (decltype(n.create))dlsym(n.h, "nvrtcCreateProgram");
    n.compile = (decltype(n.compile))dlsym(n.h, "nvrtcCompileProgram");
    n.log_size = (decltype(n.log_size))dlsym(n.h, "nvrtcGetProgramLogSize");
    n.log = (decltype(n.log))dlsym(n.h, "nvrtcGetProgramLog");
    n.cubin_size = (decltype(n.cubin_size))dlsym(n.h, "nvrtcGetCUBINSize");
    n.cubin = (decltype(n.cubin))dlsym(n.h, "nvrtcGetCUBIN");
    n.destroy = (decltype(n.destroy))dlsym(n.h, "nvrtcDestroyProgram");
    n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
  });
  return n;
}

// ---- driver entry points (through the runtime) ----
struct Driver {
  decltype(&cuModuleLoadData) load = nullptr;
  decltype(&cuModuleUnload) unload = nullptr;
  decltype(&cuModuleGetFunction) get = nullptr;
  decltype(&cuFuncSetAttribute) set_attr = nullptr;
  decltype(&cuOccupancyMaxActiveBlocksPerMultiprocessor) occupancy = nullptr;
  decltype(&cuLaunchKernel) launch = nullptr;
  decltype(&cuFuncGetAttribute) get_attr = nullptr;
  bool ok = false;
};

Driver &driver() {
  static Driver d;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [](const char *sym, void **fn) {
      cudaDriverEntryPointQueryResult q;
      return cudaGetDriverEntryPointByVersion(sym, fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
             q == cudaDriverEntryPointSuccess;
    };
    d.ok = get("cuModuleLoadData", (void **)&d.load) && get("cuModuleUnload", (void **)&d.unload) &&
           get("cuModuleGetFunction", (void **)&d.get) &&
           get("cuFuncSetAttribute", (void **)&d.set_attr) &&
           get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void **)&d.occupancy) &&
           get("cuLaunchKernel", (void **)&d.launch) &&
           get("cuFuncGetAttribute", (void **)&d.get_attr);
  });
  return d;
}

int sm_count_now() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

std::string jit_compile_uncached(const std::string &src, std::string *log,
                                 const std::vector<std::string> &extra);

struct JitModule {
  CUmodule mod = nullptr;
  CUfunction real = nullptr, enumerate = nullptr, blocks = nullptr;
  Layout L{};
  bool global = false;  // per-thread scratch in global memory
  size_t smem_real = 0, smem_enum = 0;
  int bpsm_real = 0, bpsm_enum = 0, bpsm_blocks = 0;
  ~JitModule() {
    if (mod && driver().ok) driver().unload(mod);
  }
};

namespace {

// The traits struct TcK of a generated source: degree, block size and the
// scratch layout of tc_layout.h (both back ends' offsets).
void emit_traits(std::ostringstream &o, const Layout &L, int d, int V, bool global, int min_blocks) {
  o << "struct TcK {\n";
  auto c = [&](const char *n, long v) { o << "  static constexpr unsigned " << n << " = " << v << "u;\n"; };
  c("D", d); c("V", V); c("NPOINTS", (d + 1) * (d + 2) / 2); c("RMAX", L.rmax); c("NB", L.nb);
  c("THREADS", L.threads); c("HASH", L.hash); c("LBYTES", L.lbytes); c("CODE64", L.code64);
  c("PCAP", L.pcap); c("WODD", L.wodd); c("WORDS", L.words); c("B", d + 1); c("SNAPW", L.snapw);
  c("WLAB", L.wlab); c("EPW", L.epw); c("OFF_SNAP", snap_offset(L));
  c("GSCR", global ? 1 : 0); c("MINB", min_blocks);
  c("W", L.sw); c("CW", L.cw); c("WIDE", L.wide);
  c("OFF_LPAR", L.off_lpar); c("OFF_CAND", L.off_cand); c("OFF_LAB", L.off_lab);
  c("OFF_BPAIR", L.off_bpair); c("OFF_PEND", L.off_pend); c("OFF_ADJ", L.off_adj);
  c("OFF_RLAB", L.off_rlab); c("OFF_TPAR", L.off_tpar); c("OFF_ORDER", L.off_order);
  c("OFF_CLEN", L.off_clen); c("OFF_ODD", L.off_odd); c("OFF_CODE", L.off_code);
  c("OFF_WPAR", L.off_wpar); c("OFF_WFC", L.off_wfc); c("OFF_WNS", L.off_wns);
  c("OFF_WENT", L.off_went); c("OFF_WARENA", L.off_warena); c("OFF_WTEMP", L.off_wtemp);
  c("WARENA", L.warena_words);
  o << "};\n";
}

// Straight-line code of one vertex of the sweep (Alg. 1, lines 3-4): its
// sign from TC_BIT (or, with mid_sig, from that expression: the block sweep's
// middle-row pattern), its label from the first same-sign fan entry or a
// fresh one, a join per further same-sign run of its fan, its antipodal
// join and, for odd d, the crossed boundary edges it completes.  flush: apply
// the pending joins first (the static schedule of flush_schedule).
struct VertexEmitter {
  const Diamond &D;
  std::ostringstream &o;
  std::vector<std::vector<int>> anti_at, bedge_at;  // pairs / boundary edges completed at v
  VertexEmitter(const Diamond &DD, std::ostringstream &oo)
      : D(DD), o(oo), anti_at(DD.V), bedge_at(DD.V) {
    for (size_t i = 0; i < D.anti.size(); ++i) anti_at[D.anti[i].second].push_back((int)i);
    if (D.d % 2)
      for (size_t i = 0; i < D.bedge.size(); ++i)
        bedge_at[std::max(D.bedge[i].first, D.bedge[i].second)].push_back((int)i);
  }
  void emit(int v, const char *ind, const char *mid_sig, bool flush) {
    const auto &fan = D.fan[v];
    const auto &lk = D.link[v];
    const int m = (int)fan.size();
    o << ind << "// vertex " << v << " (" << D.x[v] << "," << D.y[v] << ")\n";
    if (flush) o << ind << "tc_unions(S, np); np = 0;  // scheduled flush of the join list\n";
    if (mid_sig && D.y[v] == 0)
      o << ind << "const u32 s" << v << " = ((" << mid_sig << " >> " << D.k[v] << ") & 1u) ^ " << D.c[v]
        << "u;\n";
    else
      o << ind << "const u32 s" << v << " = TC_BIT(" << D.k[v] << ") ^ " << D.c[v] << "u;\n";
    o << ind << "u32 L" << v << ";\n";
    if (m == 0) {
      o << ind << "L" << v << " = nl; tc_newlab(S, nl, TcS::NONE); ++nl;\n";
    } else {
      o << ind << "{\n";
      for (int i = 0; i < m; ++i)
        o << ind << "  const u32 e" << i << " = s" << fan[i] << " ^ s" << v << " ^ 1u;\n";
      o << ind << "  L" << v << " = ";
      for (int i = 0; i < m; ++i) o << "e" << i << " ? L" << fan[i] << " : ";
      o << "nl;\n" << ind << "  if (!(";
      for (int i = 0; i < m; ++i) o << (i ? " | " : "") << "e" << i;
      o << ")) { tc_newlab(S, nl, L" << fan[0] << "); ++nl; }\n";
      // a same-sign entry that starts a new run after an earlier run: join
      if (m >= 2) {
        o << ind << "  u32 any = e0;\n";
        for (int i = 1; i < m; ++i) {
          o << ind << "  { const u32 st = e" << i;
          if (lk[i]) o << " & (e" << i - 1 << " ^ 1u)";
          o << "; if (st & any) S.word(TcK::OFF_PEND, np) = L" << v << " | (L" << fan[i]
            << " << 16); np += st & any; any |= st; }\n";
        }
      }
      o << ind << "}\n";
    }
    for (int i : anti_at[v])
      o << ind << "S.word(TcK::OFF_PEND, np) = L" << D.anti[i].first << " | (L" << v
        << " << 16) | 0x80000000u; ++np;\n";
    for (int i : bedge_at[v]) {
      const int a = D.bedge[i].first, b = D.bedge[i].second;
      o << ind << "if (s" << a << " ^ s" << b << ") { tc_bpair(S, nb, L" << a << ", L" << b
        << "); ++nb; }\n";
    }
  }
};

}  // namespace

std::string jit_source(const Diamond &D, bool global, int min_blocks) {
  const Layout L = layout_for(D, global);
  const int d = D.d, V = D.V;
  std::ostringstream o;
  o << "// T-curve real-scheme kernels specialised to one triangulation of " << d
    << "*Delta_2 (generated)\n";
  emit_traits(o, L, d, V, global, min_blocks);
  o << "#define TC_HEAVY_FN __forceinline__\n";
  o << kRuntimeSrc;
  o << "#define TC_BIT(k) ((k) < 32 ? ((slo >> ((k) & 31)) & 1u) : ((shi >> ((k) & 31)) & 1u))\n"
    << "typedef TcScratch<TcK> TcS;\n\n";
  // the triangulation tables, for the table-driven half-diamonds of the block
  // sweep (warp-uniform reads: constant memory)
  std::vector<uint32_t> tab;
  TableLayout tl{};
  if (!pack_diamond_tables(D, tab, tl)) return std::string();
  o << "__constant__ u32 tc_ctab[" << tab.size() << "] = {";
  for (size_t i = 0; i < tab.size(); ++i) o << (i % 12 ? " " : "\n  ") << tab[i] << "u,";
  o << "\n};\n\n";
  VertexEmitter em(D, o);
  const auto &anti_at = em.anti_at;
  const auto &bedge_at = em.bedge_at;
  // Static flush schedules of the join list: the whole sweep (per-mask
  // kernels) and the middle row alone (block sweep, empty list at its start).
  const int Vo0 = V - (2 * d + 1);
  const std::vector<char> flush_full = flush_schedule(D, 0, V, L.pcap);
  const std::vector<char> flush_mid = flush_schedule(D, Vo0, V, L.pcap);
  auto emit_vertex = [&](int v, const char *ind, const char *mid_sig, bool flush) {
    em.emit(v, ind, mid_sig, flush);
  };
  const int Vo = V - (2 * d + 1);  // the middle row comes last in the sweep

  // ---- the whole sweep for one mask ----
  o << "__device__ __forceinline__ u64 tc_classify(u64 sig, const TcS &S, u32 &err) {\n"
    << "  const u32 slo = (u32)sig, shi = (u32)(sig >> 32);\n  u32 nl = 0, nb = 0, np = 0;\n"
    << "  tc_clear_odd(S);\n";
  for (int v = 0; v < V; ++v) emit_vertex(v, "  ", nullptr, flush_full[v] != 0);
  o << "  tc_unions(S, np);\n  return tc_backend(S, nl, nb, err);\n}\n\n";

  // ---- block sweep: halves once, middle row per instance ----
  o << "__device__ __forceinline__ void tc_sweep_amortised(u64 sig_hi, u32 ishift, u32 ireps,\n"
    << "    const TcS &S, u32 &err,\n"
    << "    u64 *hkeys, unsigned long long *hcnt, u64 *gkeys, unsigned long long *gcnt, u64 gslots,\n"
    << "    u32 *gerr, unsigned long long &failed) {\n"
    << "  const u32 lane = threadIdx.x & 31u;\n"
    << "  const u32 slo = (u32)sig_hi, shi = (u32)(sig_hi >> 32);\n  u32 nl = 0, nb = 0, np = 0;\n"
    << "  tc_clear_odd(S);\n";
  // the half-diamonds: one table-driven loop (they run once per warp for
  // 32 x ireps instances; straight-line code for them would crowd the
  // instruction caches)
  o << "  tc_sweep_table(TcSig<1>{{sig_hi}}, tc_ctab + " << tl.off_vdesc << "u, tc_ctab + "
    << tl.off_fan << "u, tc_ctab + " << tl.off_vext << "u, 0u, " << Vo << "u, S, nl, nb, np);\n";
  o << "  tc_unions(S, np);\n  np = 0;\n  const u32 nl_o = nl, nb_o = nb;\n"
    << "  tc_flatten(S, nl_o);  // every instance of the warp then finds a half's root in one hop\n"
    << "  u32 skip = 0;  // half labels that are no roots (they never become roots again)\n"
    << "  for (u32 l = 0; l < nl_o && l < 32u; ++l)\n"
    << "    skip |= ((S.lpar(l) & TcS::LOW) != l ? 1u : 0u) << l;\n";
  // signs and labels of the half-diamond vertices the middle row reads
  std::vector<char> used(V, 0);
  for (int v = Vo; v < V; ++v) {
    for (int u : D.fan[v]) used[u] = 1;
    for (int i : anti_at[v]) used[D.anti[i].first] = 1;
    for (int i : bedge_at[v]) used[D.bedge[i].first] = used[D.bedge[i].second] = 1;
  }
  const std::vector<int> slot = lab_slots(D, nullptr);  // where the table sweep left each label
  for (int u = 0; u < Vo; ++u)
    if (used[u])
      o << "  const u32 s" << u << " = TC_BIT(" << D.k[u] << ") ^ " << D.c[u] << "u, L" << u
        << " = *S.lab(TcK::OFF_LAB, " << slot[u] << ") & TcS::LOW;\n";
  // snapshot of the half-diamonds' union-find: the first SNAPW words of the
  // parents and the first word of odd flags in registers, the rest (many
  // half labels at d >= 8) in the [snap] region
  for (int w = 0; w < L.snapw; ++w)
    o << "  const u32 snap" << w << " = S.word(TcK::OFF_LPAR, " << w << ");\n";
  const bool even = d % 2 == 0;  // only even degrees keep odd-cycle flags
  o << "  const u32 nw = (nl_o + TcK::EPW - 1u) / TcK::EPW;\n"
    << "  for (u32 w = TcK::SNAPW; w < nw; ++w) S.word(TcK::OFF_SNAP, w) = S.word(TcK::OFF_LPAR, w);\n";
  if (even)
    o << "  const u32 osnap = S.word(TcK::OFF_ODD, 0), nwo = (nl_o + 31u) / 32u;\n"
      << "  for (u32 w = 1; w < nwo; ++w) S.word(TcK::OFF_SNAP + TcK::WLAB, w) = S.word(TcK::OFF_ODD, w);\n";
  else  // the half-diamonds' crossed boundary edges by their roots: one lookup each per instance
    o << "  for (u32 i = 0; i < nb_o; ++i) {\n"
      << "    const u32 e = S.word(TcK::OFF_BPAIR, i);\n"
      << "    S.word(TcK::OFF_BPAIR, i) = (S.lpar(e & 0xFFFFu) & TcS::LOW) | ((S.lpar(e >> 16) & TcS::LOW) << 16);\n"
      << "  }\n";
  // The per-lane loop: every instance restores the snapshot, sweeps the
  // middle row and classifies.  Emitted twice: warps whose half-diamonds left
  // at most 32 labels restore from registers only (the common case below
  // d = 8, and measured faster), the others also from the [snap] region.
  auto emit_lane_loop = [&](bool with_snap, const char *ind) {
    const std::string in(ind), in2 = in + "  ";
    o << in << "for (u32 j = 0; j < ireps; ++j) {\n";
    for (int w = 0; w < L.snapw; ++w)
      o << in2 << "S.word(TcK::OFF_LPAR, " << w << ") = snap" << w << ";\n";
    if (with_snap)
      o << in2 << "for (u32 w = TcK::SNAPW; w < nw; ++w) S.word(TcK::OFF_LPAR, w) = S.word(TcK::OFF_SNAP, w);\n";
    if (even) {
      o << in2 << "S.word(TcK::OFF_ODD, 0) = osnap;\n";
      if (with_snap)
        o << in2 << "for (u32 w = 1; w < TcK::WODD; ++w)\n"
          << in2 << "  S.word(TcK::OFF_ODD, w) = w < nwo ? S.word(TcK::OFF_SNAP + TcK::WLAB, w) : 0u;\n";
      else
        o << in2 << "for (u32 w = 1; w < TcK::WODD; ++w) S.word(TcK::OFF_ODD, w) = 0u;\n";
    }
    o << in2 << "nl = nl_o; nb = nb_o; np = 0;\n"
      << in2 << "const u32 sm = slo | ((lane + 32u * j) << ishift);\n";
    // the middle row starts from an empty join list
    for (int v = Vo; v < V; ++v) emit_vertex(v, in2.c_str(), "sm", flush_mid[v] != 0);
    o << in2 << "tc_unions(S, np);\n"
      << in2 << "const u64 key = tc_backend(S, nl, nb, err, skip);\n"
      << in2 << "failed += key == 0;\n"
      << in2 << "tc_hist_add<TcK::HASH>(key, hkeys, hcnt, gkeys, gcnt, gslots, gerr);\n"
      << in << "}\n";
  };
  o << "  if (nl_o <= 32u) {\n";
  emit_lane_loop(false, "    ");
  o << "  } else {\n";
  emit_lane_loop(true, "    ");
  o << "  }\n}\n";

  o << kKernelsSrc;
  return o.str();
}

std::string jit_compile_cubin(const std::string &src, std::string *log,
                              const std::vector<std::string> &extra) {
  // identical triangulations generate identical sources: compile once
  static std::mutex cache_mu;
  static std::map<std::string, std::pair<std::string, std::string>> cache;  // options + src -> (cubin, log)
  std::string key;
  for (const auto &x : extra) key += x + "\n";
  key += src;
  {
    std::lock_guard<std::mutex> g(cache_mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      if (log) *log = it->second.second;
      return it->second.first;
    }
  }
  std::string lg;
  std::string out = jit_compile_uncached(src, &lg, extra);
  if (log) *log = lg;
  if (!out.empty()) {
    std::lock_guard<std::mutex> g(cache_mu);
    cache.emplace(key, std::make_pair(out, lg));
  }
  return out;
}

std::string jit_compile_uncached(const std::string &src, std::string *log,
                                 const std::vector<std::string> &extra) {
  Nvrtc &nv = nvrtc();
  if (!nv.ok) {
    if (log) *log = "NVRTC library not found";
    return {};
  }
  nvrtcProgram prog;
  if (nv.create(&prog, src.c_str(), "tcurve_specialised.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    if (log) *log = "nvrtcCreateProgram failed";
    return {};
  }
  std::vector<const char *> opts = {"-arch=sm_103a", "--std=c++17", "-lineinfo", "--ptxas-options=-v"};
  for (const auto &x : extra) opts.push_back(x.c_str());
  nvrtcResult r = nv.compile(prog, (int)opts.size(), opts.data());
  size_t ls = 0;
  nv.log_size(prog, &ls);
  std::string lg(ls, '\0');
  if (ls) nv.log(prog, &lg[0]);
  while (!lg.empty() && lg.back() == '\0') lg.pop_back();  // the size counts the terminator
  if (log) *log = lg;
  std::string out;
  if (r == NVRTC_SUCCESS) {
    size_t cs = 0;
    nv.cubin_size(prog, &cs);
    out.resize(cs);
    nv.cubin(prog, &out[0]);
  }
  nv.destroy(&prog);
  return out;
}

// Configuration of the specialised kernels of a triangulation.  Scratch:
// global from d = 7 unless asked otherwise (TS_SCRATCH_*); blocks per SM from
// ts_set_occupancy, else the register budget measured fastest on GB300 for
// the degree (d = 7: 7 blocks of 128 threads, 72 registers; d = 8: 6, 80;
// d = 9: 4, 128), 4 for other degrees with global scratch, 2 with shared.
void jit_config(int d, int scratch, int occupancy, bool *global, int *min_blocks) {
  *global = scratch == TS_SCRATCH_GLOBAL || (scratch == TS_SCRATCH_AUTO && d >= kGlobalScratchFrom);
  int def = 2;
  if (*global) def = d == 7 ? 7 : d == 8 ? 6 : 4;
  *min_blocks = occupancy > 0 ? occupancy : def;
}

cudaError_t jit_prepare(ts_tri *t) {
  if (t->d > kMaxSpecialized) return cudaErrorNotSupported;
  std::lock_guard<std::mutex> g(t->jit_mu);
  if (t->jit) return cudaSuccess;
  Driver &dr = driver();
  if (!dr.ok) return cudaErrorNotSupported;
  cudaError_t e = cudaFree(0);  // make the primary context current
  if (e != cudaSuccess) return e;
  bool global = false;
  int minb = 2;
  jit_config(t->d, t->scratch, t->occupancy, &global, &minb);
  const std::string src = jit_source(t->dia, global, minb);
  const std::string cubin = jit_compile_cubin(src, &t->jit_log);
  if (cubin.empty()) return cudaErrorInvalidSource;
  auto mod = std::make_shared<JitModule>();
  mod->L = layout_for(t->dia, global);
  mod->global = global;
  if (dr.load(&mod->mod, cubin.data()) != CUDA_SUCCESS) return cudaErrorInvalidKernelImage;
  if (dr.get(&mod->real, mod->mod, "tc_real_schemes") != CUDA_SUCCESS ||
      dr.get(&mod->enumerate, mod->mod, "tc_enumerate") != CUDA_SUCCESS ||
      dr.get(&mod->blocks, mod->mod, "tc_enumerate_blocks") != CUDA_SUCCESS)
    return cudaErrorSymbolNotFound;
  const Layout &L = mod->L;
  mod->smem_real = global ? 0 : (size_t)L.words * 4 * L.threads;
  mod->smem_enum = mod->smem_real + (size_t)L.hash * 16 + 16;
  if (dr.set_attr(mod->real, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)mod->smem_real) !=
          CUDA_SUCCESS ||
      dr.set_attr(mod->enumerate, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                  (int)mod->smem_enum) != CUDA_SUCCESS ||
      dr.set_attr(mod->blocks, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES,
                  (int)mod->smem_enum) != CUDA_SUCCESS)
    return cudaErrorInvalidConfiguration;
  if (dr.occupancy(&mod->bpsm_real, mod->real, L.threads, mod->smem_real) != CUDA_SUCCESS ||
      dr.occupancy(&mod->bpsm_enum, mod->enumerate, L.threads, mod->smem_enum) != CUDA_SUCCESS ||
      dr.occupancy(&mod->bpsm_blocks, mod->blocks, L.threads, mod->smem_enum) != CUDA_SUCCESS ||
      mod->bpsm_real < 1 || mod->bpsm_enum < 1 || mod->bpsm_blocks < 1)
    return cudaErrorInvalidConfiguration;
  t->jit = mod;
  return cudaSuccess;
}

void jit_release(ts_tri *t) {
  std::lock_guard<std::mutex> g(t->jit_mu);
  t->jit.reset();
}

// Global scratch of one launch of a module that keeps it in global memory
// (grid x threads x words, stream-ordered; nothing for shared scratch).
struct JitScratch {
  const JitModule &m;
  unsigned grid;
  cudaStream_t st;
  uint32_t *p = nullptr;
  JitScratch(const JitModule &mm, unsigned g, cudaStream_t s) : m(mm), grid(g), st(s) {}
  cudaError_t alloc() {
    if (!m.global) return cudaSuccess;
    return scratch_alloc((void **)&p, (size_t)grid * m.L.words * m.L.threads * 4, st);
  }
  ~JitScratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

cudaError_t launch_real_schemes_jit(ts_tri *t, const uint64_t *signs, uint64_t n, uint64_t *codes,
                                    cudaStream_t st) {
  cudaError_t e = jit_prepare(t);
  if (e != cudaSuccess) return e;
  std::shared_ptr<JitModule> m = t->jit;
  const uint64_t want = (n + m->L.threads - 1) / m->L.threads;
  const uint64_t cap = (uint64_t)m->bpsm_real * sm_count_now();
  const unsigned grid = (unsigned)std::min(want, cap);
  JitScratch gs(*m, grid, st);
  if ((e = gs.alloc()) != cudaSuccess) return e;
  void *args[] = {(void *)&signs, (void *)&n, (void *)&codes, (void *)&t->d_err, (void *)&gs.p};
  if (driver().launch(m->real, grid, 1, 1, m->L.threads, 1, 1, (unsigned)m->smem_real, (CUstream)st,
                      args, nullptr) != CUDA_SUCCESS)
    return cudaErrorLaunchFailure;
  return cudaSuccess;
}

namespace {

// One launch of the per-mask sweep kernel over masks m(k), k in [lo, hi).
cudaError_t enumerate_range(JitModule &m, ts_hist *h, uint64_t lo, uint64_t hi, uint32_t flags,
                            cudaStream_t st) {
  const uint64_t total = hi - lo;
  const uint64_t chunk = (uint64_t)m.L.threads * 16;
  const uint64_t want = (total + chunk - 1) / chunk;
  const uint64_t cap = (uint64_t)m.bpsm_enum * sm_count_now();
  const unsigned grid = (unsigned)std::min(want, cap);
  cudaError_t e = cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  JitScratch gs(m, grid, st);
  if ((e = gs.alloc()) != cudaSuccess) return e;
  uint64_t slots = h->slots;
  void *args[] = {(void *)&lo,       (void *)&total,       (void *)&flags,
                  (void *)&h->d_keys, (void *)&h->d_counts, (void *)&slots,
                  (void *)&h->d_err,  (void *)&h->d_failed, (void *)&h->d_work,
                  (void *)&gs.p};
  if (driver().launch(m.enumerate, grid, 1, 1, m.L.threads, 1, 1, (unsigned)m.smem_enum,
                      (CUstream)st, args, nullptr) != CUDA_SUCCESS)
    return cudaErrorLaunchFailure;
  return cudaSuccess;
}

// One launch of the block sweep: masks (h << oshift) | (t << ishift) for
// h in [hi0, hi0 + n_hi) and t < 32 * ireps (all middle-row patterns).
cudaError_t enumerate_blocks(JitModule &m, ts_hist *h, uint64_t hi0, uint64_t n_hi, uint32_t oshift,
                             uint32_t ishift, uint32_t ireps, uint32_t flags, cudaStream_t st) {
  const uint64_t warps = m.L.threads / 32;
  const uint64_t want = (n_hi + warps - 1) / warps;
  const uint64_t cap = (uint64_t)m.bpsm_blocks * sm_count_now();
  const unsigned grid = (unsigned)std::min(want, cap);
  cudaError_t e = cudaMemsetAsync(h->d_work, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  JitScratch gs(m, grid, st);
  if ((e = gs.alloc()) != cudaSuccess) return e;
  uint64_t slots = h->slots;
  void *args[] = {(void *)&hi0,       (void *)&n_hi,      (void *)&oshift,     (void *)&ishift,
                  (void *)&ireps,     (void *)&flags,     (void *)&h->d_keys,  (void *)&h->d_counts,
                  (void *)&slots,     (void *)&h->d_err,  (void *)&h->d_failed, (void *)&h->d_work,
                  (void *)&gs.p};
  if (driver().launch(m.blocks, grid, 1, 1, m.L.threads, 1, 1, (unsigned)m.smem_enum, (CUstream)st,
                      args, nullptr) != CUDA_SUCCESS)
    return cudaErrorLaunchFailure;
  return cudaSuccess;
}

}  // namespace

// Sweeps run whole middle-row blocks through the block sweep and the ragged
// head and tail of the range through the per-mask kernel.  In terms of the
// sweep index k, the mask m(k) is (h << oshift) | (t << ishift) with
// t = k mod 2^ib the middle-row pattern (ib free middle-row bits) and
// h = k >> ib: ib = d + 1 without flags, d with TS_ENUM_FLIP (bit 0 fixed),
// d - 1 with TS_ENUM_REDUCED (bits 0, 1 and d + 1 fixed), d + 1 with
// TS_ENUM_ORBITS (bit d + 1 fixed, h the block's high part with its pivots
// zero, tc_orbit_high).
cudaError_t launch_enumerate_jit(ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                                 cudaStream_t st) {
  cudaError_t e = jit_prepare(t);
  if (e != cudaSuccess) return e;
  std::shared_ptr<JitModule> m = t->jit;
  const int d = t->d;
  uint32_t ib = d + 1, ishift = 0, oshift = d + 1;
  if (flags & TS_ENUM_FLIP) { ib = d; ishift = 1; oshift = d + 1; }
  if (flags & TS_ENUM_REDUCED) { ib = d - 1; ishift = 2; oshift = d + 2; }
  if (flags & TS_ENUM_ORBITS) { ib = d + 1; ishift = 0; oshift = d + 2; }  // every pattern
  if (ib < 5 || (flags & TS_ENUM_SPLITMIX))  // fewer patterns than lanes / sampled masks
    return enumerate_range(*m, h, lo, hi, flags, st);
  const uint64_t a = ((lo + (1ull << ib) - 1) >> ib) << ib, b = (hi >> ib) << ib;
  if (a >= b) return enumerate_range(*m, h, lo, hi, flags, st);
  if (lo < a && (e = enumerate_range(*m, h, lo, a, flags, st)) != cudaSuccess) return e;
  uint64_t h0 = a >> ib, h1 = b >> ib;  // whole blocks [h0, h1)
  if ((flags & TS_ENUM_FLIP) && !(flags & TS_ENUM_REDUCED) && t->np - 1 - ib < 63) {
    // Global sign flip: block h (masks with bit 0 clear) and block M - h
    // (all high bits complemented) hold one representative of each class
    // {sigma, ~sigma} whose high part is h or M - h; flipping the second
    // block's masks gives block h with bit 0 set.  So a pair of blocks in
    // the range is swept as the one unreduced block h with all 2^(d+1)
    // middle-row patterns: the same schemes (the flip keeps the curve), and
    // twice the patterns per half-diamond sweep.  Paired: h in [p, q]
    // (symmetric about M / 2, both ends in the range); the rest as before.
    const uint64_t M = (1ull << (t->np - 1 - ib)) - 1;
    const uint64_t p = std::max<uint64_t>(h0, h1 > M ? 0 : M + 1 - h1);
    const uint64_t q1 = std::min<uint64_t>(h1, h0 > M ? 0 : M - h0 + 1);  // q + 1
    if (p < q1) {
      const uint64_t half = (q1 - p) / 2;  // q1 - p is even: p + q = M, M odd
      if (h0 < p &&
          (e = enumerate_blocks(*m, h, h0, p - h0, oshift, ishift, (1u << ib) / 32u, 0, st)) !=
              cudaSuccess)
        return e;
      if ((e = enumerate_blocks(*m, h, p, half, d + 1, 0, (1u << (d + 1)) / 32u, 0, st)) !=
          cudaSuccess)
        return e;
      h0 = q1;
    }
  }
  if (h0 < h1 &&
      (e = enumerate_blocks(*m, h, h0, h1 - h0, oshift, ishift, (1u << ib) / 32u,
                            flags & (TS_ENUM_ORBITS | 0xFFFF00u), st)) != cudaSuccess)
    return e;
  if (b < hi && (e = enumerate_range(*m, h, b, hi, flags, st)) != cudaSuccess) return e;
  return cudaSuccess;
}


// ---------------------------------------------------------------------------
// Specialised code for batches of many triangulations (ts_batch).
//
// Every distinct triangulation of a batch gets its own relocatable object:
// the per-mask sweep of Algorithm 1 as straight-line code (as tc_classify
// above, for one to three sign words), the union pass and the narrow or wide
// back end, all inside a namespace of its own and exported as one plain
// device function tcj_<i>.  One more object per degree holds the persistent
// kernel tcj_jobs, which pulls (job, chunk) work items, draws the splitmix64
// sign vectors, calls the job's function through a switch on its index and
// adds the codes to the job's histogram.  The objects are compiled by NVRTC
// in parallel host threads and linked per degree with nvJitLink, so one
// kernel per degree serves every job of that degree.

namespace {

constexpr int kJobThreads = 128;  // block size (the stride of the word-interleaved scratch)

struct JitLink {
  void *h = nullptr;
  nvJitLinkResult (*create)(nvJitLinkHandle *, uint32_t, const char **) = nullptr;
  nvJitLinkResult (*destroy)(nvJitLinkHandle *) = nullptr;
  nvJitLinkResult (*add)(nvJitLinkHandle, nvJitLinkInputType, const void *, size_t,
                         const char *) = nullptr;
  nvJitLinkResult (*complete)(nvJitLinkHandle) = nullptr;
  nvJitLinkResult (*cubin_size)(nvJitLinkHandle, size_t *) = nullptr;
  nvJitLinkResult (*cubin)(nvJitLinkHandle, void *) = nullptr;
  nvJitLinkResult (*log_size)(nvJitLinkHandle, size_t *) = nullptr;
  nvJitLinkResult (*log)(nvJitLinkHandle, char *) = nullptr;
  bool ok = false;
};

JitLink &jitlink() {
  static JitLink j;
  static std::once_flag once;
  std::call_once(once, [] {
    const char *names[] = {"libnvJitLink.so.13", "libnvJitLink.so",
                           "/usr/local/cuda/lib64/libnvJitLink.so.13",
                           "/usr/local/cuda/lib64/libnvJitLink.so"};
    for (const char *nm : names)
      if ((j.h = dlopen(nm, RTLD_NOW | RTLD_GLOBAL))) break;
    if (!j.h) return;
    auto sym = [&](const char *versioned, const char *plain) {
      void *f = dlsym(j.h, versioned);
      return f ? f : dlsym(j.h, plain);
    };
    j.create = (decltype(j.create))sym("__nvJitLinkCreate_13_0", "nvJitLinkCreate");
    j.destroy = (decltype(j.destroy))sym("__nvJitLinkDestroy_13_0", "nvJitLinkDestroy");
    j.add = (decltype(j.add))sym("__nvJitLinkAddData_13_0", "nvJitLinkAddData");
    j.complete = (decltype(j.complete))sym("__nvJitLinkComplete_13_0", "nvJitLinkComplete");
    j.cubin_size =
        (decltype(j.cubin_size))sym("__nvJitLinkGetLinkedCubinSize_13_0", "nvJitLinkGetLinkedCubinSize");
    j.cubin = (decltype(j.cubin))sym("__nvJitLinkGetLinkedCubin_13_0", "nvJitLinkGetLinkedCubin");
    j.log_size = (decltype(j.log_size))sym("__nvJitLinkGetErrorLogSize_13_0", "nvJitLinkGetErrorLogSize");
    j.log = (decltype(j.log))sym("__nvJitLinkGetErrorLog_13_0", "nvJitLinkGetErrorLog");
    j.ok = j.create && j.destroy && j.add && j.complete && j.cubin_size && j.cubin && j.log_size &&
           j.log;
  });
  return j;
}

// One job of a batch as the generated code sees it: the layout of the host's
// job table (72 bytes, DevJob of batch.cu).
const char kJobStructSrc[] = R"TCJS(
struct TcjJob {
  const unsigned *tab;
  unsigned long long n, base;          // sign vectors; splitmix64 counter of the first
  unsigned long long *codes;           // per-instance codes (or null)
  unsigned long long *hkeys;           // the job's histogram
  unsigned long long *hcnt;
  unsigned long long hslots, chunk0;   // its slots; its first work item
  unsigned fn, pad;                    // index of its specialised function
};
)TCJS";

// Scratch layout of the batch kernels: one label per vertex (the wide back
// end reuses that region), 128-thread blocks, global memory.
Layout job_layout(int d) {
  Layout L = tc_layout(d, true, kJobThreads);
  L.threads = kJobThreads;
  return L;
}

// Resident 128-thread blocks per SM the batch kernels of degree d are
// compiled for (their register budget: 65536 / (128 x blocks) registers).
int job_min_blocks(int d) { return d <= 5 ? 6 : d <= 10 ? 4 : 3; }

// Registers per thread for `blocks` resident 128-thread blocks per SM.
int job_max_registers(int blocks) {
  const int r = 65536 / (kJobThreads * blocks);
  return std::min(255, r / 8 * 8);
}

// Words of global scratch per block: the per-thread layout.
size_t job_slab_words(const Layout &L) { return (size_t)L.words * L.threads; }

}  // namespace

std::string jit_job_source(const Diamond &D, int idx, int min_blocks) {
  const Layout L = job_layout(D.d);
  const int d = D.d, V = D.V;
  if (L.sw > 3 || L.cw > 4) return std::string();
  std::ostringstream o;
  o << "// T-curve real-scheme function for one triangulation of " << d
    << "*Delta_2 in a batch (generated, relocatable)\n";
  o << "namespace tcj" << idx << " {\n";
  emit_traits(o, L, d, V, true, min_blocks);
  o << "#define TC_HEAVY_FN __forceinline__\n";
  o << kRuntimeSrc;
  o << "#define TC_BIT(k) ((((k) < 32 ? w0 : (k) < 64 ? w1 : (k) < 96 ? w2 : (k) < 128 ? w3 : "
       "(k) < 160 ? w4 : w5) >> ((k) & 31)) & 1u)\n"
    << "typedef TcScratch<TcK> TcS;\n\n";
  o << "__device__ __forceinline__ void classify(u64 sg0, u64 sg1, u64 sg2, const TcS &S, u32 &err,\n"
    << "                                         u64 *code) {\n"
    << "  const u32 w0 = (u32)sg0, w1 = (u32)(sg0 >> 32), w2 = (u32)sg1, w3 = (u32)(sg1 >> 32),\n"
    << "            w4 = (u32)sg2, w5 = (u32)(sg2 >> 32);\n"
    << "  (void)w2; (void)w3; (void)w4; (void)w5;\n"
    << "  u32 nl = 0, nb = 0, np = 0;\n  tc_clear_odd(S);\n";
  VertexEmitter em(D, o);
  const std::vector<char> flush = flush_schedule(D, 0, V, L.pcap);
  for (int v = 0; v < V; ++v) em.emit(v, "  ", nullptr, flush[v] != 0);
  o << "  tc_unions(S, np);\n";
  if (L.wide)
    o << "  tc_backend_wide(S, nl, nb, err, code);\n";
  else
    o << "  code[0] = tc_backend(S, nl, nb, err);\n";
  o << "}\n\n";
  o << kJobStructSrc;
  o << R"TCJF(
// One work item of a job: sign vectors first .. first + chunk - 1 (those below
// the job's count), drawn from the job's splitmix64 stream, classified by the
// sweep above and added to the job's histogram (warp-aggregated); returns
// the number of failed instances.
__device__ __forceinline__ unsigned long long chunk_body(const TcjJob *J, unsigned long long first,
                                                         unsigned chunk, unsigned *scr,
                                                         unsigned *err_word) {
  const TcS S{scr};
  const u32 lane = threadIdx.x & 31u;
  const u64 top = tc_top_mask(TcK::NPOINTS, TcK::W);
  u32 err = 0;
  unsigned long long failed = 0;
  for (unsigned k = 0; k < chunk; k += TcK::THREADS) {
    const u64 idx = first + k + threadIdx.x;
    u64 code[TcK::CW];
#pragma unroll
    for (u32 w = 0; w < TcK::CW; ++w) code[w] = 0;
    if (idx < J->n) {
      u64 sg[3] = {0, 0, 0};
#pragma unroll
      for (u32 w = 0; w < TcK::W; ++w) sg[w] = tc_splitmix64((J->base + idx) * TcK::W + w);
      sg[TcK::W - 1] &= top;
      classify(sg[0], sg[1], sg[2], S, err, code);
      u64 any = 0;
#pragma unroll
      for (u32 w = 0; w < TcK::CW; ++w) {
        any |= code[w];
        if (J->codes) J->codes[idx * TcK::CW + w] = code[w];
      }
      failed += any == 0;
    }
    if (TcK::CW == 1) {
      const unsigned peers = __match_any_sync(0xffffffffu, code[0]);
      if (code[0] != 0 && lane == (u32)(__ffs(peers) - 1))
        tc_global_add(J->hkeys, J->hcnt, J->hslots, err_word, code[0], (u64)__popc(peers));
    } else {
      tc_hist_add_wide<TcK::CW>(code, J->hkeys, J->hcnt, J->hslots, err_word);
    }
  }
  if (err) atomicOr(err_word, err);
  return failed;
}
)TCJF";
  o << "}  // namespace tcj" << idx << "\n\n";
  o << "extern \"C\" __device__ unsigned long long tcj_" << idx
    << "(const void *job, unsigned long long first, unsigned chunk, unsigned int *scr,\n"
    << "    unsigned int *err_word) {\n"
    << "  return tcj" << idx << "::chunk_body(static_cast<const tcj" << idx
    << "::TcjJob *>(job), first, chunk, scr, err_word);\n"
    << "}\n";
  return o.str();
}

std::string jit_jobs_kernel_source(int d, int nfn, int min_blocks) {
  const Layout L = job_layout(d);
  std::ostringstream o;
  o << "// T-curve batch kernel of degree " << d << " over " << nfn
    << " specialised functions (generated, relocatable)\n";
  o << kJobStructSrc;
  for (int i = 0; i < nfn; ++i)
    o << "extern \"C\" __device__ unsigned long long tcj_" << i
      << "(const void *, unsigned long long, unsigned, unsigned int *, unsigned int *);\n";
  o << "#define TCJ_THREADS " << L.threads << "u\n#define TCJ_SLAB " << (size_t)L.words * L.threads
    << "ull\n#define TCJ_MINB " << min_blocks << "\n";
  o << R"TCJOBS(
// Persistent kernel of the degree's jobs: blocks pull work items (job, chunk)
// from a counter; the job's own function classifies the item's sign vectors.
extern "C" __global__ void __launch_bounds__(TCJ_THREADS, TCJ_MINB)
    tcj_jobs(const TcjJob *__restrict__ jobs, unsigned njobs, unsigned long long total_items,
             unsigned chunk, unsigned long long *work, unsigned *err_word,
             unsigned long long *failed_word, unsigned *gscr) {
  typedef unsigned long long u64;
  __shared__ u64 slot;
  unsigned *scr = gscr + (u64)blockIdx.x * TCJ_SLAB + threadIdx.x;
  u64 failed = 0;
  for (;;) {
    if (threadIdx.x == 0) slot = atomicAdd(work, 1ull);
    __syncthreads();
    const u64 c = slot;
    __syncthreads();
    if (c >= total_items) break;
    unsigned lo = 0, hi = njobs;  // the job holding item c: last j with chunk0 <= c
    while (hi - lo > 1) {
      const unsigned mid = (lo + hi) / 2;
      if (jobs[mid].chunk0 <= c) lo = mid; else hi = mid;
    }
    const TcjJob *J = jobs + lo;
    const u64 first = (c - J->chunk0) * (u64)chunk;
    switch (J->fn) {
)TCJOBS";
  for (int i = 0; i < nfn; ++i)
    o << "      case " << i << "u: failed += tcj_" << i << "(J, first, chunk, scr, err_word); break;\n";
  o << R"TCJOBS(      default:
        if (threadIdx.x == 0) atomicOr(err_word, 1u);  // no function: an internal error
    }
  }
  if (failed) atomicAdd(failed_word, failed);
}
)TCJOBS";
  return o.str();
}

struct JitJobsModule {
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
  int d = 0, bpsm = 0;
  size_t slab_words = 0;
  ~JitJobsModule() {
    if (mod && driver().ok) driver().unload(mod);
  }
};

namespace {

// Compile the sources in parallel host threads (NVRTC is thread-safe);
// returns false and the first failure's log if any source fails, else true
// and the compiler logs (ptxas resource lines) of all objects.
bool compile_parallel(const std::vector<std::string> &srcs,
                      const std::vector<std::vector<std::string>> &opts,
                      std::vector<std::string> &cubins, std::string *log) {
  cubins.assign(srcs.size(), std::string());
  std::vector<std::string> logs(srcs.size());
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t i; (i = next.fetch_add(1)) < srcs.size();)
      cubins[i] = jit_compile_cubin(srcs[i], &logs[i], opts[i]);
  };
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nth = std::min<size_t>(hw, srcs.size());
  std::vector<std::thread> pool;
  for (size_t t = 1; t < nth; ++t) pool.emplace_back(work);
  work();
  for (auto &t : pool) t.join();
  for (size_t i = 0; i < srcs.size(); ++i)
    if (cubins[i].empty()) {
      if (log) *log = "compile of batch object " + std::to_string(i) + " failed:\n" + logs[i];
      return false;
    }
  if (log) {
    log->clear();
    for (size_t i = 0; i < srcs.size(); ++i) *log += "object " + std::to_string(i) + ":\n" + logs[i];
  }
  return true;
}

// Link relocatable cubins into one cubin for sm_103a.
std::string link_cubins(const std::vector<const std::string *> &objs, std::string *log) {
  JitLink &jl = jitlink();
  if (!jl.ok) {
    if (log) *log = "nvJitLink library not found";
    return {};
  }
  nvJitLinkHandle h = nullptr;
  const char *opts[] = {"-arch=sm_103a"};
  if (jl.create(&h, 1, opts) != NVJITLINK_SUCCESS) {
    if (log) *log = "nvJitLinkCreate failed";
    return {};
  }
  bool ok = true;
  for (size_t i = 0; i < objs.size() && ok; ++i) {
    const std::string name = "tcj" + std::to_string(i);
    ok = jl.add(h, NVJITLINK_INPUT_CUBIN, objs[i]->data(), objs[i]->size(), name.c_str()) ==
         NVJITLINK_SUCCESS;
  }
  if (ok) ok = jl.complete(h) == NVJITLINK_SUCCESS;
  std::string out;
  if (ok) {
    size_t n = 0;
    ok = jl.cubin_size(h, &n) == NVJITLINK_SUCCESS;
    if (ok) {
      out.resize(n);
      ok = jl.cubin(h, &out[0]) == NVJITLINK_SUCCESS;
    }
  }
  if (!ok) {
    size_t n = 0;
    std::string lg;
    if (jl.log_size(h, &n) == NVJITLINK_SUCCESS && n) {
      lg.resize(n);
      jl.log(h, &lg[0]);
    }
    if (log) *log = "nvJitLink failed:\n" + lg;
    out.clear();
  }
  jl.destroy(&h);
  return out;
}

}  // namespace

std::string jit_jobs_link(const std::vector<const Diamond *> &tris, std::string *log) {
  if (tris.empty()) return {};
  const int d = tris[0]->d;
  std::vector<std::string> srcs;
  std::vector<std::vector<std::string>> opts;
  const int mb = job_min_blocks(d);
  const std::vector<std::string> o = {"-rdc=true", "-maxrregcount=" + std::to_string(job_max_registers(mb))};
  for (size_t i = 0; i < tris.size(); ++i) {
    srcs.push_back(jit_job_source(*tris[i], (int)i, mb));
    if (srcs.back().empty()) {
      if (log) *log = "no batch source for this degree";
      return {};
    }
    opts.push_back(o);
  }
  srcs.push_back(jit_jobs_kernel_source(d, (int)tris.size(), mb));
  opts.push_back(o);
  std::vector<std::string> cubins;
  std::string clog;
  if (!compile_parallel(srcs, opts, cubins, &clog)) {
    if (log) *log = clog;
    return {};
  }
  std::vector<const std::string *> objs;
  for (auto &c : cubins) objs.push_back(&c);
  std::string llog;
  std::string out = link_cubins(objs, &llog);
  if (log) *log = out.empty() ? llog : clog;
  return out;
}

cudaError_t jit_jobs_build(const std::vector<std::vector<const Diamond *>> &groups,
                           const std::vector<int> &min_blocks,
                           std::vector<std::shared_ptr<JitJobsModule>> *mods,
                           std::vector<std::string> *logs) {
  mods->assign(groups.size(), nullptr);
  logs->assign(groups.size(), std::string());
  Driver &dr = driver();
  if (!dr.ok) return cudaErrorNotSupported;
  cudaError_t e = cudaFree(0);  // make the primary context current
  if (e != cudaSuccess) return e;
  // every object of every group in one parallel compile, then one link per group
  std::vector<std::string> srcs;
  std::vector<std::vector<std::string>> opts;
  std::vector<size_t> first(groups.size() + 1, 0);
  for (size_t g = 0; g < groups.size(); ++g) {
    first[g] = srcs.size();
    if (groups[g].empty()) continue;
    const int d = groups[g][0]->d;
    const int mb = g < min_blocks.size() && min_blocks[g] > 0 ? min_blocks[g] : job_min_blocks(d);
    const std::vector<std::string> o = {"-rdc=true",
                                        "-maxrregcount=" + std::to_string(job_max_registers(mb))};
    for (size_t i = 0; i < groups[g].size(); ++i) {
      srcs.push_back(jit_job_source(*groups[g][i], (int)i, mb));
      opts.push_back(o);
    }
    srcs.push_back(jit_jobs_kernel_source(d, (int)groups[g].size(), mb));
    opts.push_back(o);
  }
  first[groups.size()] = srcs.size();
  for (const auto &src : srcs)
    if (src.empty()) return cudaErrorNotSupported;
  std::vector<std::string> cubins(srcs.size());
  std::string lg;
  if (!compile_parallel(srcs, opts, cubins, &lg)) {
    for (auto &l : *logs) l = lg;
    return cudaErrorInvalidSource;
  }
  lg.clear();
  for (size_t g = 0; g < groups.size(); ++g) {
    if (groups[g].empty()) continue;
    std::vector<const std::string *> objs;
    for (size_t i = first[g]; i < first[g + 1]; ++i) objs.push_back(&cubins[i]);
    const std::string linked = link_cubins(objs, &(*logs)[g]);
    if (linked.empty()) continue;
    auto m = std::make_shared<JitJobsModule>();
    m->d = groups[g][0]->d;
    m->slab_words = job_slab_words(job_layout(m->d));
    if (dr.load(&m->mod, linked.data()) != CUDA_SUCCESS ||
        dr.get(&m->fn, m->mod, "tcj_jobs") != CUDA_SUCCESS ||
        dr.occupancy(&m->bpsm, m->fn, kJobThreads, 0) != CUDA_SUCCESS || m->bpsm < 1) {
      (*logs)[g] = "loading the linked batch module failed";
      continue;
    }
    (*mods)[g] = m;
  }
  return cudaSuccess;
}

int jit_jobs_threads() { return kJobThreads; }
void jit_jobs_attrs(const JitJobsModule &m, int *regs, int *local_bytes) {
  *regs = *local_bytes = 0;
  driver().get_attr(regs, CU_FUNC_ATTRIBUTE_NUM_REGS, m.fn);
  driver().get_attr(local_bytes, CU_FUNC_ATTRIBUTE_LOCAL_SIZE_BYTES, m.fn);
}
int jit_jobs_blocks_per_sm(const JitJobsModule &m) { return m.bpsm; }
size_t jit_jobs_slab_bytes(const JitJobsModule &m) { return m.slab_words * 4; }

cudaError_t jit_jobs_launch(const JitJobsModule &m, unsigned grid, const void *jobs, uint32_t njobs,
                            uint64_t items, uint32_t chunk, unsigned long long *work, uint32_t *err,
                            unsigned long long *failed, uint32_t *scratch, cudaStream_t st) {
  void *args[] = {(void *)&jobs, (void *)&njobs, (void *)&items, (void *)&chunk,
                  (void *)&work, (void *)&err,   (void *)&failed, (void *)&scratch};
  if (driver().launch(m.fn, grid, 1, 1, kJobThreads, 1, 1, 0, (CUstream)st, args, nullptr) !=
      CUDA_SUCCESS)
    return cudaErrorLaunchFailure;
  return cudaSuccess;
}

}  // namespace tcurve
