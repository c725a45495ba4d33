// host.cpp -- host side of libtcurve: validation of the input triangulation,
// construction of the reflected triangulation T^diamond (Alg. 1, line 1) and
// of the per-vertex tables the kernels stage into shared memory, device
// object management and the C ABI of include/tcurve.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"
#include "tc_layout.h"

using namespace tcurve;

namespace {

int lattice_index(int d, int i, int j) { return j * (d + 1) - j * (j - 1) / 2 + i; }

int harnack(int d) { return (d - 1) * (d - 2) / 2 + 1; }

struct Pt {
  int x, y;
  bool operator<(const Pt &o) const { return y != o.y ? y < o.y : x < o.x; }
  bool operator==(const Pt &o) const { return x == o.x && y == o.y; }
};

long cross(int ax, int ay, int bx, int by) { return (long)ax * by - (long)ay * bx; }

// Triangles of T from the edge list: 3-cliques of area 1/2 (unimodular).
// Returns false if the edges do not form a unimodular triangulation.
bool triangles_of(int d, const int32_t *e, int n_edges, std::vector<std::array<Pt, 3>> &tris) {
  std::map<Pt, std::set<Pt>> nb;
  for (int r = 0; r < n_edges; ++r) {
    Pt a{e[4 * r], e[4 * r + 1]}, b{e[4 * r + 2], e[4 * r + 3]};
    for (const Pt &p : {a, b})
      if (p.x < 0 || p.y < 0 || p.x + p.y > d) return false;
    if (a == b || nb[a].count(b)) return false;
    nb[a].insert(b);
    nb[b].insert(a);
  }
  if ((int)nb.size() != (d + 1) * (d + 2) / 2) return false;  // every point used
  std::map<std::pair<Pt, Pt>, int> uses;
  for (auto &kv : nb) {
    const Pt &a = kv.first;
    for (const Pt &b : kv.second) {
      if (!(a < b)) continue;
      for (const Pt &c : kv.second) {
        if (!(b < c) || !nb[b].count(c)) continue;
        long o = cross(b.x - a.x, b.y - a.y, c.x - a.x, c.y - a.y);
        if (o != 1 && o != -1) continue;
        tris.push_back(o > 0 ? std::array<Pt, 3>{a, b, c} : std::array<Pt, 3>{a, c, b});
        uses[{a, b}]++;
        uses[{a, c}]++;
        uses[{b, c}]++;
      }
    }
  }
  if ((int)tris.size() != d * d) return false;
  for (auto &kv : nb)
    for (const Pt &b : kv.second) {
      const Pt &a = kv.first;
      if (!(a < b)) continue;
      bool side = (a.x == 0 && b.x == 0) || (a.y == 0 && b.y == 0) ||
                  (a.x + a.y == d && b.x + b.y == d);
      auto it = uses.find({a, b});
      int u = it == uses.end() ? 0 : it->second;
      if (u != (side ? 1 : 2)) return false;
    }
  return true;
}

// Build T^diamond (Alg. 1, line 1) in sweep order.
//
// Sweep order: the lower half (y < 0) row by row upwards, then the upper half
// (y > 0) row by row downwards, then the middle row y = 0; x ascending in
// every row.  No edge of T^diamond crosses the x-axis (each edge lies in one
// quadrant), so the two halves never meet before the middle row.  The "back
// neighbours" of v (neighbours earlier in the sweep) then lie in one angular
// range around v, listed counter-clockwise from the +x direction; two
// consecutive entries span a triangle with v unless the range is cut by the
// boundary of the diamond, which the link bit records.  Every vertex except
// the first of each half, (0,-d) and (0,d), has a back neighbour, and those two
// are antipodal, which the region-tree construction relies on.
bool build_diamond(int d, const std::vector<std::array<Pt, 3>> &tris, Diamond &D) {
  std::vector<Pt> verts;
  for (int y = -d; y <= -1; ++y)
    for (int x = -d; x <= d; ++x)
      if (std::abs(x) + std::abs(y) <= d) verts.push_back({x, y});
  for (int y = d; y >= 1; --y)
    for (int x = -d; x <= d; ++x)
      if (std::abs(x) + std::abs(y) <= d) verts.push_back({x, y});
  for (int x = -d; x <= d; ++x) verts.push_back({x, 0});
  const int V = (int)verts.size();
  std::map<Pt, int> pos;
  for (int v = 0; v < V; ++v) pos[verts[v]] = v;

  static const int qx[4] = {1, -1, -1, 1}, qy[4] = {1, 1, -1, -1};
  std::set<std::array<int, 3>> dtris;
  std::vector<std::set<int>> adj(V);
  for (int q = 0; q < 4; ++q)
    for (auto &tr : tris) {
      std::array<int, 3> id;
      for (int k = 0; k < 3; ++k) id[k] = pos.at({qx[q] * tr[k].x, qy[q] * tr[k].y});
      for (int k = 0; k < 3; ++k) {
        adj[id[k]].insert(id[(k + 1) % 3]);
        adj[id[(k + 1) % 3]].insert(id[k]);
      }
      std::sort(id.begin(), id.end());
      dtris.insert(id);
    }
  if ((int)dtris.size() != 4 * d * d) return false;
  auto has_tri = [&](int a, int b, int c) {
    std::array<int, 3> id{a, b, c};
    std::sort(id.begin(), id.end());
    return dtris.count(id) > 0;
  };
  D.d = d;
  D.V = V;
  D.x.resize(V);
  D.y.resize(V);
  D.k.resize(V);
  D.c.resize(V);
  D.fan.assign(V, {});
  D.link.assign(V, {});
  for (int v = 0; v < V; ++v) {
    int x = verts[v].x, y = verts[v].y, i = std::abs(x), j = std::abs(y);
    D.x[v] = x;
    D.y[v] = y;
    D.k[v] = lattice_index(d, i, j);
    D.c[v] = ((x < 0) ? (i & 1) : 0) ^ ((y < 0) ? (j & 1) : 0);  // Eq. 2
  }
  for (int v = 0; v < V; ++v) {
    std::vector<int> back;
    for (int u : adj[v])
      if (u < v) back.push_back(u);
    // counter-clockwise angle from the +x direction, in (0, 2 pi]
    auto half = [](int dx, int dy) { return (dy > 0 || (dy == 0 && dx < 0)) ? 0 : 1; };
    std::sort(back.begin(), back.end(), [&](int a, int b) {
      int ax = verts[a].x - verts[v].x, ay = verts[a].y - verts[v].y;
      int bx = verts[b].x - verts[v].x, by = verts[b].y - verts[v].y;
      int ha = half(ax, ay), hb = half(bx, by);
      if (ha != hb) return ha < hb;
      return cross(ax, ay, bx, by) > 0;
    });
    D.fan[v] = back;
    for (size_t n = 0; n < back.size(); ++n)
      D.link[v].push_back((n > 0 && has_tri(v, back[n - 1], back[n])) ? 1 : 0);
  }
  for (int v = 0; v < V; ++v) {
    const Pt p = verts[v];
    if (std::abs(p.x) + std::abs(p.y) != d) continue;
    int w = pos.at({-p.x, -p.y});
    if (v < w) D.anti.push_back({v, w});
  }
  std::set<std::pair<int, int>> seen;
  for (int a = 0; a < V; ++a)
    for (int b : adj[a]) {
      if (b < a) continue;
      const Pt pa = verts[a], pb = verts[b];
      if (std::abs(pa.x) + std::abs(pa.y) != d || std::abs(pb.x) + std::abs(pb.y) != d) continue;
      int a2 = pos.at({-pa.x, -pa.y}), b2 = pos.at({-pb.x, -pb.y});
      if (seen.count({std::min(a2, b2), std::max(a2, b2)})) continue;
      seen.insert({a, b});
      D.bedge.push_back({a, b});
    }
  return (int)D.anti.size() == 2 * d && (int)D.bedge.size() == 2 * d;
}

}  // namespace

namespace tcurve {
int vertex_pushes(const Diamond &D, int v) {
  const auto &lk = D.link[v];
  const int m = (int)D.fan[v].size();
  int f0 = 0, f1 = m ? 1 : 0;  // most run starts so far, last entry 0 / 1
  for (int i = 1; i < m; ++i) {
    const int n0 = std::max(f0, f1), n1 = std::max(f0 + 1, f1 + (lk[i] ? 0 : 1));
    f0 = n0;
    f1 = n1;
  }
  const int starts = std::max(f0, f1);
  int anti = 0;
  for (auto &p : D.anti) anti += p.second == v;
  return (starts > 1 ? starts - 1 : 0) + anti;
}

std::vector<char> flush_schedule(const Diamond &D, int v0, int v1, int pcap) {
  std::vector<char> flush(D.V, 0);
  int acc = 0;
  for (int v = v0; v < v1; ++v) {
    const int p = vertex_pushes(D, v);
    if (acc + p > pcap) {
      flush[v] = 1;
      acc = 0;
    }
    acc += p;
  }
  return flush;
}

// Label slots of the table-driven sweep.  A vertex's label is written when
// the sweep reaches it and read by later vertices: those whose fan holds it,
// its antipodal partner and the far end of a boundary edge.  Its slot is
// taken at its own step and freed after its last reader, and every vertex
// takes the lowest free slot (greedy colouring of the live intervals in sweep
// order), so the sweep touches only as many label slots as are live at once:
// about two rows of T^diamond plus the boundary vertices that wait for their
// partners, instead of one per vertex.
std::vector<int> lab_slots(const Diamond &D, int *nslots) {
  const int V = D.V;
  std::vector<int> last(V);
  for (int v = 0; v < V; ++v) last[v] = v;
  for (int w = 0; w < V; ++w)
    for (int u : D.fan[w]) last[u] = std::max(last[u], w);
  for (auto &p : D.anti) last[p.first] = std::max(last[p.first], p.second);
  for (auto &e : D.bedge) {
    const int lo = std::min(e.first, e.second), hi = std::max(e.first, e.second);
    last[lo] = std::max(last[lo], hi);
  }
  std::vector<int> slot(V), free_slots;
  std::vector<std::vector<int>> release(V + 1);
  int next = 0;
  for (int v = 0; v < V; ++v) {
    for (int u : release[v]) free_slots.push_back(slot[u]);
    if (free_slots.empty()) {
      slot[v] = next++;
    } else {
      auto it = std::min_element(free_slots.begin(), free_slots.end());
      slot[v] = *it;
      free_slots.erase(it);
    }
    release[last[v] + 1].push_back(v);
  }
  if (nslots) *nslots = next;
  return slot;
}

// Pack the diamond into the tables the table-driven kernels stage into
// shared memory and the specialised kernels keep in constant memory (format
// in tc_runtime.cuh; bit 30 of vext[v]: apply the pending joins before v).
// Vertex references (fan entries, antipodal and boundary-edge partners) are
// label slots (lab_slots).  Returns false if a field does not fit: a vertex
// id or slot (10 bits), a fan longer than the join list of the kernels takes
// (tc_pcap), or more than 2^16 fan entries.
bool pack_diamond_tables(const Diamond &D, std::vector<uint32_t> &tables, TableLayout &lay) {
  const int V = D.V;
  constexpr uint32_t kNone = 1023u;
  if (V > (int)kNone) return false;
  int nslots = 0;
  const std::vector<int> slot = lab_slots(D, &nslots);
  std::vector<uint32_t> vdesc(V), fan, vext(V, kNone | (kNone << 10) | (kNone << 20));
  for (int v = 0; v < V; ++v) {
    const int m = (int)D.fan[v].size();
    if (m > 127 || m + 1 > tc_pcap(D.d) || fan.size() > 65535 || D.k[v] > 255 ||
        slot[v] >= (int)kNone)
      return false;
    vdesc[v] = (uint32_t)D.k[v] | ((uint32_t)D.c[v] << 8) | ((uint32_t)m << 9) |
               ((uint32_t)slot[v] << 16);
    for (int n = 0; n < m; ++n) {
      int u = D.fan[v][n];
      fan.push_back((uint32_t)slot[u] | ((uint32_t)D.k[u] << 10) | ((uint32_t)D.c[u] << 18) |
                    ((uint32_t)D.link[v][n] << 19));
    }
  }
  for (auto &p : D.anti) vext[p.second] = (vext[p.second] & ~kNone) | (uint32_t)slot[p.first];
  const std::vector<char> flush = flush_schedule(D, 0, V, tc_pcap(D.d));
  for (int v = 0; v < V; ++v)
    if (flush[v]) vext[v] |= 1u << 30;
  if (D.d % 2) {
    for (auto &e : D.bedge) {
      const int late = std::max(e.first, e.second), early = std::min(e.first, e.second);
      uint32_t &w = vext[late];
      if (((w >> 10) & kNone) == kNone) w = (w & ~(kNone << 10)) | ((uint32_t)slot[early] << 10);
      else if (((w >> 20) & kNone) == kNone) w = (w & ~(kNone << 20)) | ((uint32_t)slot[early] << 20);
      else return false;
    }
  }
  // bit 26 of vdesc: vext[v] says something (a flush, an antipodal partner,
  // a boundary edge); interior vertices skip it
  for (int v = 0; v < V; ++v)
    if (vext[v] != (kNone | (kNone << 10) | (kNone << 20))) vdesc[v] |= 1u << 26;
  TableLayout L{};
  L.V = V;
  L.NF = (uint32_t)fan.size();
  L.off_vdesc = 0;
  L.off_fan = L.off_vdesc + V;
  L.off_vext = L.off_fan + L.NF;
  L.words = (L.off_vext + V + 3) & ~3u;
  L.nslots = (uint32_t)nslots;
  tables.assign(L.words, 0);
  std::copy(vdesc.begin(), vdesc.end(), tables.begin() + L.off_vdesc);
  std::copy(fan.begin(), fan.end(), tables.begin() + L.off_fan);
  std::copy(vext.begin(), vext.end(), tables.begin() + L.off_vext);
  lay = L;
  return true;
}
bool pack_warp_tables(const Diamond &D, std::vector<uint32_t> &tables, WarpLayout &lay) {
  const int V = D.V;
  if (V > 1022) return false;
  std::vector<uint32_t> wv(V), wedge;
  for (int v = 0; v < V; ++v) {
    const size_t f = D.fan[v].size();
    if (f > 64 || wedge.size() + f > 0xFFFF) return false;
    wv[v] = (uint32_t)D.k[v] | ((uint32_t)D.c[v] << 8) | ((uint32_t)f << 9) |
            ((uint32_t)wedge.size() << 16);
    for (size_t n = 0; n < f; ++n)
      wedge.push_back((uint32_t)D.fan[v][n] | ((uint32_t)D.link[v][n] << 15) | ((uint32_t)v << 16));
  }
  WarpLayout L{};
  L.V = V;
  L.E = (uint32_t)wedge.size();
  L.nanti = (uint32_t)D.anti.size();
  L.nbedge = (uint32_t)D.bedge.size();
  L.off_v = 0;
  L.off_e = L.off_v + V;
  L.off_anti = L.off_e + L.E;
  L.off_bedge = L.off_anti + L.nanti;
  L.words = (L.off_bedge + L.nbedge + 3) & ~3u;
  tables.assign(L.words, 0);
  std::copy(wv.begin(), wv.end(), tables.begin() + L.off_v);
  std::copy(wedge.begin(), wedge.end(), tables.begin() + L.off_e);
  for (uint32_t i = 0; i < L.nanti; ++i)
    tables[L.off_anti + i] = (uint32_t)D.anti[i].first | ((uint32_t)D.anti[i].second << 16);
  for (uint32_t i = 0; i < L.nbedge; ++i)
    tables[L.off_bedge + i] = (uint32_t)D.bedge[i].first | ((uint32_t)D.bedge[i].second << 16);
  lay = L;
  return true;
}
}  // namespace tcurve

namespace {

bool pack_tables(const Diamond &D, ts_tri *t) {
  if (!pack_diamond_tables(D, t->host_tables, t->lay)) return false;
  if (!pack_warp_tables(D, t->host_wtables, t->wlay)) return false;
  t->V = D.V;
  return true;
}

ts_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return TS_OK;
  if (e == cudaErrorMemoryAllocation) return TS_ENOMEM;
  return TS_ECUDA;
}

ts_status err_word_status(uint32_t w) {
  if (w & kErrTimeout) return TS_ETIMEOUT;
  if (w & kErrOverflow) return TS_EOVERFLOW;
  if (w & kErrInternal) return TS_EINTERNAL;
  return TS_OK;
}

void put_scheme(std::string &out, const std::vector<std::vector<int>> &kids, int node) {
  // children encodings are already in canonical (descending) order; group
  // equal consecutive siblings as k or k<X>
  std::vector<std::string> parts;
  for (int c : kids[node]) {
    std::string s;
    put_scheme(s, kids, c);
    parts.push_back(s);
  }
  std::string res;
  for (size_t a = 0; a < parts.size();) {
    size_t b = a;
    while (b < parts.size() && parts[b] == parts[a]) ++b;
    if (!res.empty()) res += " + ";
    res += std::to_string(b - a);
    if (!parts[a].empty()) res += "<" + parts[a] + ">";
    a = b;
  }
  out += res;
}

}  // namespace

extern "C" {

const char *ts_status_str(int s) {
  switch (s) {
    case TS_OK: return "TS_OK";
    case TS_EINVAL: return "TS_EINVAL: invalid argument";
    case TS_ENOTTRI: return "TS_ENOTTRI: not a unimodular triangulation of d*Delta_2";
    case TS_ENOMEM: return "TS_ENOMEM: out of memory";
    case TS_ECUDA: return "TS_ECUDA: CUDA error or no usable device";
    case TS_EOVERFLOW: return "TS_EOVERFLOW: capacity exceeded";
    case TS_ETIMEOUT: return "TS_ETIMEOUT: bounded device wait gave up";
    case TS_EINTERNAL: return "TS_EINTERNAL: invariant violated on some instance";
    case TS_EUNSUPPORTED: return "TS_EUNSUPPORTED: degree not supported by this build";
    default: return "unknown ts_status";
  }
}

int ts_max_degree(void) { return kMaxDegree; }

ts_status ts_load_triangulation(int d, const int32_t *edges_ij, int n_edges, ts_tri **out) {
  if (!out || (!edges_ij && n_edges > 0) || n_edges < 0) return TS_EINVAL;
  *out = nullptr;
  if (d < 1) return TS_EINVAL;
  if (d > kMaxDegree) return TS_EUNSUPPORTED;
  std::vector<std::array<Pt, 3>> tris;
  if (!triangles_of(d, edges_ij, n_edges, tris)) return TS_ENOTTRI;
  ts_tri *t = new (std::nothrow) ts_tri();
  if (!t) return TS_ENOMEM;
  t->d = d;
  t->np = (d + 1) * (d + 2) / 2;
  t->sw = (t->np + 63) / 64;
  t->nmax = (d % 2 == 0) ? harnack(d) : harnack(d) - 1;
  t->cw = (2 * t->nmax + 1 + 63) / 64;
  if (!build_diamond(d, tris, t->dia) || !pack_tables(t->dia, t)) {
    delete t;
    return TS_ENOTTRI;
  }
  cudaError_t e = cudaGetDevice(&t->device);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_tables, t->lay.words * sizeof(uint32_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(t->d_tables, t->host_tables.data(), t->lay.words * sizeof(uint32_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_wtables, t->wlay.words * sizeof(uint32_t));
  if (e == cudaSuccess)
    e = cudaMemcpy(t->d_wtables, t->host_wtables.data(), t->wlay.words * sizeof(uint32_t),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&t->d_err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemset(t->d_err, 0, sizeof(uint32_t));
  if (e != cudaSuccess) {
    ts_status s = cuda_status(e);
    ts_free_triangulation(t);
    return s;
  }
  *out = t;
  return TS_OK;
}

void ts_free_triangulation(ts_tri *t) {
  if (!t) return;
  jit_release(t);
  if (t->d_tables) cudaFree(t->d_tables);
  if (t->d_wtables) cudaFree(t->d_wtables);
  if (t->d_err) cudaFree(t->d_err);
  delete t;
}

int ts_degree(const ts_tri *t) { return t ? t->d : 0; }
int ts_num_points(const ts_tri *t) { return t ? t->np : 0; }
int ts_sign_words(const ts_tri *t) { return t ? t->sw : 0; }
int ts_code_words(const ts_tri *t) { return t ? t->cw : 0; }

namespace {
// Kernel choice: the specialised kernel for sweeps and large batches (AUTO),
// the table-driven kernel otherwise or when specialisation is unavailable.
bool want_specialised(ts_tri *t, uint64_t n, bool sweep) {
  if (t->kernel == TS_KERNEL_TABLE || t->kernel == TS_KERNEL_WARP || t->d > kMaxSpecialized)
    return false;
  if (t->kernel == TS_KERNEL_SPECIALIZED) return true;
  if (!sweep && n < (1u << 16)) return false;
  return jit_prepare(t) == cudaSuccess;
}
}  // namespace

ts_status ts_real_schemes(const ts_tri *tc, const uint64_t *signs, uint64_t n, uint64_t *codes,
                          void *stream) {
  if (!tc || (n && (!signs || !codes))) return TS_EINVAL;
  if (n == 0) return TS_OK;
  ts_tri *t = const_cast<ts_tri *>(tc);  // only the lazily compiled kernel cache changes
  if (t->kernel == TS_KERNEL_WARP)
    return cuda_status(launch_real_schemes_warp(t, signs, n, codes, (cudaStream_t)stream));
  if (want_specialised(t, n, false))
    return cuda_status(launch_real_schemes_jit(t, signs, n, codes, (cudaStream_t)stream));
  return cuda_status(launch_real_schemes(t, signs, n, codes, (cudaStream_t)stream));
}

ts_status ts_set_kernel(ts_tri *t, int kind) {
  if (!t || kind < TS_KERNEL_AUTO || kind > TS_KERNEL_WARP) return TS_EINVAL;
  if (kind == TS_KERNEL_SPECIALIZED && t->d > kMaxSpecialized) return TS_EUNSUPPORTED;
  t->kernel = kind;
  return TS_OK;
}

ts_status ts_set_scratch(ts_tri *t, int where) {
  if (!t || where < TS_SCRATCH_AUTO || where > TS_SCRATCH_GLOBAL) return TS_EINVAL;
  if (where != t->scratch) jit_release(t);  // the specialised kernels are rebuilt for it
  t->scratch = where;
  return TS_OK;
}

ts_status ts_set_occupancy(ts_tri *t, int blocks_per_sm) {
  if (!t || blocks_per_sm < 0 || blocks_per_sm > 16) return TS_EINVAL;
  if (blocks_per_sm != t->occupancy) jit_release(t);
  t->occupancy = blocks_per_sm;
  return TS_OK;
}

ts_status ts_prepare(ts_tri *t) {
  if (!t) return TS_EINVAL;
  if (t->d > kMaxSpecialized) return TS_EUNSUPPORTED;
  return cuda_status(jit_prepare(t));
}

ts_status ts_specialized_log(const ts_tri *t, char *buf, size_t len) {
  if (!t || !buf || !len) return TS_EINVAL;
  std::string lg = t->jit_log;
  size_t n = std::min(len - 1, lg.size());
  std::memcpy(buf, lg.data(), n);
  buf[n] = 0;
  return lg.size() + 1 > len ? TS_EOVERFLOW : TS_OK;
}

ts_status ts_specialized_source(int d, const int32_t *edges_ij, int n_edges, int compile, char *buf,
                                size_t len, size_t *needed) {
  if ((!edges_ij && n_edges > 0) || n_edges < 0 || d < 1 || (len && !buf)) return TS_EINVAL;
  if (d > kMaxSpecialized) return TS_EUNSUPPORTED;
  std::vector<std::array<Pt, 3>> tris;
  if (!triangles_of(d, edges_ij, n_edges, tris)) return TS_ENOTTRI;
  Diamond D;
  if (!build_diamond(d, tris, D)) return TS_ENOTTRI;
  bool global = false;
  int minb = 2;
  jit_config(d, TS_SCRATCH_AUTO, 0, &global, &minb);  // what runs by default
  std::string out = jit_source(D, global, minb);
  ts_status st = TS_OK;
  if (compile) {
    std::string log;
    std::string cubin = jit_compile_cubin(out, &log);
    out = log;
    if (cubin.empty()) st = TS_ECUDA;
  }
  if (needed) *needed = out.size() + 1;
  if (len) {
    size_t n = std::min(len - 1, out.size());
    std::memcpy(buf, out.data(), n);
    buf[n] = 0;
    if (out.size() + 1 > len && st == TS_OK) st = TS_EOVERFLOW;
  }
  return st;
}

ts_status ts_batch_specialized_link(int d, int ntri, const int32_t *const *edges_ij,
                                    const int *n_edges, size_t *linked_bytes, char *log, size_t len) {
  if (d < 1 || ntri < 1 || !edges_ij || !n_edges || (len && !log)) return TS_EINVAL;
  if (d > kMaxDegree) return TS_EUNSUPPORTED;
  std::vector<Diamond> dias(ntri);
  std::vector<const Diamond *> ptrs;
  for (int i = 0; i < ntri; ++i) {
    std::vector<std::array<Pt, 3>> tris;
    if (n_edges[i] < 0 || (!edges_ij[i] && n_edges[i] > 0)) return TS_EINVAL;
    if (!triangles_of(d, edges_ij[i], n_edges[i], tris) || !build_diamond(d, tris, dias[i]))
      return TS_ENOTTRI;
    ptrs.push_back(&dias[i]);
  }
  std::string lg;
  const std::string cubin = jit_jobs_link(ptrs, &lg);
  if (linked_bytes) *linked_bytes = cubin.size();
  if (len) {
    const size_t n = std::min(len - 1, lg.size());
    std::memcpy(log, lg.data(), n);
    log[n] = 0;
  }
  return cubin.empty() ? TS_ECUDA : TS_OK;
}

ts_status ts_sync(const ts_tri *t, void *stream) {
  if (!t) return TS_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e);
  uint32_t w = 0;
  e = cudaMemcpy(&w, t->d_err, sizeof(w), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && w) e = cudaMemset(t->d_err, 0, sizeof(uint32_t));
  if (e != cudaSuccess) return cuda_status(e);
  return err_word_status(w);
}

ts_status ts_real_schemes_host(const ts_tri *t, const uint64_t *signs_host, uint64_t n,
                               uint64_t *codes_host) {
  if (!t || (n && (!signs_host || !codes_host))) return TS_EINVAL;
  if (n == 0) return TS_OK;
  if (n > (SIZE_MAX / sizeof(uint64_t)) / (size_t)std::max(t->sw, t->cw)) return TS_EINVAL;
  uint64_t *ds = nullptr, *dc = nullptr;
  size_t bs = n * t->sw * sizeof(uint64_t), bc = n * t->cw * sizeof(uint64_t);
  cudaError_t e = cudaMalloc(&ds, bs);
  if (e == cudaSuccess) e = cudaMalloc(&dc, bc);
  if (e == cudaSuccess) e = cudaMemcpy(ds, signs_host, bs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    ts_status ls = ts_real_schemes(t, ds, n, dc, nullptr);
    if (ls != TS_OK) e = cudaErrorLaunchFailure;
  }
  if (e == cudaSuccess) e = cudaMemcpy(codes_host, dc, bc, cudaMemcpyDeviceToHost);
  if (ds) cudaFree(ds);
  if (dc) cudaFree(dc);
  if (e != cudaSuccess) return cuda_status(e);
  return ts_sync(t, 0);
}

ts_status ts_splitmix_masks(int d, uint64_t base, uint64_t n, uint64_t *out, void *stream) {
  if (d < 1 || (n && !out)) return TS_EINVAL;
  if (d > kMaxDegree) return TS_EUNSUPPORTED;
  if (n == 0) return TS_OK;
  return cuda_status(launch_splitmix_masks(d, base, n, out, (cudaStream_t)stream));
}

ts_status ts_hist_create(uint64_t capacity, int code_words, ts_hist **out) {
  if (!out || code_words < 1 || code_words > 4 || capacity == 0 || capacity > (1ull << 30))
    return TS_EINVAL;
  *out = nullptr;
  ts_hist *h = new (std::nothrow) ts_hist();
  if (!h) return TS_ENOMEM;
  h->cw = code_words;
  uint64_t s = 16;
  while (s < 2 * capacity) s <<= 1;
  h->slots = s;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_keys, s * code_words * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_counts, s * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_failed, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_work, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_ckeys, s * code_words * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_ccnt, s * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_cn, sizeof(unsigned long long));
  if (e == cudaSuccess) e = launch_hist_clear(h, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    ts_status st = cuda_status(e);
    ts_hist_free(h);
    return st;
  }
  *out = h;
  return TS_OK;
}

void ts_hist_free(ts_hist *h) {
  if (!h) return;
  if (h->d_keys) cudaFree(h->d_keys);
  if (h->d_counts) cudaFree(h->d_counts);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_failed) cudaFree(h->d_failed);
  if (h->d_work) cudaFree(h->d_work);
  if (h->d_ckeys) cudaFree(h->d_ckeys);
  if (h->d_ccnt) cudaFree(h->d_ccnt);
  if (h->d_cn) cudaFree(h->d_cn);
  delete h;
}

ts_status ts_hist_clear(ts_hist *h, void *stream) {
  if (!h) return TS_EINVAL;
  return cuda_status(launch_hist_clear(h, (cudaStream_t)stream));
}

ts_status ts_enumerate(const ts_tri *t, uint64_t lo, uint64_t hi, uint32_t flags, ts_hist *h,
                       void *stream) {
  const uint32_t kinds =
      flags & (TS_ENUM_FLIP | TS_ENUM_REDUCED | TS_ENUM_SPLITMIX | TS_ENUM_ORBITS);
  if (!t || !h || hi < lo || (flags & ~kinds) || (kinds & (kinds - 1))) return TS_EINVAL;
  if (h->cw != t->cw) return TS_EINVAL;
  int free_bits = t->np - ((flags & TS_ENUM_FLIP) ? 1 : 0) -
                  ((flags & (TS_ENUM_REDUCED | TS_ENUM_ORBITS)) ? 3 : 0);
  if (!(flags & TS_ENUM_SPLITMIX) && free_bits < 64 && hi > (1ull << free_bits)) return TS_EINVAL;
  if (flags & TS_ENUM_ORBITS) {  // the kernels read the pivots from bits 8-23 of the flags
    int p1 = 0, p2 = 0;
    if (t->d > 9) return TS_EUNSUPPORTED;
    if (!tc_orbit_pivots(t->d, &p1, &p2)) return TS_EINVAL;
    flags |= ((uint32_t)p1 << 8) | ((uint32_t)p2 << 16);
  }
  if (lo == hi) return TS_OK;
  ts_tri *tm = const_cast<ts_tri *>(t);
  if (tm->kernel == TS_KERNEL_WARP)
    return cuda_status(launch_enumerate_warp(tm, lo, hi, flags, h, (cudaStream_t)stream));
  if (want_specialised(tm, hi - lo, true))
    return cuda_status(launch_enumerate_jit(tm, lo, hi, flags, h, (cudaStream_t)stream));
  return cuda_status(launch_enumerate(t, lo, hi, flags, h, (cudaStream_t)stream));
}

ts_status ts_hist_read(ts_hist *h, uint64_t *codes, uint64_t *counts, uint64_t cap,
                       uint64_t *n_out, uint64_t *n_failed, void *stream) {
  if (!h || !n_out || (cap && (!codes || !counts))) return TS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // pack the occupied slots on the device; only those cross to the host
  cudaError_t e = launch_hist_compact(h, st);
  unsigned long long n = 0, failed = 0;
  uint32_t err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&n, h->d_cn, sizeof(n), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, h->d_err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&failed, h->d_failed, sizeof(failed), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  const int cw = h->cw;
  std::vector<uint64_t> keys(n * cw);
  std::vector<unsigned long long> cnt(n);
  if (n) {
    e = cudaMemcpyAsync(keys.data(), h->d_ckeys, keys.size() * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cnt.data(), h->d_ccnt, n * sizeof(unsigned long long),
                          cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  std::vector<uint64_t> idx(n);
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](uint64_t a, uint64_t b) {
    for (int w = cw - 1; w >= 0; --w)
      if (keys[a * cw + w] != keys[b * cw + w]) return keys[a * cw + w] < keys[b * cw + w];
    return false;
  });
  *n_out = n;
  if (n_failed) *n_failed = failed;
  for (uint64_t r = 0; r < n && r < cap; ++r) {
    for (int w = 0; w < cw; ++w) codes[r * cw + w] = keys[idx[r] * cw + w];
    counts[r] = cnt[idx[r]];
  }
  if (n > cap) return TS_EOVERFLOW;
  return err_word_status(err);
}

ts_status ts_selftest_wait(uint64_t iters, void *stream) {
  if (iters == 0 || iters > (1ull << 20)) return TS_EINVAL;
  uint32_t *d_err = nullptr, err = 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMalloc(&d_err, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(uint32_t), st);
  if (e == cudaSuccess) e = launch_selftest_wait(iters, d_err, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&err, d_err, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (d_err) cudaFree(d_err);
  if (e != cudaSuccess) return cuda_status(e);
  return err_word_status(err);
}

ts_status ts_scheme_string(int d, const uint64_t *code, int code_words, char *buf, size_t len) {
  if (!code || !buf || len == 0 || code_words < 1 || d < 1) return TS_EINVAL;
  int top = -1;
  for (int b = 64 * code_words - 1; b >= 0; --b)
    if ((code[b >> 6] >> (b & 63)) & 1) { top = b; break; }
  if (top < 0 || (top & 1)) return TS_EINVAL;  // code 0, or odd bit count
  // parse the Dyck word below the sentinel into a tree (node 0 = root)
  std::vector<std::vector<int>> kids(1);
  std::vector<int> stack{0};
  for (int b = top - 1; b >= 0; --b) {
    int bit = (int)((code[b >> 6] >> (b & 63)) & 1);
    if (bit) {
      int n = (int)kids.size();
      kids.push_back({});
      kids[stack.back()].push_back(n);
      stack.push_back(n);
    } else {
      if (stack.size() < 2) return TS_EINVAL;
      stack.pop_back();
    }
  }
  if (stack.size() != 1) return TS_EINVAL;
  std::string body;
  put_scheme(body, kids, 0);
  std::string s = "<";
  if (d % 2) s += body.empty() ? "J" : "J + " + body;
  else s += body.empty() ? "0" : body;
  s += ">";
  if (s.size() + 1 > len) return TS_EOVERFLOW;
  std::memcpy(buf, s.c_str(), s.size() + 1);
  return TS_OK;
}

}  // extern "C"
