// api.cu — the C ABI (include/gpm.h): handles, errors, pattern analysis,
// plan construction (Section 4.2 pattern analyzer, Section 7.2 memory
// management) and the count / list entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "enum_common.cuh"
#include "gpm_internal.cuh"

namespace gpm {

cudaError_t launch_clique(int k, bool list, const EnumArgs& a, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s);
cudaError_t occupancy_clique(int k, bool list, int threads, size_t smem, int* blocks, int* regs);
cudaError_t launch_small(int family, bool induced, bool list, bool co, const EnumArgs& a,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t s);
cudaError_t occupancy_small(int family, bool induced, bool list, bool co, int threads, size_t smem,
                            int* blocks, int* regs);
cudaError_t widen_offsets(const int32_t* in, uint64_t count, int64_t* out, cudaStream_t s);
cudaError_t relabel_by_degree(gpm_graph* G, cudaStream_t s);
cudaError_t launch_generic(bool list, const EnumArgs& a, dim3 grid, dim3 block, size_t smem,
                           cudaStream_t s);
cudaError_t occupancy_generic(bool list, int threads, size_t smem, int* blocks, int* regs);
bool analyze_pattern(uint32_t k, const std::vector<std::pair<int, int>>& edges, int induced,
                     double n, double avg_degree, GenTable* T, std::string* why);
std::string describe_gen(const GenTable& T);
cudaError_t unrename_ids(const gpm_graph* G, uint32_t* ids, uint64_t count, cudaStream_t s);
uint32_t lgs_warp_max_degree();
uint32_t lgs_block_max_degree();
cudaError_t lgs_launch_warp(int k, const LgsArgs& a, unsigned blocks, cudaStream_t s);
cudaError_t lgs_launch_block(int k, int nw, bool arc, const LgsArgs& a, unsigned blocks_per_sm,
                             unsigned sms, cudaStream_t s);
int lgs_block_occupancy(int k, int nw);
uint32_t wedge_threads();
cudaError_t degrees32(const DevCsr& g, uint32_t* deg, int sms, cudaStream_t s);
cudaError_t launch_cycle4_wedge(const DevCsr& g, const uint32_t* deg, uint32_t* cnt, unsigned blocks,
                                Control* ctl, unsigned long long* stats, cudaStream_t s);

namespace {
thread_local std::string t_err;

gpm_status fail(gpm_status st, const std::string& msg) {
  t_err = msg;
  return st;
}

gpm_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(GPM_E_OOM, std::string(where) + ": out of device memory");
  return fail(GPM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------- pattern analysis

struct NamedPattern {
  const char* name;
  int family;
  uint32_t k;
  std::vector<std::pair<int, int>> edges;  // matching order
};

std::vector<NamedPattern> named_patterns() {
  std::vector<NamedPattern> v = {
      {"wedge", kWedge, 3, {{0, 1}, {0, 2}}},
      {"3-star", kStar3, 4, {{0, 1}, {0, 2}, {0, 3}}},
      {"4-path", kPath4, 4, {{0, 1}, {0, 2}, {1, 3}}},
      {"4-cycle", kCycle4, 4, {{0, 1}, {1, 2}, {2, 3}, {3, 0}}},
      {"tailed-triangle", kTailedTriangle, 4, {{0, 1}, {0, 2}, {1, 2}, {0, 3}}},
      {"diamond", kDiamond, 4, {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}}},
  };
  for (uint32_t k = 3; k <= 8; k++) {
    NamedPattern p{nullptr, kClique, k, {}};
    for (uint32_t i = 0; i < k; i++)
      for (uint32_t j = i + 1; j < k; j++) p.edges.push_back({(int)i, (int)j});
    v.push_back(p);
  }
  return v;
}

uint64_t adj_bits(uint32_t k, const std::vector<std::pair<int, int>>& e) {
  uint64_t m = 0;
  for (auto& pr : e) {
    m |= 1ull << (pr.first * 8 + pr.second);
    m |= 1ull << (pr.second * 8 + pr.first);
  }
  (void)k;
  return m;
}

bool isomorphic(uint32_t k, uint64_t a, uint64_t b) {
  int perm[8];
  for (uint32_t i = 0; i < k; i++) perm[i] = (int)i;
  do {
    bool ok = true;
    for (uint32_t i = 0; i < k && ok; i++)
      for (uint32_t j = i + 1; j < k; j++)
        if (((a >> (i * 8 + j)) & 1) != ((b >> (perm[i] * 8 + perm[j])) & 1)) { ok = false; break; }
    if (ok) return true;
  } while (std::next_permutation(perm, perm + k));
  return false;
}

// Identify the plan family of a user pattern (k, edge list) up to isomorphism.
bool identify(const gpm_pattern* p, int* family, uint32_t* k) {
  if (p->k < 2 || p->k > 8 || p->n_edges > 28) return false;
  std::vector<std::pair<int, int>> e;
  for (uint32_t i = 0; i < p->n_edges; i++) {
    int a = p->edges[i][0], b = p->edges[i][1];
    if (a >= (int)p->k || b >= (int)p->k || a == b) return false;
    e.push_back({std::min(a, b), std::max(a, b)});
  }
  std::sort(e.begin(), e.end());
  e.erase(std::unique(e.begin(), e.end()), e.end());
  const uint64_t bits = adj_bits(p->k, e);
  for (auto& np : named_patterns()) {
    if (np.k != p->k || np.edges.size() != e.size()) continue;
    if (isomorphic(p->k, adj_bits(np.k, np.edges), bits)) {
      *family = np.family;
      *k = np.k;
      return true;
    }
  }
  return false;
}

// Buffered DFS levels X per warp (Section 7.2 (3): X <= k - 3 for counting;
// listing and vertex-induced plans buffer their difference sets too).
uint32_t plan_levels(int family, uint32_t k, bool induced, bool list, bool co) {
  switch (family) {
    case kClique: return list ? k - 2 : (k > 3 ? k - 3 : 0);
    case kDiamond: return induced ? (list ? 2 : 1) : ((co && !list) ? 0 : 1);
    case kCycle4: return induced ? (list ? 3 : 2) : (list ? 1 : 0);
    case kTailedTriangle: return induced ? (list ? 3 : 2) : (list ? 1 : 0);
    case kStar3: return induced ? (list ? 2 : 1) : 0;
    case kPath4: return induced ? (list ? 3 : 2) : 0;
    case kWedge: return (induced && list) ? 1 : 0;
    case kGeneric: return k - 1;  // positions 2..k-1 and one scratch level
    default: return 0;
  }
}

TaskKind task_kind_of(int family) {
  switch (family) {
    case kClique: return kTasksDag;
    case kDiamond: case kCycle4: case kPath4: return kTasksLower;
    default: return kTasksAll;
  }
}

cudaError_t occupancy(const gpm_plan_t* p, int threads, size_t smem, int* blocks, int* regs) {
  const bool list = p->mode == GPM_LIST;
  if (p->family == kClique) return occupancy_clique((int)p->k, list, threads, smem, blocks, regs);
  if (p->family == kGeneric) return occupancy_generic(list, threads, smem, blocks, regs);
  return occupancy_small(p->family, p->induced, list, p->count_only, threads, smem, blocks, regs);
}

}  // namespace

void set_error(const std::string& msg) { t_err = msg; }
const std::string& get_error() { return t_err; }

size_t enum_smem_bytes(const gpm_plan_t* p) {
  return (size_t)p->cfg.warps_per_block * p->cfg.levels * p->cfg.smem_cap * sizeof(uint32_t);
}

cudaError_t launch_enum(gpm_plan_t* p, uint64_t lo, uint64_t hi, uint32_t* list_out,
                        uint64_t list_cap, cudaStream_t s) {
  EnumArgs a;
  a.g = p->csr;
  a.src = p->tasks.src;
  a.dst = p->tasks.dst;
  a.lo = lo;
  a.hi = hi;
  a.ctl = p->ctl_d;
  a.list_out = list_out;
  a.list_cap = list_cap;
  a.gstack = p->gstack_d;
  a.gcap = p->cfg.gstack_cap;
  a.scap = p->cfg.smem_cap;
  a.levels = p->cfg.levels;
  a.chunk = p->cfg.chunk;
  a.ratio = p->cfg.ratio;
  a.stats = p->cfg.stats ? p->ctl_d->stats : nullptr;
  a.idx = nullptr;
  a.arc_lo = 0;
  a.arc_hi = 0;
  a.idx_count = nullptr;
  a.gen = p->gen_d;
  a.vertex_tasks = p->vertex_tasks ? 1u : 0u;
  a.vkind = (uint32_t)p->task_kind;
  const dim3 grid(p->cfg.blocks), block(p->cfg.warps_per_block * 32);
  const size_t smem = enum_smem_bytes(p);
  const bool list = p->mode == GPM_LIST;
  if (p->family == kClique) return launch_clique((int)p->k, list, a, grid, block, smem, s);
  if (p->family == kGeneric) return launch_generic(list, a, grid, block, smem, s);
  return launch_small(p->family, p->induced, list, p->count_only, a, grid, block, smem, s);
}

// Local graph search: the three vertex-rooted size classes, then the arcs of
// roots too large for one shared-memory local graph, each rooted at its own
// arc-level local graph (members N+(u) ∩ N+(v)); arcs whose arc-level local
// graph is still too large go to the sorted-set kernel.  Each launch restarts
// the queue head; counts accumulate in ctl->result.
cudaError_t launch_lgs(gpm_plan_t* p, uint64_t lo, uint64_t hi, cudaStream_t s) {
  gpm_graph* G = p->graph;
  LgsArgs la{};
  la.dag = p->csr;
  la.uoff = G->g.off;
  la.lo = lo;
  la.hi = hi;
  la.next = &p->ctl_d->next;
  la.result = &p->ctl_d->result;
  la.stats = p->cfg.stats ? p->ctl_d->stats : nullptr;
  la.src = p->tasks.src;
  la.overflow = p->overflow_d;
  la.overflow_count = &p->ctl_d->overflow;
  cudaError_t e = cudaSuccess;
  static const int kClassWords[4] = {0, 8, 16, 32};
  for (int c = 0; c < 4 && e == cudaSuccess; c++) {
    if (!p->lgs_count[c]) continue;
    la.verts = p->lgs_verts[c];
    la.nverts = p->lgs_count[c];
    e = cudaMemsetAsync(&p->ctl_d->next, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) break;
    if (c == 0) e = lgs_launch_warp((int)p->k, la, p->lgs_warp_blocks, s);
    else e = lgs_launch_block((int)p->k, kClassWords[c], false, la, p->lgs_bps[c],
                              (unsigned)G->num_sms, s);
  }
  if (e == cudaSuccess && p->heavy_count) {
    la.verts = nullptr;
    la.nverts = 0;
    la.idx = p->heavy_idx;
    la.nidx = p->heavy_count;
    e = cudaMemsetAsync(&p->ctl_d->next, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess)
      e = lgs_launch_block((int)p->k, 32, true, la, p->lgs_bps[3], (unsigned)G->num_sms, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&p->ctl_d->next, 0, sizeof(unsigned long long), s);
    EnumArgs a{};
    a.g = p->csr;
    a.src = p->tasks.src;
    a.dst = p->tasks.dst;
    a.lo = 0;
    a.hi = p->heavy_count;
    a.ctl = p->ctl_d;
    a.gstack = p->gstack_d;
    a.gcap = p->cfg.gstack_cap;
    a.scap = p->cfg.smem_cap;
    a.levels = p->cfg.levels;
    a.chunk = 1;
    a.ratio = p->cfg.ratio;
    a.stats = la.stats;
    a.idx = p->overflow_d;
    a.arc_lo = lo;
    a.arc_hi = hi;
    a.idx_count = &p->ctl_d->overflow;
    if (e == cudaSuccess)
      e = launch_clique((int)p->k, false, a, dim3(p->cfg.blocks), dim3(p->cfg.warps_per_block * 32),
                        enum_smem_bytes(p), s);
  }
  return e;
}

}  // namespace gpm

using namespace gpm;

// ====================================================================== ABI

extern "C" {

const char* gpm_last_error(void) { return t_err.c_str(); }
const char* gpm_version(void) { return "gpm-gb300 0.1 (sm_103a)"; }

gpm_status gpm_pattern_named(const char* name, gpm_pattern* out) {
  if (!name || !out) return fail(GPM_E_INVALID_ARG, "gpm_pattern_named: NULL argument");
  std::string n(name);
  if (n == "triangle") n = "3-clique";
  for (auto& np : named_patterns()) {
    std::string nm = np.name ? np.name : (std::to_string(np.k) + "-clique");
    if (nm != n) continue;
    gpm_pattern p;
    memset(&p, 0, sizeof(p));
    p.k = np.k;
    p.n_edges = (uint32_t)np.edges.size();
    for (size_t i = 0; i < np.edges.size(); i++) {
      p.edges[i][0] = (uint8_t)np.edges[i].first;
      p.edges[i][1] = (uint8_t)np.edges[i].second;
    }
    *out = p;
    return GPM_OK;
  }
  return fail(GPM_E_UNSUPPORTED_PATTERN, "gpm_pattern_named: unknown pattern '" + n + "'");
}

gpm_status gpm_load_csr(const void* offsets, int offsets_is_64, const uint32_t* nbrs, uint32_t n,
                        uint64_t nnz, uint32_t flags, void* stream, gpm_graph** out) {
  if (!out) return fail(GPM_E_INVALID_ARG, "gpm_load_csr: out is NULL");
  if (!offsets || (!nbrs && nnz)) return fail(GPM_E_INVALID_ARG, "gpm_load_csr: NULL array");
  if (n == 0xffffffffu) return fail(GPM_E_INVALID_ARG, "gpm_load_csr: n must be < 2^32 - 1");
  const bool dev = flags & GPM_DEVICE_PTRS, borrow = flags & GPM_BORROW;
  if (borrow && (!dev || !offsets_is_64))
    return fail(GPM_E_INVALID_ARG, "gpm_load_csr: GPM_BORROW needs device pointers and int64 offsets");
  if (!offsets_is_64 && nnz > 0x7fffffffull)
    return fail(GPM_E_INVALID_ARG, "gpm_load_csr: nnz exceeds int32 offsets");
  cudaStream_t s = (cudaStream_t)stream;
  gpm_graph* G = new gpm_graph();
  cudaError_t e = cudaGetDevice(&G->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&G->num_sms, cudaDevAttrMultiProcessorCount, G->device);
  if (e != cudaSuccess) { delete G; return cuda_fail(e, "gpm_load_csr"); }
  G->g.n = n;
  G->g.nnz = nnz;
  if (borrow) {
    G->borrowed = true;
    G->off_d = (int64_t*)offsets;
    G->nbr_d = (uint32_t*)nbrs;
  } else {
    e = cudaMalloc((void**)&G->off_d, ((size_t)n + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&G->nbr_d, (nnz + 1) * sizeof(uint32_t));
    if (e != cudaSuccess) { gpm_graph_free(G); return cuda_fail(e, "gpm_load_csr"); }
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (nnz) e = cudaMemcpyAsync(G->nbr_d, nbrs, nnz * sizeof(uint32_t), kind, s);
    if (e == cudaSuccess) {
      if (offsets_is_64) {
        e = cudaMemcpyAsync(G->off_d, offsets, ((size_t)n + 1) * sizeof(int64_t), kind, s);
      } else if (dev) {
        e = widen_offsets((const int32_t*)offsets, (uint64_t)n + 1, G->off_d, s);
      } else {
        std::vector<int64_t> w((size_t)n + 1);
        const int32_t* o32 = (const int32_t*)offsets;
        for (size_t i = 0; i <= n; i++) w[i] = o32[i];
        e = cudaMemcpyAsync(G->off_d, w.data(), w.size() * sizeof(int64_t), kind, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // w goes out of scope
      }
    }
    if (e != cudaSuccess) { gpm_graph_free(G); return cuda_fail(e, "gpm_load_csr copy"); }
  }
  G->g.off = G->off_d;
  G->g.nbr = G->nbr_d;
  unsigned bad = 0;
  uint32_t maxdeg = 0;
  e = validate_csr(G->g, !(flags & GPM_SKIP_VALIDATE), s, &bad, &maxdeg);
  if (e != cudaSuccess) { gpm_graph_free(G); return cuda_fail(e, "gpm_load_csr validate"); }
  if (bad & kBadOffsets) { gpm_graph_free(G); return fail(GPM_E_RANGE, "gpm_load_csr: offsets not monotone / offsets[n] != nnz"); }
  if (bad & kBadRange) { gpm_graph_free(G); return fail(GPM_E_RANGE, "gpm_load_csr: neighbour ID >= n"); }
  if (!(flags & GPM_SKIP_VALIDATE)) {
    gpm_status st = GPM_OK;
    const char* msg = nullptr;
    if (bad & kBadRange) { st = GPM_E_RANGE; msg = "neighbour ID >= n"; }
    else if (bad & kBadSelfLoop) { st = GPM_E_SELF_LOOP; msg = "self-loop"; }
    else if (bad & kBadDuplicate) { st = GPM_E_DUPLICATE; msg = "duplicate neighbour"; }
    else if (bad & kBadUnsorted) { st = GPM_E_UNSORTED; msg = "neighbour list not ascending"; }
    else if (bad & kBadAsymmetric) { st = GPM_E_ASYMMETRIC; msg = "edge present in one direction only"; }
    if (st != GPM_OK) { gpm_graph_free(G); return fail(st, std::string("gpm_load_csr: ") + msg); }
  }
  G->max_degree = maxdeg;
  if (flags & GPM_RELABEL) {
    e = relabel_by_degree(G, s);
    if (e != cudaSuccess) { gpm_graph_free(G); return cuda_fail(e, "gpm_load_csr renaming"); }
  }
  *out = G;
  return GPM_OK;
}

gpm_status gpm_graph_info(const gpm_graph* g, uint32_t* n, uint64_t* n_edges, uint32_t* max_degree,
                          uint32_t* max_out_degree) {
  if (!g) return fail(GPM_E_INVALID_ARG, "gpm_graph_info: NULL graph");
  if (n) *n = g->g.n;
  if (n_edges) *n_edges = g->g.nnz / 2;
  if (max_degree) *max_degree = g->max_degree;
  if (max_out_degree) *max_out_degree = g->max_out_degree;
  return GPM_OK;
}

gpm_status gpm_graph_export(const gpm_graph* g, int64_t* offsets, uint32_t* nbrs, uint32_t* perm,
                            void* stream) {
  if (!g || !offsets || (!nbrs && g->g.nnz))
    return fail(GPM_E_INVALID_ARG, "gpm_graph_export: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const uint32_t n = g->g.n;
  cudaError_t e = cudaMemcpyAsync(offsets, g->g.off, ((size_t)n + 1) * sizeof(int64_t),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && g->g.nnz)
    e = cudaMemcpyAsync(nbrs, g->g.nbr, g->g.nnz * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && perm && n && g->perm_d)
    e = cudaMemcpyAsync(perm, g->perm_d, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "gpm_graph_export");
  if (perm && !g->perm_d)
    for (uint32_t v = 0; v < n; v++) perm[v] = v;
  return GPM_OK;
}

void gpm_graph_free(gpm_graph* g) {
  if (!g) return;
  if (!g->borrowed) {
    cudaFree(g->off_d);
    cudaFree(g->nbr_d);
  }
  cudaFree(g->doff_d);
  cudaFree(g->dnbr_d);
  cudaFree(g->dsrc_d);
  cudaFree(g->row_d);
  cudaFree(g->lsrc_d);
  cudaFree(g->ldst_d);
  cudaFree(g->deg32_d);
  cudaFree(g->perm_d);
  delete g;
}

gpm_status gpm_plan(gpm_graph* G, const gpm_pattern* pattern, int induced, int mode,
                    const gpm_plan_opts* opts, void* stream, gpm_plan_t** out) {
  if (!G || !pattern || !out) return fail(GPM_E_INVALID_ARG, "gpm_plan: NULL argument");
  if (mode != GPM_COUNT && mode != GPM_LIST) return fail(GPM_E_INVALID_ARG, "gpm_plan: bad mode");
  cudaStream_t s = (cudaStream_t)stream;
  gpm_plan_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  int family = 0;
  uint32_t k = 0;
  GenTable gt{};
  if (!identify(pattern, &family, &k) || o.generic_plan) {
    // any other connected pattern: the analyzer's search plan for the
    // generic interpreter
    if (pattern->k < 3 || pattern->k > (uint32_t)kGenMaxK || pattern->n_edges > 28)
      return fail(GPM_E_UNSUPPORTED_PATTERN, "gpm_plan: patterns have 3 to 8 vertices");
    std::vector<std::pair<int, int>> edges;
    for (uint32_t i = 0; i < pattern->n_edges; i++) {
      const int a = pattern->edges[i][0], b = pattern->edges[i][1];
      edges.push_back({std::min(a, b), std::max(a, b)});
    }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    std::string why;
    const double n = G->g.n, d = G->g.n ? (double)G->g.nnz / G->g.n : 0.0;
    if (!analyze_pattern(pattern->k, edges, induced ? 1 : 0, n, d, &gt, &why))
      return fail(GPM_E_UNSUPPORTED_PATTERN, "gpm_plan: " + why);
    family = kGeneric;
    k = pattern->k;
  }
  gpm_plan_t* p = new gpm_plan_t();
  p->graph = G;
  p->family = family;
  p->k = k;
  p->induced = (family == kClique) ? 0 : (induced ? 1 : 0);
  p->mode = mode;
  p->count_only = o.no_count_only ? 0 : 1;
  p->task_kind = family == kGeneric ? (gt.root_lower ? kTasksLower : kTasksAll) : task_kind_of(family);
  if (family == kGeneric) {
    p->gen = gt;
    cudaError_t eg = cudaMalloc((void**)&p->gen_d, sizeof(GenTable));
    if (eg == cudaSuccess) eg = cudaMemcpy(p->gen_d, &gt, sizeof(GenTable), cudaMemcpyHostToDevice);
    if (eg != cudaSuccess) { gpm_plan_free(p); return cuda_fail(eg, "gpm_plan search plan"); }
  }
  cudaError_t e = cudaSuccess;
  uint32_t bound = G->max_degree;  // per-level buffer bound
  // vertex parallelism: the root tasks of a vertex are walked from its row,
  // so no task list is built (local graph search is vertex-rooted already
  // and keeps arc ranges, so it is not combined with it)
  p->vertex_tasks = o.vertex_parallel != 0;
  switch (p->task_kind) {
    case kTasksDag:
      e = build_dag(G, s);
      p->csr = DevCsr{G->doff_d, G->dnbr_d, G->g.n, G->dag_arcs};
      p->tasks = DevTasks{G->dsrc_d, G->dnbr_d, G->dag_arcs};
      bound = G->max_out_degree;
      break;
    case kTasksLower:
      if (!p->vertex_tasks) e = build_lower(G, s);
      p->csr = G->g;
      p->tasks = DevTasks{G->lsrc_d, G->ldst_d, G->lower_count};
      break;
    case kTasksAll:
      if (!p->vertex_tasks) e = build_rows(G, s);
      p->csr = G->g;
      p->tasks = DevTasks{G->row_d, G->nbr_d, G->g.nnz};
      break;
  }
  if (p->vertex_tasks) p->tasks = DevTasks{nullptr, nullptr, G->g.n};
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "gpm_plan preprocessing"); }

  LaunchCfg& c = p->cfg;
  c.levels = plan_levels(family, k, p->induced, mode == GPM_LIST, p->count_only);
  c.warps_per_block = o.warps_per_block ? std::min(o.warps_per_block, 8u) : 8u;
  c.ratio = o.bsearch_ratio ? o.bsearch_ratio : 8u;
  c.stats = o.collect_stats ? 1u : 0u;
  // shared-memory slab per warp and level: the whole bound when it is small,
  // else 512 entries (larger tasks spill to the per-warp HBM slice)
  c.smem_cap = c.levels ? std::min<uint32_t>(std::max<uint32_t>(bound, 1u), 512u) : 0u;
  c.gstack_cap = (c.levels && bound > c.smem_cap) ? bound : 0u;
  if (family == kGeneric && c.gstack_cap) c.smem_cap = 0;  // all its levels live in one place
  int occ = 0, regs = 0;
  e = occupancy(p, c.warps_per_block * 32, enum_smem_bytes(p), &occ, &regs);
  if (e != cudaSuccess) { delete p; return cuda_fail(e, "gpm_plan occupancy"); }
  if (occ < 1) occ = 1;
  if (o.blocks_per_sm) occ = (int)std::min<uint32_t>(o.blocks_per_sm, (uint32_t)occ);
  uint64_t blocks = (uint64_t)G->num_sms * occ;
  // never more warps than tasks (Section 7.2 (3): min(Y / (X Δ), |Ω|))
  const uint64_t ntask = std::max<uint64_t>(p->tasks.count, 1);
  blocks = std::min<uint64_t>(blocks, (ntask + c.warps_per_block - 1) / c.warps_per_block);
  // adaptive buffering: the HBM slices must fit in free memory
  if (c.gstack_cap) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const uint64_t per_warp = (uint64_t)c.levels * c.gstack_cap * sizeof(uint32_t);
    const uint64_t budget = free_b / 2;
    const uint64_t max_warps = std::max<uint64_t>(1, budget / per_warp);
    blocks = std::min<uint64_t>(blocks, std::max<uint64_t>(1, max_warps / c.warps_per_block));
  }
  c.blocks = (uint32_t)std::max<uint64_t>(blocks, 1);
  const uint64_t total_warps = (uint64_t)c.blocks * c.warps_per_block;
  c.chunk = o.chunk ? o.chunk
                    : (uint32_t)std::min<uint64_t>(256, std::max<uint64_t>(1, ntask / (total_warps * 64)));
  if (c.gstack_cap) {
    p->gstack_bytes = total_warps * c.levels * (uint64_t)c.gstack_cap * sizeof(uint32_t);
    e = cudaMalloc((void**)&p->gstack_d, p->gstack_bytes);
    if (e != cudaSuccess) { delete p; return cuda_fail(e, "gpm_plan DFS buffers"); }
  }
  if (family == kClique && mode == GPM_COUNT && k >= 4 && !o.no_lgs && !p->vertex_tasks) {
    p->lgs = true;
    const uint32_t bounds[4] = {lgs_warp_max_degree(), 256, 512, lgs_block_max_degree()};
    e = build_lgs_classes(G, k - 1, bounds, 4, p->lgs_verts, p->lgs_count, &p->heavy_idx,
                          &p->heavy_count, s);
    if (e != cudaSuccess) { gpm_plan_free(p); return cuda_fail(e, "gpm_plan local graph classes"); }
    if (p->heavy_count) {
      e = cudaMalloc((void**)&p->overflow_d, p->heavy_count * sizeof(uint64_t));
      if (e != cudaSuccess) { gpm_plan_free(p); return cuda_fail(e, "gpm_plan overflow list"); }
    }
    p->lgs_warp_blocks = (unsigned)std::min<uint64_t>(
        (uint64_t)G->num_sms * 8, std::max<uint64_t>(1, (p->lgs_count[0] + 7) / 8));
    p->lgs_bps[1] = (unsigned)lgs_block_occupancy((int)k, 8);
    p->lgs_bps[2] = (unsigned)lgs_block_occupancy((int)k, 16);
    p->lgs_bps[3] = (unsigned)lgs_block_occupancy((int)k, 32);
  }
  if (family == kCycle4 && mode == GPM_COUNT && !p->induced && p->count_only && G->g.n) {
    if (!G->deg32_d) {
      e = cudaMalloc((void**)&G->deg32_d, (size_t)G->g.n * sizeof(uint32_t));
      if (e == cudaSuccess) e = degrees32(G->g, G->deg32_d, G->num_sms, s);
      if (e != cudaSuccess) { cudaFree(G->deg32_d); G->deg32_d = nullptr; gpm_plan_free(p); return cuda_fail(e, "gpm_plan degrees"); }
    }
    // one dense counter array (n uint32) per resident CTA, within half of free memory
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const uint64_t per = (uint64_t)G->g.n * sizeof(uint32_t);
    uint64_t blocks_w = (uint64_t)G->num_sms * 2;
    blocks_w = std::min<uint64_t>(blocks_w, std::max<uint64_t>(1, (free_b / 2) / per));
    blocks_w = std::min<uint64_t>(blocks_w, std::max<uint64_t>(1, G->g.n));
    e = cudaMalloc((void**)&p->wedge_cnt, blocks_w * per);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->wedge_cnt, 0, blocks_w * per, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { gpm_plan_free(p); return cuda_fail(e, "gpm_plan wedge counters"); }
    p->wedge = true;
    p->wedge_blocks = (unsigned)blocks_w;
  }
  e = cudaMalloc((void**)&p->ctl_d, sizeof(Control));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&p->host_pinned, sizeof(Control));
  if (e != cudaSuccess) { gpm_plan_free(p); return cuda_fail(e, "gpm_plan control block"); }
  *out = p;
  return GPM_OK;
}

gpm_status gpm_plan_info(const gpm_plan_t* p, uint64_t* n_tasks, uint32_t* k) {
  if (!p) return fail(GPM_E_INVALID_ARG, "gpm_plan_info: NULL plan");
  if (n_tasks) *n_tasks = p->tasks.count;
  if (k) *k = p->k;
  return GPM_OK;
}

gpm_status gpm_pattern_describe(const gpm_pattern* pattern, int induced, uint32_t n, uint64_t nnz,
                                int generic, char* buf, size_t len) {
  if (!pattern || !buf || len == 0) return fail(GPM_E_INVALID_ARG, "gpm_pattern_describe: bad argument");
  int family = 0;
  uint32_t k = 0;
  std::string d;
  if (identify(pattern, &family, &k) && !generic) {
    static const char* kNames[] = {"", "k-clique", "diamond", "4-cycle", "tailed-triangle",
                                   "3-star", "4-path", "wedge", "generic"};
    d = std::string("family: ") + kNames[family] + " (k = " + std::to_string(k) + ")";
  } else {
    if (pattern->k < 3 || pattern->k > (uint32_t)kGenMaxK || pattern->n_edges > 28)
      return fail(GPM_E_UNSUPPORTED_PATTERN, "gpm_pattern_describe: patterns have 3 to 8 vertices");
    std::vector<std::pair<int, int>> edges;
    for (uint32_t i = 0; i < pattern->n_edges; i++) {
      const int a = pattern->edges[i][0], b = pattern->edges[i][1];
      edges.push_back({std::min(a, b), std::max(a, b)});
    }
    std::sort(edges.begin(), edges.end());
    edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
    GenTable gt{};
    std::string why;
    if (!analyze_pattern(pattern->k, edges, induced ? 1 : 0, (double)n, n ? (double)nnz / n : 0.0,
                         &gt, &why))
      return fail(GPM_E_UNSUPPORTED_PATTERN, "gpm_pattern_describe: " + why);
    d = "family: generic (k = " + std::to_string(pattern->k) + "); " + describe_gen(gt);
  }
  const size_t nb = std::min(len - 1, d.size());
  memcpy(buf, d.data(), nb);
  buf[nb] = 0;
  return d.size() < len ? GPM_OK : fail(GPM_E_CAPACITY, "gpm_pattern_describe: text truncated");
}

gpm_status gpm_plan_describe(const gpm_plan_t* p, char* buf, size_t len) {
  if (!p || !buf || len == 0) return fail(GPM_E_INVALID_ARG, "gpm_plan_describe: bad argument");
  static const char* kNames[] = {"", "k-clique", "diamond", "4-cycle", "tailed-triangle",
                                 "3-star", "4-path", "wedge", "generic"};
  std::string d = std::string("family: ") + kNames[p->family] + " (k = " + std::to_string(p->k) + ")";
  if (p->family == kGeneric) d += "; " + describe_gen(p->gen);
  else if (p->lgs) d += "; local graph search";
  const size_t nb = std::min(len - 1, d.size());
  memcpy(buf, d.data(), nb);
  buf[nb] = 0;
  return d.size() < len ? GPM_OK : fail(GPM_E_CAPACITY, "gpm_plan_describe: text truncated");
}

}  // extern "C"

namespace gpm {

// Enqueue one evaluation of plan p over tasks [lo, hi) on stream s and the
// copy of its control block to pinned host memory; no synchronisation.
cudaError_t plan_launch_async(gpm_plan_t* p, uint64_t lo, uint64_t hi, uint32_t* list_out,
                              uint64_t cap, cudaStream_t s) {
  hi = std::min(hi, p->tasks.count);
  lo = std::min(lo, hi);
  cudaError_t e = cudaMemsetAsync(p->ctl_d, 0, sizeof(Control), s);
  if (e == cudaSuccess && hi > lo) {
    if (p->wedge && lo == 0 && hi == p->tasks.count)
      e = launch_cycle4_wedge(p->csr, p->graph->deg32_d, p->wedge_cnt, p->wedge_blocks, p->ctl_d,
                              p->cfg.stats ? p->ctl_d->stats : nullptr, s);
    else
      e = p->lgs ? launch_lgs(p, lo, hi, s) : launch_enum(p, lo, hi, list_out, cap, s);
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(p->host_pinned, p->ctl_d, sizeof(Control), cudaMemcpyDeviceToHost, s);
  return e;
}

// Result of the plan's last evaluation once its stream work has completed.
gpm_status plan_finish(gpm_plan_t* p, Control* res) {
  memcpy(res, p->host_pinned, sizeof(Control));
  p->last = *res;
  if (res->error & kErrStack) return fail(GPM_E_CUDA, "device check failed: DFS buffer overflow");
  return GPM_OK;
}

// Device bytes a plan owns for its evaluations (DFS buffers, wedge counters,
// root lists, control block); the graph's cached structures are not counted.
size_t plan_exec_bytes(const gpm_plan_t* p) {
  size_t b = sizeof(Control) + p->gstack_bytes;
  if (p->wedge) b += (size_t)p->wedge_blocks * p->graph->g.n * sizeof(uint32_t);
  for (int c = 0; c < 4; c++) b += p->lgs_count[c] * sizeof(uint32_t);
  b += 2 * p->heavy_count * sizeof(uint64_t);
  return b;
}

gpm_status api_fail(gpm_status st, const std::string& msg) { return fail(st, msg); }

}  // namespace gpm

extern "C" {

static gpm_status run_plan(gpm_plan_t* p, uint64_t lo, uint64_t hi, uint32_t* list_out,
                           uint64_t cap, cudaStream_t s, Control* res) {
  cudaError_t e = plan_launch_async(p, lo, hi, list_out, cap, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "enumeration kernel");
  return plan_finish(p, res);
}

gpm_status gpm_count(gpm_plan_t* p, uint64_t* out_count, void* stream) {
  return gpm_count_range(p, 0, ~0ull, out_count, stream);
}

gpm_status gpm_count_range(gpm_plan_t* p, uint64_t task_lo, uint64_t task_hi, uint64_t* out_count,
                           void* stream) {
  if (!p || !out_count) return fail(GPM_E_INVALID_ARG, "gpm_count: NULL argument");
  if (p->mode != GPM_COUNT) return fail(GPM_E_INVALID_ARG, "gpm_count: plan was built for listing");
  Control r;
  gpm_status st = run_plan(p, task_lo, task_hi, nullptr, 0, (cudaStream_t)stream, &r);
  if (st != GPM_OK) return st;
  *out_count = r.result;
  return GPM_OK;
}

gpm_status gpm_list(gpm_plan_t* p, uint32_t* out_dev, uint64_t capacity, uint64_t* n_written,
                    uint64_t* n_total, void* stream) {
  if (!p || !n_written || !n_total || (!out_dev && capacity))
    return fail(GPM_E_INVALID_ARG, "gpm_list: NULL argument");
  if (p->mode != GPM_LIST) return fail(GPM_E_INVALID_ARG, "gpm_list: plan was built for counting");
  Control r;
  gpm_status st = run_plan(p, 0, ~0ull, out_dev, capacity, (cudaStream_t)stream, &r);
  if (st != GPM_OK) return st;
  const uint64_t written = std::min<uint64_t>(r.result, capacity);
  const cudaError_t e = unrename_ids(p->graph, out_dev, written * p->k, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "gpm_list renaming");
  *n_total = r.result;
  *n_written = written;
  if (r.result > capacity)
    return fail(GPM_E_CAPACITY, "gpm_list: output truncated to capacity");
  return GPM_OK;
}

gpm_status gpm_plan_stats(const gpm_plan_t* p, uint64_t* alg_bytes, uint64_t* set_ops,
                          uint64_t* word_ops) {
  if (!p) return fail(GPM_E_INVALID_ARG, "gpm_plan_stats: NULL plan");
  if (!p->cfg.stats) return fail(GPM_E_INVALID_ARG, "gpm_plan_stats: plan built without collect_stats");
  if (alg_bytes) *alg_bytes = p->last.stats[0];
  if (set_ops) *set_ops = p->last.stats[1];
  if (word_ops) *word_ops = p->last.stats[2];
  return GPM_OK;
}

void gpm_plan_free(gpm_plan_t* p) {
  if (!p) return;
  cudaFree(p->ctl_d);
  cudaFree(p->gstack_d);
  for (int c = 0; c < 4; c++) cudaFree(p->lgs_verts[c]);
  cudaFree(p->heavy_idx);
  cudaFree(p->overflow_d);
  cudaFree(p->wedge_cnt);
  cudaFree(p->gen_d);
  if (p->host_pinned) cudaFreeHost(p->host_pinned);
  delete p;
}

}  // extern "C"
