// batch.cu — C ABI of motif counting over one graph or a batch of graphs:
// per-graph preprocessing, the device task spaces, the captured CUDA graph of
// the four kernel families, the autotuner and the edge- to vertex-induced
// inversion.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "enum_common.cuh"
#include "gpm_internal.cuh"
#include "motif.cuh"

namespace gpm {

cudaError_t degrees32(const DevCsr& g, uint32_t* deg, int sms, cudaStream_t s);
void set_error(const std::string& msg);
uint32_t lgs_warp_max_degree();
uint32_t lgs_block_max_degree();
cudaError_t lgs_launch_warp(int k, const LgsArgs& a, unsigned blocks, cudaStream_t s);
cudaError_t lgs_launch_block(int k, int nw, bool arc, const LgsArgs& a, unsigned blocks_per_sm,
                             unsigned sms, cudaStream_t s);
int lgs_block_occupancy(int k, int nw);

}  // namespace gpm

using namespace gpm;

struct gpm_batch_s {
  uint32_t n_graphs = 0;
  uint32_t k = 0;
  int num_sms = 0;
  MotifGraph* graphs_d = nullptr;
  uint64_t* prefix_d[3] = {nullptr, nullptr, nullptr};  // edge tasks, arcs, vertices
  uint64_t totals[3] = {0, 0, 0};
  unsigned long long* sums_d = nullptr;   // [n_graphs][kNumSums]
  unsigned long long* next_d = nullptr;   // kQueues queue heads and counters
  unsigned long long* sums_h = nullptr;   // pinned
  uint32_t* c4_cnt = nullptr;
  uint32_t max_n = 0;
  unsigned c4_blocks = 0;
  uint32_t k4_scap = 0;
  // 4-cliques by local graph search (unless disabled): root lists of the
  // whole batch, per-graph descriptors, heavy arcs whose arc-level local graph
  // is too large (counted by k_motif_k4 from their list)
  bool lgs = false;
  BatchRoots roots;
  LgsGraph* lgs_graphs_d = nullptr;
  uint64_t* overflow_d = nullptr;
  unsigned lgs_warp_blocks = 1;
  unsigned lgs_bps[4] = {1, 1, 1, 1};
  uint32_t chunk = 16, ratio = 8, wpb = 8;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// next_d slots: queue heads of the edge, vertex, k4 and c4 kernels, of the
// four LGS classes and the heavy arcs, of the overflow pass, and the overflow
// list length
constexpr int kQueues = 11;
constexpr int kQLgs = 4, kQHeavy = 8, kQOverflow = 9, kOverflowCount = 10;

gpm_status fail(gpm_status st, const std::string& m) {
  set_error(m);
  return st;
}
gpm_status cfail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation) return fail(GPM_E_OOM, std::string(where) + ": out of device memory");
  return fail(GPM_E_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

MotifBatchArgs args_for(const gpm_batch_s* b, int space, int queue) {
  MotifBatchArgs a;
  a.graphs = b->graphs_d;
  a.n_graphs = b->n_graphs;
  a.prefix = b->prefix_d[space];
  a.next = b->next_d + queue;
  a.sums = b->sums_d;
  a.chunk = b->chunk;
  a.ratio = b->ratio;
  a.idx = nullptr;
  a.idx_count = nullptr;
  return a;
}

// 4-cliques of the whole batch by local graph search: one launch per
// out-degree class, one over the arcs of heavier roots, then the sorted-set
// kernel over the arcs whose arc-level local graph is still too large.
cudaError_t enqueue_lgs_k4(gpm_batch_s* b, cudaStream_t s) {
  static const int kClassWords[4] = {0, 8, 16, 32};
  const unsigned sms = (unsigned)b->num_sms;
  LgsArgs la{};
  la.lo = 0;
  la.hi = ~0ull;
  la.graphs = b->lgs_graphs_d;
  la.gsums = b->sums_d;
  la.gstride = kNumSums;
  la.gslot = kK4;
  la.overflow = b->overflow_d;
  la.overflow_count = b->next_d + kOverflowCount;
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < 4 && e == cudaSuccess; c++) {
    if (!b->roots.count[c]) continue;
    la.broots = b->roots.roots[c];
    la.nverts = b->roots.count[c];
    la.next = b->next_d + kQLgs + c;
    if (c == 0) e = lgs_launch_warp(4, la, b->lgs_warp_blocks, s);
    else e = lgs_launch_block(4, kClassWords[c], false, la, b->lgs_bps[c], sms, s);
  }
  if (e == cudaSuccess && b->roots.heavy_count) {
    la.broots = b->roots.heavy;
    la.nverts = 0;
    la.nidx = b->roots.heavy_count;
    la.next = b->next_d + kQHeavy;
    e = lgs_launch_block(4, 32, true, la, b->lgs_bps[3], sms, s);
    MotifBatchArgs m = args_for(b, 1, kQOverflow);
    m.idx = b->overflow_d;
    m.idx_count = b->next_d + kOverflowCount;
    if (e == cudaSuccess) e = launch_motif_k4(m, sms * (64 / b->wpb), b->wpb * 32, b->k4_scap, s);
  }
  return e;
}

// Enqueue one full batch evaluation on stream s (also used under capture).
cudaError_t enqueue(gpm_batch_s* b, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(b->sums_d, 0, (size_t)b->n_graphs * kNumSums * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->next_d, 0, kQueues * sizeof(unsigned long long), s);
  const unsigned sms = (unsigned)b->num_sms;
  if (e == cudaSuccess && b->totals[0])
    e = launch_motif_edges(args_for(b, 0, 0), sms * (64 / b->wpb), b->wpb * 32, s);
  if (e == cudaSuccess && b->totals[2])
    e = launch_motif_vertices(args_for(b, 2, 1), sms * 4, s);
  if (b->k == 4) {
    if (e == cudaSuccess && b->lgs) e = enqueue_lgs_k4(b, s);
    else if (e == cudaSuccess && b->totals[1])
      e = launch_motif_k4(args_for(b, 1, 2), sms * (64 / b->wpb), b->wpb * 32, b->k4_scap, s);
    if (e == cudaSuccess && b->totals[2])
      e = launch_motif_c4(args_for(b, 2, 3), b->c4_blocks, b->c4_cnt, b->max_n, s);
  }
  return e;
}

cudaError_t capture(gpm_batch_s* b) {
  if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
  if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
  cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e2 = enqueue(b, b->cap_stream);
  e = cudaStreamEndCapture(b->cap_stream, &b->graph);
  if (e2 != cudaSuccess) return e2;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&b->exec, b->graph, 0);
}

// Vertex-induced counts from the per-graph sums (the inversion).
void finish(const unsigned long long* s, uint32_t k, uint64_t* out) {
  const uint64_t T = s[kSt] / 3;
  if (k == 3) {
    out[0] = s[kSw] - 3 * T;  // induced wedges
    out[1] = T;
    return;
  }
  const uint64_t P4 = s[kSp4] - 3 * T, S3 = s[kSs], C4 = s[kC4], TT = s[kStt] / 2,
                 DI = s[kSdia], K4 = s[kK4];
  const uint64_t k4 = K4;
  const uint64_t di = DI - 6 * k4;
  const uint64_t c4 = C4 - di - 3 * k4;
  const uint64_t tt = TT - 4 * di - 12 * k4;
  const uint64_t s3 = S3 - tt - 2 * di - 4 * k4;
  const uint64_t p4 = P4 - 2 * tt - 4 * c4 - 6 * di - 12 * k4;
  out[0] = p4; out[1] = s3; out[2] = c4; out[3] = tt; out[4] = di; out[5] = k4;
}

float time_once(gpm_batch_s* b, cudaStream_t s) {
  cudaEvent_t a, z;
  cudaEventCreate(&a);
  cudaEventCreate(&z);
  cudaEventRecord(a, s);
  cudaError_t e = enqueue(b, s);
  cudaEventRecord(z, s);
  cudaEventSynchronize(z);
  float ms = 1e30f;
  if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, z);
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  return ms;
}

}  // namespace

extern "C" {

gpm_status gpm_batch_create(gpm_graph* const* graphs, uint32_t n_graphs, uint32_t k,
                            const gpm_plan_opts* opts, void* stream, gpm_batch_t** out) {
  if (!graphs || !out || n_graphs == 0) return fail(GPM_E_INVALID_ARG, "gpm_batch_create: bad arguments");
  if (k != 3 && k != 4) return fail(GPM_E_INVALID_ARG, "gpm_batch_create: k must be 3 or 4");
  for (uint32_t i = 0; i < n_graphs; i++)
    if (!graphs[i]) return fail(GPM_E_INVALID_ARG, "gpm_batch_create: NULL graph");
  cudaStream_t s = (cudaStream_t)stream;
  gpm_batch_s* b = new gpm_batch_s();
  b->n_graphs = n_graphs;
  b->k = k;
  b->num_sms = graphs[0]->num_sms;
  std::vector<MotifGraph> hg(n_graphs);
  std::vector<uint64_t> pre[3];
  for (auto& v : pre) v.assign(n_graphs + 1, 0);
  uint32_t max_dplus = 1;
  uint64_t max_arcs = 0;
  cudaError_t e = cudaSuccess;
  for (uint32_t i = 0; i < n_graphs && e == cudaSuccess; i++) {
    gpm_graph* G = graphs[i];
    e = build_lower(G, s);
    if (e == cudaSuccess && k == 4) e = build_dag(G, s);
    if (e == cudaSuccess && !G->deg32_d && G->g.n) {
      e = cudaMalloc((void**)&G->deg32_d, (size_t)G->g.n * sizeof(uint32_t));
      if (e == cudaSuccess) e = degrees32(G->g, G->deg32_d, G->num_sms, s);
    }
    if (e != cudaSuccess) break;
    hg[i].g = G->g;
    hg[i].dag = DevCsr{G->doff_d, G->dnbr_d, G->g.n, G->dag_arcs};
    hg[i].lsrc = G->lsrc_d;
    hg[i].ldst = G->ldst_d;
    hg[i].dsrc = G->dsrc_d;
    hg[i].deg = G->deg32_d;
    pre[0][i + 1] = pre[0][i] + G->lower_count;
    pre[1][i + 1] = pre[1][i] + (k == 4 ? G->dag_arcs : 0);
    pre[2][i + 1] = pre[2][i] + G->g.n;
    b->max_n = std::max(b->max_n, G->g.n);
    max_dplus = std::max(max_dplus, G->max_out_degree);
    max_arcs = std::max<uint64_t>(max_arcs, G->dag_arcs);
  }
  if (e != cudaSuccess) { gpm_batch_free(b); return cfail(e, "gpm_batch_create preprocessing"); }
  for (int sp = 0; sp < 3; sp++) b->totals[sp] = pre[sp][n_graphs];
  e = cudaMalloc((void**)&b->graphs_d, n_graphs * sizeof(MotifGraph));
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->graphs_d, hg.data(), n_graphs * sizeof(MotifGraph), cudaMemcpyHostToDevice, s);
  for (int sp = 0; sp < 3 && e == cudaSuccess; sp++) {
    e = cudaMalloc((void**)&b->prefix_d[sp], (n_graphs + 1) * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->prefix_d[sp], pre[sp].data(), (n_graphs + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->sums_d, (size_t)n_graphs * kNumSums * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->next_d, kQueues * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->sums_h, (size_t)n_graphs * kNumSums * sizeof(unsigned long long));
  if (e == cudaSuccess && k == 4) {
    b->k4_scap = std::min<uint32_t>(max_dplus, 512);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const uint64_t per = (uint64_t)std::max<uint32_t>(b->max_n, 1) * sizeof(uint32_t);
    uint64_t blocks = (uint64_t)b->num_sms * 2;
    blocks = std::min<uint64_t>(blocks, std::max<uint64_t>(1, (free_b / 2) / per));
    b->c4_blocks = (unsigned)blocks;
    e = cudaMalloc((void**)&b->c4_cnt, blocks * per);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->c4_cnt, 0, blocks * per, s);
  }
  gpm_plan_opts o;
  memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  // packed roots hold the graph index in the top 24 bits of an arc root
  const bool packable = n_graphs < (1u << 24) && max_arcs < (1ull << 40);
  if (e == cudaSuccess && k == 4 && !o.no_lgs && b->totals[1] && packable) {
    // vertex roots by out-degree class, the arcs of heavier roots, and the
    // descriptors the LGS kernels read their graph from
    b->lgs = true;
    const uint32_t bounds[4] = {lgs_warp_max_degree(), 256, 512, lgs_block_max_degree()};
    MotifBatchArgs va = args_for(b, 2, 0);
    e = build_batch_roots(va, b->totals[2], 3, bounds, 4, b->num_sms, &b->roots, s);
    std::vector<LgsGraph> lg(n_graphs);
    for (uint32_t i = 0; i < n_graphs; i++) lg[i] = LgsGraph{hg[i].dag, hg[i].g.off, hg[i].dsrc};
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->lgs_graphs_d, n_graphs * sizeof(LgsGraph));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->lgs_graphs_d, lg.data(), n_graphs * sizeof(LgsGraph), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && b->roots.heavy_count)
      e = cudaMalloc((void**)&b->overflow_d, b->roots.heavy_count * sizeof(uint64_t));
    b->lgs_warp_blocks = (unsigned)std::min<uint64_t>(
        (uint64_t)b->num_sms * 8, std::max<uint64_t>(1, (b->roots.count[0] + 7) / 8));
    b->lgs_bps[1] = (unsigned)lgs_block_occupancy(4, 8);
    b->lgs_bps[2] = (unsigned)lgs_block_occupancy(4, 16);
    b->lgs_bps[3] = (unsigned)lgs_block_occupancy(4, 32);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { gpm_batch_free(b); return cfail(e, "gpm_batch_create"); }

  if (o.chunk || o.bsearch_ratio || o.warps_per_block) {
    b->chunk = o.chunk ? o.chunk : 16;
    b->ratio = o.bsearch_ratio ? o.bsearch_ratio : 8;
    b->wpb = o.warps_per_block ? std::min(o.warps_per_block, 8u) : 8;
  } else {
    // autotuner: task chunk x intersection threshold x CTA shape, one timed
    // pass each on this batch (after one warm-up pass), fastest kept
    const uint32_t chunks[] = {4, 32};
    const uint32_t ratios[] = {4, 16};
    const uint32_t wpbs[] = {4, 8};
    float best = 1e30f;
    uint32_t bc = 16, br = 8, bw = 8;
    b->chunk = bc; b->ratio = br; b->wpb = bw;
    time_once(b, s);
    for (uint32_t c : chunks)
      for (uint32_t r : ratios)
        for (uint32_t w : wpbs) {
          b->chunk = c; b->ratio = r; b->wpb = w;
          const float ms = time_once(b, s);
          if (ms < best) { best = ms; bc = c; br = r; bw = w; }
        }
    b->chunk = bc; b->ratio = br; b->wpb = bw;
    e = cudaGetLastError();
    if (e != cudaSuccess) { gpm_batch_free(b); return cfail(e, "gpm_batch_create autotune"); }
  }
  e = capture(b);
  if (e != cudaSuccess) { gpm_batch_free(b); return cfail(e, "gpm_batch_create graph capture"); }
  *out = b;
  return GPM_OK;
}

gpm_status gpm_batch_count(gpm_batch_t* b, uint64_t* out, void* stream) {
  if (!b || !out) return fail(GPM_E_INVALID_ARG, "gpm_batch_count: NULL argument");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = (size_t)b->n_graphs * kNumSums * sizeof(unsigned long long);
  cudaError_t e = cudaGraphLaunch(b->exec, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->sums_h, b->sums_d, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cfail(e, "gpm_batch_count");
  const uint32_t w = b->k == 3 ? 2 : 6;
  for (uint32_t i = 0; i < b->n_graphs; i++) finish(b->sums_h + (size_t)i * kNumSums, b->k, out + (size_t)i * w);
  return GPM_OK;
}

gpm_status gpm_batch_info(const gpm_batch_t* b, uint32_t* chunk, uint32_t* bsearch_ratio,
                          uint32_t* warps_per_block) {
  if (!b) return fail(GPM_E_INVALID_ARG, "gpm_batch_info: NULL batch");
  if (chunk) *chunk = b->chunk;
  if (bsearch_ratio) *bsearch_ratio = b->ratio;
  if (warps_per_block) *warps_per_block = b->wpb;
  return GPM_OK;
}

void gpm_batch_free(gpm_batch_t* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  cudaFree(b->graphs_d);
  for (auto p : b->prefix_d) cudaFree(p);
  cudaFree(b->sums_d);
  cudaFree(b->next_d);
  if (b->sums_h) cudaFreeHost(b->sums_h);
  cudaFree(b->c4_cnt);
  free_batch_roots(&b->roots);
  cudaFree(b->lgs_graphs_d);
  cudaFree(b->overflow_d);
  delete b;
}

gpm_status gpm_motif_count(gpm_graph* g, uint32_t k, uint64_t* out, void* stream) {
  if (!g || !out) return fail(GPM_E_INVALID_ARG, "gpm_motif_count: NULL argument");
  gpm_plan_opts o;
  memset(&o, 0, sizeof(o));
  o.chunk = 16;
  o.bsearch_ratio = 8;
  o.warps_per_block = 8;
  gpm_batch_t* b = nullptr;
  gpm_status st = gpm_batch_create(&g, 1, k, &o, stream, &b);
  if (st != GPM_OK) return st;
  st = gpm_batch_count(b, out, stream);
  gpm_batch_free(b);
  return st;
}

}  // extern "C"
