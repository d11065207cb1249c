// motif.cuh — types shared by the motif kernels (motif.cu) and their host
// side (batch.cu).
#pragma once
#include "gpm_internal.cuh"

namespace gpm {

// One graph of a batch, as the motif kernels see it.
struct MotifGraph {
  DevCsr g;              // undirected CSR
  DevCsr dag;            // degree-oriented DAG
  const uint32_t* lsrc;  // tasks v1 > v2
  const uint32_t* ldst;
  const uint32_t* dsrc;  // DAG arc sources
  const uint32_t* deg;   // undirected degrees
};

// Per-graph sums accumulated by the kernels.
enum MotifSum : int { kSt = 0, kSdia, kStt, kSp4, kSw, kSs, kC4, kK4, kNumSums };

struct MotifBatchArgs {
  const MotifGraph* graphs;
  uint32_t n_graphs;
  const uint64_t* prefix;    // per-graph task prefix [n_graphs + 1] of the kernel's task space
  unsigned long long* next;  // queue head
  unsigned long long* sums;  // [n_graphs][kNumSums]
  uint32_t chunk;
  uint32_t ratio;
  // k_motif_k4 only: when idx is set, the tasks are the arcs idx[0, *idx_count)
  // packed graph << 40 | arc instead of the prefix's arc space
  const uint64_t* idx;
  const unsigned long long* idx_count;
};

// Root lists of the batched local graph search for 4-cliques: the vertices of
// out-degree class c (kmin <= d+ and bounds[c-1] < d+ <= bounds[c]) of every
// graph, packed graph << 32 | vertex in (graph, vertex) order, and the arcs of
// the vertices above the last bound, packed graph << 40 | arc.
struct BatchRoots {
  uint64_t* roots[4] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t count[4] = {0, 0, 0, 0};
  uint64_t* heavy = nullptr;
  uint64_t heavy_count = 0;
};
// a.graphs / a.n_graphs / a.prefix (the vertex space) describe the batch.
cudaError_t build_batch_roots(const MotifBatchArgs& a, uint64_t nverts, uint32_t kmin,
                              const uint32_t* bounds, int nclass, int sms, BatchRoots* out,
                              cudaStream_t s);
void free_batch_roots(BatchRoots* r);

uint32_t motif_c4_threads();
cudaError_t launch_motif_edges(const MotifBatchArgs& a, unsigned blocks, unsigned threads,
                               cudaStream_t s);
cudaError_t launch_motif_vertices(const MotifBatchArgs& a, unsigned blocks, cudaStream_t s);
cudaError_t launch_motif_k4(const MotifBatchArgs& a, unsigned blocks, unsigned threads,
                            uint32_t scap, cudaStream_t s);
cudaError_t launch_motif_c4(const MotifBatchArgs& a, unsigned blocks, uint32_t* cnt, uint32_t max_n,
                            cudaStream_t s);

}  // namespace gpm
