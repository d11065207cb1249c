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
};

uint32_t motif_c4_threads();
cudaError_t launch_motif_edges(const MotifBatchArgs& a, unsigned blocks, unsigned threads,
                               cudaStream_t s);
cudaError_t launch_motif_vertices(const MotifBatchArgs& a, unsigned blocks, cudaStream_t s);
cudaError_t launch_motif_k4(const MotifBatchArgs& a, unsigned blocks, unsigned threads,
                            uint32_t scap, cudaStream_t s);
cudaError_t launch_motif_c4(const MotifBatchArgs& a, unsigned blocks, uint32_t* cnt, uint32_t max_n,
                            cudaStream_t s);

}  // namespace gpm
