// enum_common.cuh — the warp-centric, edge-parallel DFS skeleton (Section 5.1).
//
// One warp owns one root task (an edge / arc of Omega) at a time and walks its
// whole subtree; all 32 lanes cooperate on every set operation (two-level
// parallelism, Section 5.1).  Warps of a persistent grid pull chunks of tasks
// from a device-wide atomic queue head (the single-GPU form of the chunked
// scheduling of Section 7.1); the chunk shrinks to one task near the end of
// the queue so that heavy tails spread over all warps.  Intermediate sets of
// the DFS (the buffers W of Algorithm 1, at most X <= k-3 of them, Section
// 7.2 (3)) live in a per-warp shared-memory slab when the task's bound fits,
// else in a per-warp slice of an HBM buffer sized when the plan is built.
#pragma once
#include <cuda_runtime.h>

#include "gpm_internal.cuh"
#include "setops.cuh"

namespace gpm {

struct EnumArgs {
  DevCsr g;            // CSR walked by the plan (the DAG for cliques)
  const uint32_t* src;  // task sources
  const uint32_t* dst;  // task destinations
  uint64_t lo, hi;     // task range [lo, hi)
  Control* ctl;
  uint32_t* list_out;  // device listing buffer (k uint32 per match) or null
  uint64_t list_cap;   // capacity in matches
  uint32_t* gstack;    // per-warp HBM buffers: levels x gcap entries per warp
  uint32_t gcap;       // entries per level in HBM
  uint32_t scap;       // entries per level in shared memory
  uint32_t levels;     // buffered levels per warp
  uint32_t chunk;      // tasks per queue grab
  uint32_t ratio;      // binary-search vs merge threshold
  unsigned long long* stats;  // null, or {algorithmic bytes, set operations, word-ops}
  const uint64_t* idx;  // null, or: task t is arc idx[t] (counted if in [arc_lo, arc_hi))
  uint64_t arc_lo, arc_hi;
  const unsigned long long* idx_count;  // null, or the device-side length of idx
  const GenTable* gen;  // generic plans: the search plan (device memory), else null
  // vertex parallelism (Section 5.1): task t is vertex lo + t and its root
  // tasks (v1, v2) are v2 in row v1 of g (vkind = kTasksLower: only v2 < v1);
  // no task list Omega exists
  uint32_t vertex_tasks;
  uint32_t vkind;
};

// One graph of a batch as the local-graph-search kernels see it.
struct LgsGraph {
  DevCsr dag;            // degree-oriented DAG
  const int64_t* uoff;   // undirected offsets (degrees)
  const uint32_t* src;   // DAG arc sources
};

// Arguments of the local-graph-search clique kernels (enum_lgs.cu).
struct LgsArgs {
  DevCsr dag;
  const int64_t* uoff;  // undirected offsets (degrees define the DAG rank)
  const uint32_t* verts;  // root vertices of one out-degree class (ascending)
  uint64_t nverts;
  uint64_t lo, hi;  // arc (task) range
  unsigned long long* next;
  unsigned long long* result;
  unsigned long long* stats;
  // arc roots (heavy vertices): arcs idx[0, nidx) with sources src[]; arcs
  // whose member set is too large are appended to overflow[]
  const uint64_t* idx;
  uint64_t nidx;
  const uint32_t* src;
  uint64_t* overflow;
  unsigned long long* overflow_count;
  // batch mode (graphs != null): roots are broots[0, nverts or nidx) packed as
  // graph << 32 | vertex (vertex roots) or graph << 40 | arc (arc roots); each
  // root's count is added to gsums[graph * gstride + gslot]; overflow arcs are
  // appended packed the same way
  const LgsGraph* graphs;
  const uint64_t* broots;
  unsigned long long* gsums;
  uint32_t gstride, gslot;
};

// Algorithmic bytes of one set operation A∘B (|A| <= |B| after ordering):
// the operand elements the cheaper of the two textbook algorithms must read
// (a full merge reads |A| + |B|; a search reads |A| plus ceil(log2(|B|+1))
// probes per element of A), the offsets of the fetched list (16 B) and the
// written result.  Only accumulated when a plan asks for statistics.
__device__ __forceinline__ void stat_setop(const EnumArgs& a, uint32_t na, uint32_t nb,
                                           uint32_t written) {
  if (a.stats && lane_id() == 0) {
    const uint32_t lo = min(na, nb), hi = max(na, nb);
    const unsigned long long probe = (unsigned long long)lo * (32 - __clz(hi));
    const unsigned long long b = 4ull * (lo + min((unsigned long long)hi, probe)) + 16ull +
                                 4ull * written;
    atomicAdd(&a.stats[0], b);
    atomicAdd(&a.stats[1], 1ull);
  }
}

// Set operations of the plans, with optional statistics.
template <SetOut OUT>
__device__ __forceinline__ uint32_t isect(const EnumArgs& a, const uint32_t* A, uint32_t na,
                                          const uint32_t* B, uint32_t nb, uint32_t* out) {
  const uint32_t r = warp_intersect<OUT>(A, na, B, nb, out, a.ratio);
  stat_setop(a, na, nb, OUT == kWrite ? r : 0);
  return r;
}
template <SetOut OUT>
__device__ __forceinline__ uint32_t diff(const EnumArgs& a, const uint32_t* A, uint32_t na,
                                         const uint32_t* B, uint32_t nb, uint32_t* out) {
  const uint32_t r = warp_difference<OUT>(A, na, B, nb, out, a.ratio);
  stat_setop(a, na, nb, OUT == kWrite ? r : 0);
  return r;
}

__device__ __forceinline__ uint32_t deg_of(const DevCsr& g, uint32_t v) {
  return (uint32_t)(g.off[v + 1] - g.off[v]);
}
__device__ __forceinline__ const uint32_t* row_of(const DevCsr& g, uint32_t v) {
  return g.nbr + g.off[v];
}

// Per-task buffer set: level l at base + l * stride.
struct Bufs {
  uint32_t* base;
  uint32_t stride;
  uint32_t cap;
  __device__ __forceinline__ uint32_t* level(int l) const { return base + (size_t)l * stride; }
};

// Choose shared or HBM storage for a task whose every buffered set has at most
// `bound` elements.  Sets the error word (and returns cap 0) if even the HBM
// slice is too small, which a correctly sized plan never does.
__device__ __forceinline__ Bufs pick_bufs(const EnumArgs& a, uint32_t* sbuf, uint32_t* gbuf,
                                          uint32_t bound) {
  if (bound <= a.scap) return Bufs{sbuf, a.scap, a.scap};
  return Bufs{gbuf, a.gcap, a.gcap};
}

// Reserve `n` listing slots; returns the first slot index (warp-uniform).
__device__ __forceinline__ unsigned long long list_reserve(const EnumArgs& a, uint32_t n) {
  unsigned long long base = 0;
  if (lane_id() == 0 && n) base = atomicAdd(&a.ctl->list_head, (unsigned long long)n);
  return __shfl_sync(kFull, base, 0);
}

// Emit s matches of K vertices: fixed[0..K) with slot `slot` replaced by C[j].
template <int K>
__device__ __forceinline__ void emit_set(const EnumArgs& a, const uint32_t (&fixed)[K], int slot,
                                         const uint32_t* C, uint32_t s) {
  if (s == 0) return;
  const unsigned long long base = list_reserve(a, s);
  for (uint32_t j = lane_id(); j < s; j += 32) {
    const unsigned long long m = base + j;
    if (m < a.list_cap) {
      uint32_t* o = a.list_out + m * K;
#pragma unroll
      for (int q = 0; q < K; q++) o[q] = (q == slot) ? C[j] : fixed[q];
    }
  }
}

// Emit one match (lane 0 writes).
template <int K>
__device__ __forceinline__ void emit_one(const EnumArgs& a, const uint32_t (&m)[K]) {
  const unsigned long long base = list_reserve(a, 1);
  if (lane_id() == 0 && base < a.list_cap) {
    uint32_t* o = a.list_out + base * K;
#pragma unroll
    for (int q = 0; q < K; q++) o[q] = m[q];
  }
}

// The persistent task loop.  `Plan::run(a, v1, v2, sbuf, gbuf)` processes one
// root task with the whole warp and returns its match count (warp-uniform).
template <class Plan>
__device__ __forceinline__ void task_loop(const EnumArgs& a) {
  extern __shared__ uint32_t s_dyn[];
  __shared__ unsigned long long s_acc;
  const uint32_t lane = lane_id();
  const uint32_t wib = threadIdx.x >> 5;
  const uint32_t wpb = blockDim.x >> 5;
  const uint64_t gw = (uint64_t)blockIdx.x * wpb + wib;
  const uint64_t total_warps = (uint64_t)gridDim.x * wpb;
  if (threadIdx.x == 0) s_acc = 0;
  __syncthreads();
  uint32_t* sbuf = s_dyn + (size_t)wib * a.scap * a.levels;
  uint32_t* gbuf = a.gstack ? a.gstack + gw * (uint64_t)a.gcap * a.levels : nullptr;
  const uint64_t ntask = a.idx_count ? min((uint64_t)*a.idx_count, a.hi - a.lo) : a.hi - a.lo;
  unsigned long long acc = 0;
  uint64_t seen = 0;
  for (;;) {
    // shrink the grab near the end of the queue (guided self-scheduling)
    const uint32_t c = (seen + (uint64_t)a.chunk * total_warps * 2 < ntask) ? a.chunk : 1u;
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(&a.ctl->next, (unsigned long long)c);
    start = __shfl_sync(kFull, start, 0);
    if (start >= ntask) break;
    seen = start;
    const uint64_t end = min((uint64_t)start + c, ntask);
    for (uint64_t t = start; t < end; t++) {
      uint64_t e = a.lo + t;
      if (a.vertex_tasks) {
        const uint32_t v1 = (uint32_t)e;
        const uint32_t* R = row_of(a.g, v1);
        const uint32_t d = deg_of(a.g, v1);
        const uint32_t nr = (a.vkind == kTasksLower) ? warp_count_less(R, d, v1) : d;
        for (uint32_t j = 0; j < nr; j++) acc += Plan::run(a, v1, R[j], sbuf, gbuf);
        continue;
      }
      if (a.idx) {
        e = a.idx[t];
        if (e < a.arc_lo || e >= a.arc_hi) continue;  // warp-uniform
      }
      const uint32_t v1 = a.src[e];
      const uint32_t v2 = a.dst[e];
      acc += Plan::run(a, v1, v2, sbuf, gbuf);
    }
    if (a.stats && lane == 0)  // (src, dst) per task, or the offsets of a task vertex
      atomicAdd(&a.stats[0], (a.vertex_tasks ? 16ull : 8ull) * (end - start));
  }
  if (lane == 0 && acc) atomicAdd(&s_acc, acc);
  __syncthreads();
  if (threadIdx.x == 0 && s_acc) atomicAdd(&a.ctl->result, s_acc);
}

}  // namespace gpm
