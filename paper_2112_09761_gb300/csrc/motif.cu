// motif.cu — 3- and 4-motif counting over one or many graphs (Section 5.3
// multi-pattern fission, Section 5.4 (1) counting-only pruning by pattern
// decomposition), each kernel one persistent launch over a device-side task
// space of (graph, root) pairs spanning every graph of the batch.
//
// Vertex-induced motif counts follow from edge-induced ones (each pattern's
// edge-induced count is a fixed combination of the vertex-induced counts of
// its supergraphs on the same vertices), and the edge-induced counts need
// only a few per-edge and per-vertex quantities:
//   per edge e = (a, b), t_e = |N(a) ∩ N(b)|          (triangle-sharing kernel)
//       S_t   = Σ t_e            (= 3 T)
//       S_dia = Σ C(t_e, 2)      (edge-induced diamonds, Algorithm 3)
//       S_tt  = Σ t_e (d_a + d_b - 4)   (= 2 x edge-induced tailed triangles)
//       S_p4  = Σ (d_a - 1)(d_b - 1)    (4-paths + 3 T)
//   per vertex:  S_w = Σ C(d, 2) (wedges),  S_s = Σ C(d, 3) (3-stars)
//   4-cycles: wedge pairs (enum_wedge.cu);  4-cliques: DAG arcs (sorted sets).
// The patterns sharing the triangle sub-pattern (tailed triangle, diamond)
// are fused into the one per-edge kernel; 4-cycles and 4-cliques run as
// separate kernels (fission).  The host applies the inversion.
#include <algorithm>

#include "enum_common.cuh"
#include "motif.cuh"

namespace gpm {

namespace {

// Graph index holding global task t (prefix non-decreasing, prefix[0] = 0).
__device__ __forceinline__ uint32_t graph_of(const uint64_t* prefix, uint32_t n, uint64_t t,
                                             uint32_t hint) {
  if (hint < n && prefix[hint] <= t && t < prefix[hint + 1]) return hint;
  uint32_t lo = 0, hi = n;  // largest g with prefix[g] <= t
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ unsigned long long choose2u(unsigned long long x) {
  return x ? x * (x - 1) / 2 : 0;
}
__device__ __forceinline__ unsigned long long choose3u(unsigned long long x) {
  return x >= 3 ? x * (x - 1) * (x - 2) / 6 : 0;
}

// Warp-held per-graph partial sums, flushed when the warp moves to another graph.
template <int NS>
struct Partial {
  uint32_t g = 0xffffffffu;
  unsigned long long v[NS] = {};
  __device__ __forceinline__ void flush(const MotifBatchArgs& a, const int (&slot)[NS]) {
    if (g != 0xffffffffu && lane_id() == 0) {
#pragma unroll
      for (int i = 0; i < NS; i++)
        if (v[i]) atomicAdd(&a.sums[(size_t)g * kNumSums + slot[i]], v[i]);
    }
#pragma unroll
    for (int i = 0; i < NS; i++) v[i] = 0;
  }
};

// Triangle-sharing kernel: warp per edge task (v1 > v2).
__global__ void __launch_bounds__(256) k_motif_edges(MotifBatchArgs a) {
  const uint32_t lane = lane_id();
  const uint64_t total = a.prefix[a.n_graphs];
  Partial<4> part;
  const int slots[4] = {kSt, kSdia, kStt, kSp4};
  uint32_t hint = 0;
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(a.next, (unsigned long long)a.chunk);
    start = __shfl_sync(kFull, start, 0);
    if (start >= total) break;
    const uint64_t end = min((uint64_t)start + a.chunk, total);
    for (uint64_t t = start; t < end; t++) {
      const uint32_t g = graph_of(a.prefix, a.n_graphs, t, hint);
      hint = g;
      if (g != part.g) {
        part.flush(a, slots);
        part.g = g;
      }
      const MotifGraph& G = a.graphs[g];
      const uint64_t lt = t - a.prefix[g];
      const uint32_t v1 = G.lsrc[lt], v2 = G.ldst[lt];
      const uint32_t d1 = G.deg[v1], d2 = G.deg[v2];
      const unsigned long long te = warp_intersect<kCountOnly>(
          G.g.nbr + G.g.off[v1], d1, G.g.nbr + G.g.off[v2], d2, nullptr, a.ratio);
      part.v[0] += te;
      part.v[1] += choose2u(te);
      part.v[2] += te ? te * (unsigned long long)(d1 + d2 - 4) : 0ull;  // te > 0 => d1, d2 >= 2
      part.v[3] += (unsigned long long)(d1 - 1) * (d2 - 1);
    }
  }
  part.flush(a, slots);
}

// Per-vertex wedge and 3-star sums: thread per vertex of the batch.
__global__ void k_motif_vertices(MotifBatchArgs a) {
  const uint64_t total = a.prefix[a.n_graphs];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t hint = 0;
  // stride loop with warp-uniform trip count so that the graph-wise warp
  // reduction below always has all lanes
  const uint64_t trips = (total + stride - 1) / stride;
  for (uint64_t r = 0; r < trips; r++) {
    const uint64_t t = r * stride + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long w = 0, s = 0;
    uint32_t g = 0xffffffffu;
    if (t < total) {
      g = graph_of(a.prefix, a.n_graphs, t, hint);
      hint = g;
      const uint32_t d = a.graphs[g].deg[t - a.prefix[g]];
      w = choose2u(d);
      s = choose3u(d);
    }
    const unsigned peers = __match_any_sync(kFull, g);
    const int leader = __ffs(peers) - 1;
    // reduce over lanes of the same graph
    unsigned long long ws = 0, ss = 0;
    for (int l = 0; l < 32; l++) {
      const unsigned long long wl = __shfl_sync(kFull, w, l);
      const unsigned long long sl = __shfl_sync(kFull, s, l);
      if ((peers >> l) & 1u) { ws += wl; ss += sl; }
    }
    if ((int)lane_id() == leader && g != 0xffffffffu) {
      if (ws) atomicAdd(&a.sums[(size_t)g * kNumSums + kSw], ws);
      if (ss) atomicAdd(&a.sums[(size_t)g * kNumSums + kSs], ss);
    }
  }
}

// 4-cliques: warp per DAG arc (u, v); W = N+(u) ∩ N+(v), count arcs inside W.
__global__ void __launch_bounds__(256) k_motif_k4(MotifBatchArgs a, uint32_t scap) {
  extern __shared__ uint32_t s_w[];
  const uint32_t lane = lane_id();
  uint32_t* W = s_w + (threadIdx.x >> 5) * scap;
  const uint64_t total = a.idx ? (uint64_t)*a.idx_count : a.prefix[a.n_graphs];
  Partial<1> part;
  const int slots[1] = {kK4};
  uint32_t hint = 0;
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(a.next, (unsigned long long)a.chunk);
    start = __shfl_sync(kFull, start, 0);
    if (start >= total) break;
    const uint64_t end = min((uint64_t)start + a.chunk, total);
    for (uint64_t t = start; t < end; t++) {
      uint32_t g;
      uint64_t lt;
      if (a.idx) {
        const uint64_t r = a.idx[t];
        g = (uint32_t)(r >> 40);
        lt = r & ((1ull << 40) - 1);
      } else {
        g = graph_of(a.prefix, a.n_graphs, t, hint);
        hint = g;
        lt = t - a.prefix[g];
      }
      if (g != part.g) {
        part.flush(a, slots);
        part.g = g;
      }
      const MotifGraph& G = a.graphs[g];
      const uint32_t u = G.dsrc[lt], v = G.dag.nbr[lt];
      const uint32_t du = (uint32_t)(G.dag.off[u + 1] - G.dag.off[u]);
      const uint32_t dv = (uint32_t)(G.dag.off[v + 1] - G.dag.off[v]);
      const uint32_t* Nu = G.dag.nbr + G.dag.off[u];
      const uint32_t* Nv = G.dag.nbr + G.dag.off[v];
      if (min(du, dv) <= scap) {
        const uint32_t s = warp_intersect<kWrite>(Nu, du, Nv, dv, W, a.ratio);
        __syncwarp();
        for (uint32_t i = 0; i < s; i++) {
          const uint32_t w = W[i];
          const uint32_t dw = (uint32_t)(G.dag.off[w + 1] - G.dag.off[w]);
          part.v[0] += warp_intersect<kCountOnly>(W, s, G.dag.nbr + G.dag.off[w], dw, nullptr,
                                                  a.ratio);
        }
        __syncwarp();
      } else {
        // candidate set beyond the shared slab: test each w in N+(u) ∩ N+(v)
        // on the fly (no buffer): for w in N+(u) with w in N+(v), count
        // |N+(u) ∩ N+(v) ∩ N+(w)| as |(N+(u) ∩ N+(w)) ∩ N+(v)| lane by lane
        for (uint32_t i = 0; i < du; i++) {
          const uint32_t w = Nu[i];
          if (!lane_contains(Nv, dv, w)) continue;  // warp-uniform
          const uint32_t* Nw = G.dag.nbr + G.dag.off[w];
          const uint32_t dw = (uint32_t)(G.dag.off[w + 1] - G.dag.off[w]);
          unsigned long long c = 0;
          for (uint32_t j = lane; j < dw; j += 32) {
            const uint32_t x = Nw[j];
            c += (lane_contains(Nu, du, x) && lane_contains(Nv, dv, x)) ? 1u : 0u;
          }
          part.v[0] += warp_sum_u64(c);
        }
      }
    }
  }
  part.flush(a, slots);
}

// 4-cycles: CTA per root vertex of the batch (wedge pairs, see enum_wedge.cu).
constexpr int kC4Threads = 512;

__device__ __forceinline__ bool below(uint32_t dy, uint32_t y, uint32_t dx, uint32_t x) {
  return dy < dx || (dy == dx && y < x);
}

__global__ void __launch_bounds__(kC4Threads) k_motif_c4(MotifBatchArgs a, uint32_t* cnt_all,
                                                         uint32_t max_n) {
  uint32_t* cnt = cnt_all + (size_t)blockIdx.x * max_n;
  __shared__ unsigned long long s_x;
  __shared__ unsigned int s_w;
  __shared__ unsigned long long s_acc;
  const uint32_t lane = lane_id();
  const uint64_t total = a.prefix[a.n_graphs];
  uint32_t hint = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_x = atomicAdd(a.next, 1ull);
      s_w = 0;
      s_acc = 0;
    }
    __syncthreads();
    const uint64_t t = s_x;
    if (t >= total) break;
    const uint32_t g = graph_of(a.prefix, a.n_graphs, t, hint);
    hint = g;
    const MotifGraph& G = a.graphs[g];
    const uint32_t x = (uint32_t)(t - a.prefix[g]);
    const uint32_t dx = G.deg[x];
    if (dx < 2) continue;
    const uint32_t* Nx = G.g.nbr + G.g.off[x];
    unsigned long long acc = 0;
    for (int pass = 0; pass < 2; pass++) {
      for (;;) {
        unsigned int i = 0;
        if (lane == 0) i = atomicAdd(&s_w, 1u);
        i = __shfl_sync(kFull, i, 0);
        if (i >= dx) break;
        const uint32_t w = Nx[i];
        const uint32_t dw = G.deg[w];
        if (!below(dw, w, dx, x)) continue;
        const uint32_t* Nw = G.g.nbr + G.g.off[w];
        for (uint32_t j = lane; j < dw; j += 32) {
          const uint32_t y = Nw[j];
          if (!below(G.deg[y], y, dx, x)) continue;
          if (pass == 0) {
            atomicAdd(&cnt[y], 1u);
          } else {
            const unsigned long long c = atomicExch(&cnt[y], 0u);
            acc += c ? c * (c - 1) / 2 : 0;
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_w = 0;
      __syncthreads();
    }
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(&s_acc, acc);
    __syncthreads();
    if (threadIdx.x == 0 && s_acc) atomicAdd(&a.sums[(size_t)g * kNumSums + kC4], s_acc);
  }
}

// Root lists of the batched local graph search.  mode 0: flag[t] = 1 if
// vertex t of the batch (vertex space) has kmin <= d+, lo < d+ <= hi; mode 1:
// flag[t] = d+ if d+ > lo (its arcs become arc roots), else 0.
__global__ void k_broot_flags(MotifBatchArgs a, uint64_t total, uint32_t kmin, uint32_t lo,
                              uint32_t hi, int mode, uint32_t* __restrict__ flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t hint = 0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const uint32_t g = graph_of(a.prefix, a.n_graphs, t, hint);
    hint = g;
    const DevCsr& dag = a.graphs[g].dag;
    const uint64_t v = t - a.prefix[g];
    const uint32_t d = (uint32_t)(dag.off[v + 1] - dag.off[v]);
    if (mode == 0) flag[t] = (d >= kmin && d > lo && d <= hi) ? 1u : 0u;
    else flag[t] = d > lo ? d : 0u;
  }
}

__global__ void k_broot_scatter(MotifBatchArgs a, uint64_t total, const uint32_t* __restrict__ flag,
                                const int64_t* __restrict__ pos, uint64_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t hint = 0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    if (!flag[t]) continue;
    const uint32_t g = graph_of(a.prefix, a.n_graphs, t, hint);
    hint = g;
    out[pos[t]] = ((uint64_t)g << 32) | (t - a.prefix[g]);
  }
}

// warp per vertex: the arcs of a heavy vertex, packed graph << 40 | arc
__global__ void k_broot_arcs(MotifBatchArgs a, uint64_t total, const uint32_t* __restrict__ cnt,
                             const int64_t* __restrict__ pos, uint64_t* __restrict__ out) {
  const uint32_t lane = lane_id();
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t hint = 0;
  for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total; t += nwarps) {
    const uint32_t c = cnt[t];
    if (!c) continue;
    const uint32_t g = graph_of(a.prefix, a.n_graphs, t, hint);
    hint = g;
    const uint64_t first = (uint64_t)a.graphs[g].dag.off[t - a.prefix[g]];
    for (uint32_t i = lane; i < c; i += 32) out[pos[t] + i] = ((uint64_t)g << 40) | (first + i);
  }
}

}  // namespace

uint32_t motif_c4_threads() { return kC4Threads; }

cudaError_t launch_motif_edges(const MotifBatchArgs& a, unsigned blocks, unsigned threads,
                               cudaStream_t s) {
  k_motif_edges<<<blocks, threads, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_motif_vertices(const MotifBatchArgs& a, unsigned blocks, cudaStream_t s) {
  k_motif_vertices<<<blocks, 256, 0, s>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_motif_k4(const MotifBatchArgs& a, unsigned blocks, unsigned threads,
                            uint32_t scap, cudaStream_t s) {
  const size_t smem = (size_t)(threads / 32) * scap * sizeof(uint32_t);
  if (smem > 40 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_motif_k4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_motif_k4<<<blocks, threads, smem, s>>>(a, scap);
  return cudaGetLastError();
}
cudaError_t launch_motif_c4(const MotifBatchArgs& a, unsigned blocks, uint32_t* cnt, uint32_t max_n,
                            cudaStream_t s) {
  k_motif_c4<<<blocks, kC4Threads, 0, s>>>(a, cnt, max_n);
  return cudaGetLastError();
}

cudaError_t scan_offsets(const uint32_t* in, uint64_t n, int64_t* out, cudaStream_t s);

cudaError_t build_batch_roots(const MotifBatchArgs& a, uint64_t total, uint32_t kmin,
                              const uint32_t* bounds, int nclass, int sms, BatchRoots* out,
                              cudaStream_t s) {
  *out = BatchRoots{};
  if (total == 0) return cudaSuccess;
  uint32_t* flag = nullptr;
  int64_t* pos = nullptr;
  cudaError_t e = cudaMalloc((void**)&flag, (total + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&pos, (total + 1) * sizeof(int64_t));
  const unsigned blocks = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + 255) / 256, (uint64_t)sms * 8));
  for (int c = 0; c <= nclass && e == cudaSuccess; c++) {
    const bool heavy = c == nclass;
    const uint32_t lo = heavy ? bounds[nclass - 1] : (c ? bounds[c - 1] : 0u);
    const uint32_t hi = heavy ? 0u : bounds[c];
    k_broot_flags<<<blocks, 256, 0, s>>>(a, total, kmin, lo, hi, heavy ? 1 : 0, flag);
    e = scan_offsets(flag, total, pos, s);
    int64_t n = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&n, pos + total, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || n == 0) continue;
    uint64_t* list = nullptr;
    e = cudaMalloc((void**)&list, (size_t)n * sizeof(uint64_t));
    if (e != cudaSuccess) break;
    if (heavy) {
      const unsigned wb = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((total + 7) / 8, (uint64_t)sms * 16));
      k_broot_arcs<<<wb, 256, 0, s>>>(a, total, flag, pos, list);
      out->heavy = list;
      out->heavy_count = (uint64_t)n;
    } else {
      k_broot_scatter<<<blocks, 256, 0, s>>>(a, total, flag, pos, list);
      out->roots[c] = list;
      out->count[c] = (uint64_t)n;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(flag);
  cudaFree(pos);
  if (e != cudaSuccess) free_batch_roots(out);
  return e;
}

void free_batch_roots(BatchRoots* r) {
  for (auto& p : r->roots) cudaFree(p);
  cudaFree(r->heavy);
  *r = BatchRoots{};
}

}  // namespace gpm
