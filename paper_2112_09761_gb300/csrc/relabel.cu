// relabel.cu — renaming the data graph by degree order (Section 4.2 preprocessing:
// vertices sorted by degree and renamed; an optional knob, counts are invariant).
//
// New vertex i is the vertex of rank i in ascending (degree, id) order, the same
// total order the clique orientation uses, so in the renamed graph the DAG arcs
// of a vertex are exactly its neighbours with higher IDs.  Both sorts (vertices
// by (degree, id), then arcs by (new source, new target)) sort distinct 64-bit
// keys, so the renamed CSR is unique and deterministic: a bitonic network over a
// power-of-two padded key array, the passes with a compare distance below the
// 2048-key tile done in shared memory, the longer ones as one grid-wide pass per
// distance.
#include <cuda_runtime.h>

#include <algorithm>

#include "gpm_internal.cuh"

namespace gpm {

cudaError_t scan_offsets(const uint32_t* in, uint64_t n, int64_t* out, cudaStream_t s);

namespace {

constexpr uint32_t kTile = 2048;             // keys sorted in shared memory at a time
constexpr uint32_t kTileThreads = kTile / 2;  // one compare-exchange per thread

__device__ __forceinline__ void cmp_swap(uint64_t& a, uint64_t& b, bool ascending) {
  if ((a > b) == ascending) {
    const uint64_t t = a;
    a = b;
    b = t;
  }
}

// Stages k = kfirst .. klast (powers of two, k <= kTile or kfirst == klast) of
// the network on one tile; the first stage starts at distance jfirst, later ones
// at k / 2.  The sort direction of a pair follows bit k of its global index.
__global__ void __launch_bounds__(kTileThreads) k_bitonic_tile(uint64_t* __restrict__ keys,
                                                              uint64_t kfirst, uint64_t klast,
                                                              uint32_t jfirst) {
  __shared__ uint64_t s[kTile];
  const uint64_t base = (uint64_t)blockIdx.x * kTile;
  for (uint32_t t = threadIdx.x; t < kTile; t += blockDim.x) s[t] = keys[base + t];
  __syncthreads();
  for (uint64_t k = kfirst; k <= klast; k <<= 1) {
    for (uint32_t j = (k == kfirst) ? jfirst : (uint32_t)(k >> 1); j > 0; j >>= 1) {
      const uint32_t t = threadIdx.x;
      const uint32_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
      cmp_swap(s[i], s[i + j], ((base + i) & k) == 0);
      __syncthreads();
    }
  }
  for (uint32_t t = threadIdx.x; t < kTile; t += blockDim.x) keys[base + t] = s[t];
}

// One grid-wide pass at distance j >= kTile of stage k.
__global__ void k_bitonic_pass(uint64_t* __restrict__ keys, uint64_t half, uint64_t j, uint64_t k) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride) {
    const uint64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));
    uint64_t a = keys[i], b = keys[i + j];
    const bool asc = (i & k) == 0;
    if ((a > b) == asc) {
      keys[i] = b;
      keys[i + j] = a;
    }
  }
}

// Ascending sort of n2 keys (n2 a power of two, >= kTile).
cudaError_t bitonic_sort(uint64_t* keys, uint64_t n2, int sms, cudaStream_t s) {
  const unsigned tiles = (unsigned)(n2 / kTile);
  k_bitonic_tile<<<tiles, kTileThreads, 0, s>>>(keys, 2, kTile, 1);
  const unsigned grid = (unsigned)std::min<uint64_t>((n2 / 2 + 255) / 256, (uint64_t)sms * 16);
  for (uint64_t k = 2 * (uint64_t)kTile; k <= n2; k <<= 1) {
    for (uint64_t j = k >> 1; j >= kTile; j >>= 1) k_bitonic_pass<<<grid, 256, 0, s>>>(keys, n2 / 2, j, k);
    k_bitonic_tile<<<tiles, kTileThreads, 0, s>>>(keys, k, k, kTile / 2);
  }
  return cudaGetLastError();
}

uint64_t pow2_at_least(uint64_t x) {
  uint64_t p = kTile;
  while (p < x) p <<= 1;
  return p;
}

__global__ void k_vertex_keys(const int64_t* __restrict__ off, uint32_t n, uint64_t n2,
                              uint64_t* __restrict__ keys) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n2; v += stride)
    keys[v] = v < n ? ((uint64_t)(off[v + 1] - off[v]) << 32) | v : ~0ull;
}

// perm[i] = old ID of new vertex i, newid[old] = i, deg_new[i] = its degree
__global__ void k_ranks(const uint64_t* __restrict__ keys, uint32_t n, uint32_t* __restrict__ perm,
                        uint32_t* __restrict__ newid, uint32_t* __restrict__ deg_new) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint32_t old = (uint32_t)keys[i];
    perm[i] = old;
    newid[old] = (uint32_t)i;
    deg_new[i] = (uint32_t)(keys[i] >> 32);
  }
}

// warp per old vertex u: keys of its arcs (newid[u], newid[w]); padding ~0
__global__ void k_arc_keys(const int64_t* __restrict__ off, const uint32_t* __restrict__ nbr,
                           uint32_t n, const uint32_t* __restrict__ newid, uint64_t* __restrict__ keys) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nwarps) {
    const uint64_t hi = (uint64_t)newid[u] << 32;
    for (int64_t t = off[u] + lane; t < off[u + 1]; t += 32) keys[t] = hi | newid[nbr[t]];
  }
}

__global__ void k_fill_u64(uint64_t* __restrict__ p, uint64_t lo, uint64_t hi, uint64_t v) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += stride) p[i] = v;
}

__global__ void k_low_words(const uint64_t* __restrict__ keys, uint64_t nnz, uint32_t* __restrict__ nbr) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz; t += stride)
    nbr[t] = (uint32_t)keys[t];
}

__global__ void k_unrename(uint32_t* __restrict__ ids, uint64_t count, const uint32_t* __restrict__ perm) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    ids[i] = perm[ids[i]];
}

unsigned grid_of(uint64_t items, int sms) {
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((items + 255) / 256, (uint64_t)sms * 16));
}

}  // namespace

// Ascending sort of distinct 64-bit keys: keys holds n entries in an array of
// sort_capacity(n) entries (the rest is overwritten with padding).
uint64_t sort_capacity(uint64_t n) { return pow2_at_least(n); }

cudaError_t sort_keys(uint64_t* keys, uint64_t n, int sms, cudaStream_t s) {
  const uint64_t n2 = pow2_at_least(n);
  if (n2 > n) k_fill_u64<<<grid_of(n2 - n, sms), 256, 0, s>>>(keys, n, n2, ~0ull);
  return bitonic_sort(keys, n2, sms, s);
}

// Rename g in place: new arrays (owned), perm_d = old ID of every new vertex.
cudaError_t relabel_by_degree(gpm_graph* G, cudaStream_t s) {
  const uint32_t n = G->g.n;
  const uint64_t nnz = G->g.nnz;
  const int sms = G->num_sms;
  const uint64_t n2v = pow2_at_least(n), n2a = pow2_at_least(nnz);
  uint64_t* keys = nullptr;
  uint32_t *perm = nullptr, *newid = nullptr, *deg_new = nullptr, *nbr_new = nullptr;
  int64_t* off_new = nullptr;
  cudaError_t e = cudaMalloc((void**)&keys, std::max(n2v, n2a) * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&perm, ((size_t)n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&newid, ((size_t)n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&deg_new, ((size_t)n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&off_new, ((size_t)n + 1) * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&nbr_new, (nnz + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) {
    k_vertex_keys<<<grid_of(n2v, sms), 256, 0, s>>>(G->g.off, n, n2v, keys);
    e = bitonic_sort(keys, n2v, sms, s);
  }
  if (e == cudaSuccess && n) k_ranks<<<grid_of(n, sms), 256, 0, s>>>(keys, n, perm, newid, deg_new);
  if (e == cudaSuccess) e = scan_offsets(deg_new, n, off_new, s);
  if (e == cudaSuccess && nnz) {
    k_fill_u64<<<grid_of(n2a - nnz, sms), 256, 0, s>>>(keys, nnz, n2a, ~0ull);
    k_arc_keys<<<grid_of((uint64_t)n * 32, sms), 256, 0, s>>>(G->g.off, G->g.nbr, n, newid, keys);
    e = bitonic_sort(keys, n2a, sms, s);
    if (e == cudaSuccess) k_low_words<<<grid_of(nnz, sms), 256, 0, s>>>(keys, nnz, nbr_new);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(keys);
  cudaFree(newid);
  cudaFree(deg_new);
  if (e != cudaSuccess) {
    cudaFree(perm);
    cudaFree(off_new);
    cudaFree(nbr_new);
    return e;
  }
  if (!G->borrowed) {
    cudaFree(G->off_d);
    cudaFree(G->nbr_d);
  }
  G->borrowed = false;
  G->off_d = off_new;
  G->nbr_d = nbr_new;
  G->g.off = off_new;
  G->g.nbr = nbr_new;
  G->perm_d = perm;
  return cudaSuccess;
}

// Listed matches back to the caller's vertex IDs.
cudaError_t unrename_ids(const gpm_graph* G, uint32_t* ids, uint64_t count, cudaStream_t s) {
  if (!G->perm_d || !count) return cudaSuccess;
  k_unrename<<<grid_of(count, G->num_sms), 256, 0, s>>>(ids, count, G->perm_d);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace gpm
