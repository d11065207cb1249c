// prep.cu — graph loader and preprocessor kernels (Section 4.2, Section 7.2).
//
//  * validation: offsets monotone, IDs in range, rows strictly ascending
//    (sorted, no duplicates), no self-loops, both directions present;
//    maximum degree (input information, Section 4.2);
//  * orientation: u -> v iff (deg u, u) < (deg v, v) (Section 4.2; halves
//    |E| and bounds the out-degree); arcs keep ascending ID order;
//  * root task lists: DAG arcs, reduced pairs v1 > v2 (Section 7.2 (2)) and
//    all directed entries, each as (src, dst) arrays;
//  * a device-wide exclusive scan used to turn per-vertex counts into offsets.
#include <cuda_runtime.h>

#include <algorithm>

#include "gpm_internal.cuh"
#include "setops.cuh"

namespace gpm {

uint64_t sort_capacity(uint64_t n);
cudaError_t sort_keys(uint64_t* keys, uint64_t n, int sms, cudaStream_t s);

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// ------------------------------------------------------------------ scan

__device__ __forceinline__ long long block_exclusive_scan(long long x, long long* s_warp,
                                                          long long* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const long long y = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_warp[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    long long w = (lane < (int)(blockDim.x >> 5)) ? s_warp[lane] : 0;
    long long winc = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(kFull, winc, o);
      if (lane >= o) winc += y;
    }
    s_warp[lane] = winc - w;          // exclusive warp offsets
    if (lane == 31) s_warp[32] = winc;  // block total
  }
  __syncthreads();
  const long long r = s_warp[warp] + inc - x;
  *total = s_warp[32];
  __syncthreads();
  return r;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ in, uint64_t n, long long* bsum) {
  __shared__ long long s_warp[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  long long acc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    const uint64_t i = base + (uint64_t)j * kScanThreads + threadIdx.x;
    if (i < n) acc += in[i];
  }
  long long total;
  block_exclusive_scan(acc, s_warp, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_blocksums(long long* bsum, uint64_t nb) {
  __shared__ long long s_warp[33];
  long long carry = 0;
  for (uint64_t base = 0; base < nb; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    const long long x = (i < nb) ? bsum[i] : 0;
    long long total;
    const long long ex = block_exclusive_scan(x, s_warp, &total);
    if (i < nb) bsum[i] = carry + ex;
    carry += total;
  }
}

// out[i] = sum(in[0..i)), out[n] = sum(in); each thread scans kScanItems
// consecutive elements of its block's tile.
__global__ void k_scan_apply(const uint32_t* __restrict__ in, uint64_t n,
                             const long long* __restrict__ bsum, int64_t* __restrict__ out) {
  __shared__ long long s_warp[33];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  long long acc = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    v[j] = (base + j < n) ? in[base + j] : 0u;
    acc += v[j];
  }
  long long total;
  long long run = block_exclusive_scan(acc, s_warp, &total) + bsum[blockIdx.x];
#pragma unroll
  for (int j = 0; j < kScanItems; j++) {
    if (base + j < n) out[base + j] = run;
    run += v[j];
  }
  if (base < n && base + kScanItems >= n) out[n] = run;  // thread holding the last element
}

// Exclusive scan of n uint32 counts into n+1 int64 offsets.
cudaError_t exclusive_scan(const uint32_t* in, uint64_t n, int64_t* out, cudaStream_t s) {
  if (n == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  const uint64_t nb = (n + kScanTile - 1) / kScanTile;
  long long* bsum = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&bsum, nb * sizeof(long long), s);
  if (e != cudaSuccess) return e;
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum);
  k_scan_blocksums<<<1, 1024, 0, s>>>(bsum, nb);
  k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, bsum, out);
  e = cudaGetLastError();
  cudaFreeAsync(bsum, s);
  return e;
}

// ------------------------------------------------------------ validation

__global__ void k_check_offsets(const int64_t* __restrict__ off, uint32_t n, uint64_t nnz,
                                unsigned* flags) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int64_t a = off[v], b = off[v + 1];
    if (a < 0 || b < a || (uint64_t)b > nnz) atomicOr(flags, kBadOffsets);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0 && (off[0] != 0 || (uint64_t)off[n] != nnz))
    atomicOr(flags, kBadOffsets);
}

// Warp per vertex: range, order, self-loop checks and the maximum degree.
__global__ void k_check_rows(DevCsr g, unsigned* flags, unsigned* max_deg) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned bad = 0, dmax = 0;
  for (uint64_t v = warp; v < g.n; v += nwarps) {
    const int64_t s = g.off[v], e = g.off[v + 1];
    dmax = max(dmax, (unsigned)(e - s));
    for (int64_t i = s + lane; i < e; i += 32) {
      const uint32_t x = g.nbr[i];
      if (x >= g.n) bad |= kBadRange;
      if (x == v) bad |= kBadSelfLoop;
      if (i + 1 < e) {
        const uint32_t y = g.nbr[i + 1];
        if (y == x) bad |= kBadDuplicate;
        else if (y < x) bad |= kBadUnsorted;
      }
    }
  }
  bad = __reduce_or_sync(kFull, bad);
  dmax = __reduce_max_sync(kFull, dmax);
  if (lane == 0) {
    if (bad) atomicOr(flags, bad);
    atomicMax(max_deg, dmax);
  }
}

// Warp per vertex v: every u in N(v) must have v in N(u).
__global__ void k_check_symmetry(DevCsr g, unsigned* flags) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  bool bad = false;
  for (uint64_t v = warp; v < g.n; v += nwarps) {
    const int64_t s = g.off[v], e = g.off[v + 1];
    for (int64_t i = s + lane; i < e; i += 32) {
      const uint32_t u = g.nbr[i];
      const int64_t us = g.off[u], ue = g.off[u + 1];
      if (!lane_contains(g.nbr + us, (uint32_t)(ue - us), (uint32_t)v)) bad = true;
    }
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(flags, kBadAsymmetric);
}

// ------------------------------------------------------------ orientation

__device__ __forceinline__ bool arc(uint64_t du, uint32_t u, uint64_t dv, uint32_t v) {
  return du < dv || (du == dv && u < v);
}

__global__ void k_outdeg(DevCsr g, uint32_t* outdeg, unsigned* max_out) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned m = 0;
  for (uint64_t u = warp; u < g.n; u += nwarps) {
    const int64_t s = g.off[u], e = g.off[u + 1];
    const uint64_t du = (uint64_t)(e - s);
    uint32_t c = 0;
    for (int64_t i = s + lane; i < e; i += 32) {
      const uint32_t v = g.nbr[i];
      c += arc(du, (uint32_t)u, (uint64_t)(g.off[v + 1] - g.off[v]), v);
    }
    c = __reduce_add_sync(kFull, c);
    if (lane == 0) outdeg[u] = c;
    m = max(m, c);
  }
  if (lane == 0) atomicMax(max_out, m);
}

__global__ void k_fill_dag(DevCsr g, const int64_t* __restrict__ doff, uint32_t* __restrict__ dnbr,
                           uint32_t* __restrict__ dsrc) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = warp; u < g.n; u += nwarps) {
    const int64_t s = g.off[u], e = g.off[u + 1];
    const uint64_t du = (uint64_t)(e - s);
    int64_t w = doff[u];
    for (int64_t base = s; base < e; base += 32) {
      const int64_t i = base + lane;
      bool keep = false;
      uint32_t v = 0;
      if (i < e) {
        v = g.nbr[i];
        keep = arc(du, (uint32_t)u, (uint64_t)(g.off[v + 1] - g.off[v]), v);
      }
      const unsigned m = __ballot_sync(kFull, keep);
      if (keep) {
        const int64_t pos = w + __popc(m & lanemask_lt());
        dnbr[pos] = v;
        dsrc[pos] = (uint32_t)u;
      }
      w += __popc(m);
    }
  }
}

// ------------------------------------------------------------ task lists

__global__ void k_rows(DevCsr g, uint32_t* __restrict__ row) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < g.n; v += nwarps)
    for (int64_t i = g.off[v] + lane; i < g.off[v + 1]; i += 32) row[i] = (uint32_t)v;
}

__global__ void k_lower_count(DevCsr g, uint32_t* __restrict__ cnt) {
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < g.n; v += nwarps) {
    const int64_t s = g.off[v];
    const uint32_t c = warp_count_less(g.nbr + s, (uint32_t)(g.off[v + 1] - s), (uint32_t)v);
    if (lane_id() == 0) cnt[v] = c;
  }
}

__global__ void k_lower_fill(DevCsr g, const int64_t* __restrict__ loff, uint32_t* __restrict__ src,
                             uint32_t* __restrict__ dst) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < g.n; v += nwarps) {
    const int64_t s = g.off[v];
    const int64_t len = loff[v + 1] - loff[v];
    for (int64_t i = lane; i < len; i += 32) {
      src[loff[v] + i] = (uint32_t)v;
      dst[loff[v] + i] = g.nbr[s + i];
    }
  }
}

// class flag of every vertex for the local graph search
__global__ void k_lgs_flags(const int64_t* __restrict__ doff, uint32_t n, uint32_t kmin, uint32_t lo,
                            uint32_t hi, uint32_t* __restrict__ flag) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint64_t d = (uint64_t)(doff[v + 1] - doff[v]);
    flag[v] = (d >= kmin && d > lo && d <= hi) ? 1u : 0u;
  }
}

__global__ void k_lgs_scatter(const uint32_t* __restrict__ flag, const int64_t* __restrict__ pos,
                              uint32_t n, uint32_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    if (flag[v]) out[pos[v]] = (uint32_t)v;
}

// Root order inside a class: descending out-degree (then ascending ID), so the
// largest local graphs start first and the launch's tail is made of small ones.
__global__ void k_order_keys(const int64_t* __restrict__ doff, const uint32_t* __restrict__ verts,
                             uint64_t count, uint64_t* __restrict__ keys) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    const uint32_t v = verts[i];
    const uint32_t d = (uint32_t)(doff[v + 1] - doff[v]);
    keys[i] = ((uint64_t)(0xffffffffu - d) << 32) | v;
  }
}

__global__ void k_order_apply(const uint64_t* __restrict__ keys, uint64_t count,
                              uint32_t* __restrict__ verts) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    verts[i] = (uint32_t)keys[i];
}

// out-degree of heavy roots (else 0), then the arc indices of those roots
__global__ void k_heavy_deg(const int64_t* __restrict__ doff, uint32_t n, uint32_t lo,
                            uint32_t* __restrict__ cnt) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint64_t d = (uint64_t)(doff[v + 1] - doff[v]);
    cnt[v] = d > lo ? (uint32_t)d : 0u;
  }
}

__global__ void k_heavy_fill(const int64_t* __restrict__ doff, const uint32_t* __restrict__ cnt,
                             const int64_t* __restrict__ pos, uint32_t n, uint64_t* __restrict__ out) {
  const uint32_t lane = lane_id();
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < n; v += nwarps)
    for (uint32_t i = lane; i < cnt[v]; i += 32) out[pos[v] + i] = (uint64_t)doff[v] + i;
}

inline unsigned grid_for(uint64_t items_per_warp_units, int sms) {
  // warp-per-item kernels: enough blocks to fill the GPU, bounded by work
  const uint64_t want = (items_per_warp_units + 7) / 8;  // 8 warps per 256-thread block
  const uint64_t cap = (uint64_t)sms * 16;
  return (unsigned)std::max<uint64_t>(1, std::min(want, cap));
}

}  // namespace

// Exclusive scan of n uint32 counts into n + 1 int64 offsets (out[n] = total).
cudaError_t scan_offsets(const uint32_t* in, uint64_t n, int64_t* out, cudaStream_t s) {
  return exclusive_scan(in, n, out, s);
}

cudaError_t validate_csr(const DevCsr& g, bool full, cudaStream_t s, unsigned* flags_out,
                         uint32_t* max_degree_out) {
  unsigned* d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, 2 * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  cudaMemsetAsync(d, 0, 2 * sizeof(unsigned), s);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned h[2] = {0, 0};
  k_check_offsets<<<std::max(1u, std::min<unsigned>((g.n + 255) / 256, sms * 8u)), 256, 0, s>>>(
      g.off, g.n, g.nnz, d);
  e = cudaMemcpyAsync(h, d, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h[0] == 0 && g.n > 0) {
    k_check_rows<<<grid_for(g.n, sms), 256, 0, s>>>(g, d, d + 1);
    e = cudaMemcpyAsync(h, d, 2 * sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && h[0] == 0 && full) {
      k_check_symmetry<<<grid_for(g.n, sms), 256, 0, s>>>(g, d);
      e = cudaMemcpyAsync(h, d, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaFreeAsync(d, s);
  *flags_out = h[0];
  *max_degree_out = h[1];
  return e;
}

__global__ void k_widen(const int32_t* __restrict__ in, uint64_t count, int64_t* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
    out[i] = in[i];
}

// int32 device offsets -> the library's int64 offsets.
cudaError_t widen_offsets(const int32_t* in, uint64_t count, int64_t* out, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::min<uint64_t>((count + 255) / 256, 4096);
  k_widen<<<std::max(1u, blocks), 256, 0, s>>>(in, count, out);
  return cudaGetLastError();
}

cudaError_t build_dag(gpm_graph* G, cudaStream_t s) {
  if (G->doff_d) return cudaSuccess;
  const DevCsr& g = G->g;
  uint32_t* outdeg = nullptr;
  unsigned* dmax = nullptr;
  cudaError_t e = cudaMalloc((void**)&outdeg, ((size_t)g.n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dmax, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMalloc((void**)&G->doff_d, ((size_t)g.n + 1) * sizeof(int64_t));
  if (e != cudaSuccess) { cudaFree(outdeg); cudaFree(dmax); cudaFree(G->doff_d); G->doff_d = nullptr; return e; }
  cudaMemsetAsync(dmax, 0, sizeof(unsigned), s);
  if (g.n) k_outdeg<<<grid_for(g.n, G->num_sms), 256, 0, s>>>(g, outdeg, dmax);
  e = exclusive_scan(outdeg, g.n, G->doff_d, s);
  int64_t arcs = 0;
  unsigned mo = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&arcs, G->doff_d + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&mo, dmax, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMalloc((void**)&G->dnbr_d, ((size_t)arcs + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&G->dsrc_d, ((size_t)arcs + 1) * sizeof(uint32_t));
  if (e == cudaSuccess && g.n) {
    k_fill_dag<<<grid_for(g.n, G->num_sms), 256, 0, s>>>(g, G->doff_d, G->dnbr_d, G->dsrc_d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(outdeg);
  cudaFree(dmax);
  if (e != cudaSuccess) {
    cudaFree(G->doff_d); cudaFree(G->dnbr_d); cudaFree(G->dsrc_d);
    G->doff_d = nullptr; G->dnbr_d = nullptr; G->dsrc_d = nullptr;
    return e;
  }
  G->dag_arcs = (uint64_t)arcs;
  G->max_out_degree = mo;
  return cudaSuccess;
}

cudaError_t build_rows(gpm_graph* G, cudaStream_t s) {
  if (G->row_d) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&G->row_d, (G->g.nnz + 1) * sizeof(uint32_t));
  if (e != cudaSuccess) { G->row_d = nullptr; return e; }
  if (G->g.n) k_rows<<<grid_for(G->g.n, G->num_sms), 256, 0, s>>>(G->g, G->row_d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { cudaFree(G->row_d); G->row_d = nullptr; }
  return e;
}

cudaError_t build_lgs_classes(gpm_graph* G, uint32_t kmin, const uint32_t* bounds, int nclass,
                              uint32_t** verts, uint64_t* counts, uint64_t** heavy,
                              uint64_t* heavy_count, cudaStream_t s) {
  const uint32_t n = G->g.n;
  uint32_t* flag = nullptr;
  int64_t* pos = nullptr;
  cudaError_t e = cudaMalloc((void**)&flag, ((size_t)n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&pos, ((size_t)n + 1) * sizeof(int64_t));
  const unsigned blocks = std::max(1u, std::min<unsigned>((n + 255) / 256, G->num_sms * 8u));
  for (int c = 0; c < nclass && e == cudaSuccess; c++) {
    verts[c] = nullptr;
    counts[c] = 0;
    k_lgs_flags<<<blocks, 256, 0, s>>>(G->doff_d, n, kmin, c ? bounds[c - 1] : 0u, bounds[c], flag);
    e = exclusive_scan(flag, n, pos, s);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMalloc((void**)&verts[c], ((size_t)total + 1) * sizeof(uint32_t));
    if (e == cudaSuccess && n) k_lgs_scatter<<<blocks, 256, 0, s>>>(flag, pos, n, verts[c]);
    counts[c] = (uint64_t)total;
    if (e == cudaSuccess && total > 1) {
      uint64_t* keys = nullptr;
      e = cudaMalloc((void**)&keys, sort_capacity((uint64_t)total) * sizeof(uint64_t));
      const unsigned ob = std::max(1u, std::min<unsigned>((unsigned)((total + 255) / 256), G->num_sms * 8u));
      if (e == cudaSuccess) {
        k_order_keys<<<ob, 256, 0, s>>>(G->doff_d, verts[c], (uint64_t)total, keys);
        e = sort_keys(keys, (uint64_t)total, G->num_sms, s);
      }
      if (e == cudaSuccess) k_order_apply<<<ob, 256, 0, s>>>(keys, (uint64_t)total, verts[c]);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      cudaFree(keys);
    }
  }
  *heavy = nullptr;
  *heavy_count = 0;
  if (e == cudaSuccess && n) {
    k_heavy_deg<<<blocks, 256, 0, s>>>(G->doff_d, n, bounds[nclass - 1], flag);
    e = exclusive_scan(flag, n, pos, s);
    int64_t total = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, pos + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMalloc((void**)heavy, ((size_t)total + 1) * sizeof(uint64_t));
    if (e == cudaSuccess) k_heavy_fill<<<grid_for(n, G->num_sms), 256, 0, s>>>(G->doff_d, flag, pos, n, *heavy);
    *heavy_count = (uint64_t)total;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(flag);
  cudaFree(pos);
  return e;
}

cudaError_t build_lower(gpm_graph* G, cudaStream_t s) {
  if (G->lsrc_d) return cudaSuccess;
  const DevCsr& g = G->g;
  uint32_t* cnt = nullptr;
  int64_t* loff = nullptr;
  cudaError_t e = cudaMalloc((void**)&cnt, ((size_t)g.n + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&loff, ((size_t)g.n + 1) * sizeof(int64_t));
  if (e != cudaSuccess) { cudaFree(cnt); cudaFree(loff); return e; }
  if (g.n) k_lower_count<<<grid_for(g.n, G->num_sms), 256, 0, s>>>(g, cnt);
  e = exclusive_scan(cnt, g.n, loff, s);
  int64_t total = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&total, loff + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMalloc((void**)&G->lsrc_d, ((size_t)total + 1) * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&G->ldst_d, ((size_t)total + 1) * sizeof(uint32_t));
  if (e == cudaSuccess && g.n) {
    k_lower_fill<<<grid_for(g.n, G->num_sms), 256, 0, s>>>(g, loff, G->lsrc_d, G->ldst_d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(cnt);
  cudaFree(loff);
  if (e != cudaSuccess) {
    cudaFree(G->lsrc_d); cudaFree(G->ldst_d);
    G->lsrc_d = nullptr; G->ldst_d = nullptr;
    return e;
  }
  G->lower_count = (uint64_t)total;
  return cudaSuccess;
}

}  // namespace gpm
