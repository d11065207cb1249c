// enum_wedge.cu — counting-only 4-cycle kernel (pattern decomposition,
// Section 5.4 (1)).
//
// An edge-induced 4-cycle x-w1-y-w2-x is a pair of wedges x-w-y with the same
// endpoints.  Root every cycle at its highest-ranked vertex x (rank = the
// orientation key (degree, id), Section 4.2); then both middles w and the
// opposite vertex y rank below x, and the cycles rooted at x number
//     sum over y of C(c_xy, 2),   c_xy = |{w in N(x) : w, y rank below x, y in N(w)}|.
// Each cycle is counted exactly once (its top vertex fixes x, and y is the
// vertex opposite x).  Ranking by degree keeps the wedge scans on the
// low-degree side of every edge: the work is sum over w of d(w) * |{x in N(w)
// ranked above w}|.
//
// One CTA per root x (persistent grid, dynamic queue).  c_xy lives in a dense
// per-CTA counter array in HBM (n uint32, zero between roots): pass 1 adds one
// per wedge, pass 2 reads each counter back with an exchange-to-zero, so the
// first reader of y collects C(c_xy, 2) and the array is clean for the next
// root.  Warps take the lower neighbours w of x dynamically; lanes stride
// over N(w).
#include <algorithm>

#include "enum_common.cuh"

namespace gpm {
namespace {

constexpr int kWedgeThreads = 512;

__device__ __forceinline__ bool ranks_below(uint32_t dy, uint32_t y, uint32_t dx, uint32_t x) {
  return dy < dx || (dy == dx && y < x);
}

__global__ void __launch_bounds__(kWedgeThreads) k_cycle4_wedge(DevCsr g, const uint32_t* __restrict__ deg,
                                                                uint32_t* __restrict__ cnt_all,
                                                                Control* ctl, unsigned long long* stats) {
  uint32_t* cnt = cnt_all + (size_t)blockIdx.x * g.n;
  __shared__ unsigned long long s_x;
  __shared__ unsigned int s_w;
  __shared__ unsigned long long s_acc;
  const uint32_t lane = lane_id();
  if (threadIdx.x == 0) s_acc = 0;
  unsigned long long acc = 0, wedges = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_x = atomicAdd(&ctl->next, 1ull);
      s_w = 0;
    }
    __syncthreads();
    const uint64_t xq = s_x;
    if (xq >= g.n) break;
    const uint32_t x = (uint32_t)xq;
    const uint32_t dx = deg[x];
    if (dx < 2) continue;
    const uint32_t* Nx = g.nbr + g.off[x];
    for (int pass = 0; pass < 2; pass++) {
      for (;;) {
        unsigned int i = 0;
        if (lane == 0) i = atomicAdd(&s_w, 1u);
        i = __shfl_sync(kFull, i, 0);
        if (i >= dx) break;
        const uint32_t w = Nx[i];
        const uint32_t dw = deg[w];
        if (!ranks_below(dw, w, dx, x)) continue;  // warp-uniform
        const uint32_t* Nw = g.nbr + g.off[w];
        for (uint32_t j = lane; j < dw; j += 32) {
          const uint32_t y = Nw[j];
          if (!ranks_below(deg[y], y, dx, x)) continue;
          if (pass == 0) {
            atomicAdd(&cnt[y], 1u);
            if (stats) wedges++;
          } else {
            const unsigned long long c = atomicExch(&cnt[y], 0u);
            acc += c * (c - (c > 0)) / 2;  // C(c, 2), 0 for c <= 1
          }
        }
      }
      __syncthreads();
      if (threadIdx.x == 0) s_w = 0;
      __syncthreads();
    }
  }
  acc = warp_sum_u64(acc);
  if (lane == 0 && acc) atomicAdd(&s_acc, acc);
  if (stats) {
    wedges = warp_sum_u64(wedges);
    // bytes per wedge: neighbour id + its degree (8 B) and the counter's
    // read-modify-write in both passes (16 B)
    if (lane == 0 && wedges) atomicAdd(&stats[0], wedges * 24ull);
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_acc) atomicAdd(&ctl->result, s_acc);
}

__global__ void k_degrees(const int64_t* __restrict__ off, uint32_t n, uint32_t* __restrict__ deg) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
    deg[v] = (uint32_t)(off[v + 1] - off[v]);
}

}  // namespace

uint32_t wedge_threads() { return kWedgeThreads; }

cudaError_t degrees32(const DevCsr& g, uint32_t* deg, int sms, cudaStream_t s) {
  if (!g.n) return cudaSuccess;
  const unsigned blocks = std::max(1u, std::min<unsigned>((g.n + 255) / 256, (unsigned)sms * 8u));
  k_degrees<<<blocks, 256, 0, s>>>(g.off, g.n, deg);
  return cudaGetLastError();
}

cudaError_t launch_cycle4_wedge(const DevCsr& g, const uint32_t* deg, uint32_t* cnt, unsigned blocks,
                                Control* ctl, unsigned long long* stats, cudaStream_t s) {
  k_cycle4_wedge<<<blocks, kWedgeThreads, 0, s>>>(g, deg, cnt, ctl, stats);
  return cudaGetLastError();
}

}  // namespace gpm
