// noalloc.cu — triangle counting that allocates no memory.
//
// Some callers cannot allocate device memory at all: latency-critical loops in
// which cudaMalloc / cudaFree may synchronise the device and stall every other
// stream, plug-ins that run inside a host application which owns all device
// memory and forbids its guests to allocate, and processes whose device
// memory is reserved in full up front.  gpm_count_triangles_noalloc serves
// them: the caller passes the graph and the output in device memory it already
// owns, and every byte of working memory the kernels need comes from one
// fixed array in this file, reserved when the library is loaded (every GPU
// that loads the library holds it until the process exits).
//
// Working memory (kScratchWords uint64, 1 MiB):
//   word 0          task queue head
//   word 1          running triangle count
//   words 2 .. n+2  prefix[v] = number of root tasks (v1, v2), v2 < v1, of all
//                   vertices before v — lets warps map a task to its edge
//                   without a task list, and bounds n to kMaxVertices.
// Words 0 and 1 are cleared at the start of every call; the prefix is rewritten
// in full.  Every call shares the array, so calls that overlap on the GPU
// (e.g. on two streams at once) race and give wrong results.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "gpm_internal.cuh"
#include "setops.cuh"

namespace gpm {
gpm_status api_fail(gpm_status st, const std::string& msg);
}  // namespace gpm

using namespace gpm;

namespace {

constexpr uint64_t kScratchWords = 1ull << 17;             // 1 MiB of uint64
constexpr uint64_t kMaxVertices = kScratchWords - 3;       // prefix needs n + 1 words

static __device__ __align__(256) unsigned long long g_noalloc_scratch[kScratchWords];

// Per-device address of g_noalloc_scratch, looked up once with that device
// current (host code must not use the symbol itself as a device address).
std::mutex g_mu;
unsigned long long* g_addr[64] = {};

// Task counts: prefix[v + 1] = |{u in N(v) : u < v}|.
__global__ void k_na_lower(const int64_t* __restrict__ off, const uint32_t* __restrict__ nbr,
                           uint32_t n, unsigned long long* scratch) {
  unsigned long long* prefix = scratch + 2;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const uint32_t* row = nbr + off[v];
    uint32_t lo = 0, hi = (uint32_t)(off[v + 1] - off[v]);
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if (row[mid] < v) lo = mid + 1; else hi = mid;
    }
    prefix[v + 1] = lo;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    prefix[0] = 0;
    scratch[0] = 0;  // queue head
    scratch[1] = 0;  // count
  }
}

// In-place inclusive scan of prefix[1 .. n] by one CTA of 1024 threads.
__global__ void __launch_bounds__(1024) k_na_scan(uint32_t n, unsigned long long* scratch) {
  unsigned long long* prefix = scratch + 2;
  __shared__ unsigned long long s_warp[32];
  __shared__ unsigned long long s_carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint64_t base = 1; base <= n; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    unsigned long long x = (i <= n) ? prefix[i] : 0ull;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(kFull, x, o);
      if ((int)lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = s_warp[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, w, o);
        if ((int)lane >= o) w += y;
      }
      s_warp[lane] = w;
    }
    __syncthreads();
    const unsigned long long add = s_carry + (warp ? s_warp[warp - 1] : 0ull);
    if (i <= n) prefix[i] = x + add;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) s_carry += s_warp[31];
    __syncthreads();
  }
}

// Warp per root task (v1, v2), v2 < v1: count v3 in N(v1) ∩ N(v2) with
// v3 < v2, so every triangle v1 > v2 > v3 is counted once.
__global__ void __launch_bounds__(256) k_na_triangles(const int64_t* __restrict__ off,
                                                      const uint32_t* __restrict__ nbr, uint32_t n,
                                                      unsigned long long* scratch) {
  const unsigned long long* prefix = scratch + 2;
  const uint32_t lane = lane_id();
  const uint64_t total = prefix[n];
  unsigned long long acc = 0;
  uint32_t v1 = 0;
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(&scratch[0], 16ull);
    start = __shfl_sync(kFull, start, 0);
    if (start >= total) break;
    const uint64_t end = min((uint64_t)start + 16, total);
    for (uint64_t t = start; t < end; t++) {
      if (!(prefix[v1] <= t && t < prefix[v1 + 1])) {  // largest v1 with prefix[v1] <= t
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
          const uint32_t mid = (lo + hi) >> 1;
          if (prefix[mid] <= t) lo = mid; else hi = mid;
        }
        v1 = lo;
      }
      const uint32_t j = (uint32_t)(t - prefix[v1]);
      const uint32_t* N1 = nbr + off[v1];
      const uint32_t v2 = N1[j];
      const uint32_t b2 = (uint32_t)(prefix[v2 + 1] - prefix[v2]);  // neighbours of v2 below v2
      acc += warp_intersect<kCountOnly>(N1, j, nbr + off[v2], b2, nullptr, 8);
    }
  }
  if (lane == 0 && acc) atomicAdd(&scratch[1], acc);
}

__global__ void k_na_store(const unsigned long long* scratch, uint64_t* out) { *out = scratch[1]; }

}  // namespace

extern "C" gpm_status gpm_count_triangles_noalloc(const int64_t* offsets_dev,
                                                  const uint32_t* nbrs_dev, uint32_t n,
                                                  uint64_t* count_dev, void* stream) {
  // nbrs_dev may be NULL for a graph without edges (offsets all zero): no
  // neighbour is ever read then
  if (!offsets_dev || !count_dev)
    return api_fail(GPM_E_INVALID_ARG, "gpm_count_triangles_noalloc: NULL argument");
  if ((uint64_t)n > kMaxVertices)
    return api_fail(GPM_E_INVALID_ARG,
                    "gpm_count_triangles_noalloc: the graph has " + std::to_string(n) +
                        " vertices; the allocation-free path holds at most " +
                        std::to_string(kMaxVertices));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return api_fail(GPM_E_CUDA, std::string("gpm_count_triangles_noalloc: no usable device: ") +
                                    cudaGetErrorString(e));
  unsigned long long* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess)
        return api_fail(GPM_E_CUDA, std::string("gpm_count_triangles_noalloc: set-up failed: ") +
                                        cudaGetErrorString(e));
      g_addr[dev] = static_cast<unsigned long long*>(p);
    }
    scratch = g_addr[dev];
  }
  int sms = 0;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess)
    return api_fail(GPM_E_CUDA, std::string("gpm_count_triangles_noalloc: ") + cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned vblocks = std::max(1u, std::min<unsigned>((n + 255) / 256, (unsigned)sms * 8u));
  k_na_lower<<<vblocks, 256, 0, s>>>(offsets_dev, nbrs_dev, n, scratch);
  k_na_scan<<<1, 1024, 0, s>>>(n, scratch);
  if (n) k_na_triangles<<<(unsigned)sms * 8u, 256, 0, s>>>(offsets_dev, nbrs_dev, n, scratch);
  k_na_store<<<1, 1, 0, s>>>(scratch, count_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return api_fail(GPM_E_CUDA, std::string("gpm_count_triangles_noalloc: launch: ") +
                                    cudaGetErrorString(e));
  return GPM_OK;
}
