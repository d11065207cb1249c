// enum_clique.cu — k-clique counting / listing on the degree-oriented DAG.
//
// Orientation (Section 4.2) gives every clique exactly one topological order
// c1 -> c2 -> ... -> ck, so each clique is found once with no symmetry checks
// at run time.  Root task = arc (c1, c2); the candidates for c3 are
// W = N+(c1) ∩ N+(c2) (buffered, Algorithm 1's W); level by level the
// candidates shrink by intersecting with the out-list of the vertex just
// matched.  The last level is counted without materialising it (Section 6.1
// set operations in count mode).  A level whose candidate set is smaller than
// the number of vertices still to match is skipped (it holds no clique).
#include "enum_common.cuh"

namespace gpm {
namespace {

template <int K, int D, bool LIST>
__device__ __forceinline__ unsigned long long clique_rec(const EnumArgs& a, const uint32_t* C,
                                                         uint32_t s, const Bufs& B, int lvl,
                                                         uint32_t (&path)[K]) {
  if constexpr (D == K - 1) {
    if constexpr (LIST) emit_set<K>(a, path, K - 1, C, s);
    return s;
  } else {
    if (s < (uint32_t)(K - D)) return 0;
    unsigned long long total = 0;
    for (uint32_t i = 0; i < s; i++) {
      const uint32_t w = C[i];
      const uint32_t* Nw = row_of(a.g, w);
      const uint32_t dw = deg_of(a.g, w);
      if constexpr (D == K - 2 && !LIST) {
        total += isect<kCountOnly>(a, C, s, Nw, dw, nullptr);
      } else {
        uint32_t* next = B.level(lvl);
        const uint32_t s2 = isect<kWrite>(a, C, s, Nw, dw, next);
        __syncwarp();
        path[D] = w;
        total += clique_rec<K, D + 1, LIST>(a, next, s2, B, lvl + 1, path);
        __syncwarp();
      }
    }
    return total;
  }
}

template <int K, bool LIST>
struct CliquePlan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t u,
                                                           uint32_t v, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t* Nu = row_of(a.g, u);
    const uint32_t* Nv = row_of(a.g, v);
    const uint32_t du = deg_of(a.g, u), dv = deg_of(a.g, v);
    if constexpr (K == 3 && !LIST) {
      return isect<kCountOnly>(a, Nu, du, Nv, dv, nullptr);
    } else {
      const Bufs B = pick_bufs(a, sbuf, gbuf, min(du, dv));
      uint32_t* W = B.level(0);
      const uint32_t s = isect<kWrite>(a, Nu, du, Nv, dv, W);
      __syncwarp();
      uint32_t path[K];
#pragma unroll
      for (int q = 0; q < K; q++) path[q] = 0;
      path[0] = u;
      path[1] = v;
      const unsigned long long r = clique_rec<K, 2, LIST>(a, W, s, B, 1, path);
      __syncwarp();
      return r;
    }
  }
};

template <int K, bool LIST>
__global__ void __launch_bounds__(256) k_clique(EnumArgs a) {
  task_loop<CliquePlan<K, LIST>>(a);
}

template <int K, bool LIST>
cudaError_t launch_k(const EnumArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
  auto kern = k_clique<K, LIST>;
  if (smem > 40 * 1024) {  // static smem adds to the dynamic slab
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <int K, bool LIST>
cudaError_t occ_k(int threads, size_t smem, int* blocks, int* regs) {
  auto kern = k_clique<K, LIST>;
  if (smem > 40 * 1024) {  // static smem adds to the dynamic slab
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, kern);
  if (e != cudaSuccess) return e;
  *regs = at.numRegs;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, threads, smem);
}

}  // namespace

cudaError_t launch_clique(int k, bool list, const EnumArgs& a, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t s) {
#define GPM_CASE(KK)                                                          \
  case KK:                                                                    \
    return list ? launch_k<KK, true>(a, grid, block, smem, s)                 \
                : launch_k<KK, false>(a, grid, block, smem, s);
  switch (k) {
    GPM_CASE(3) GPM_CASE(4) GPM_CASE(5) GPM_CASE(6) GPM_CASE(7) GPM_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef GPM_CASE
}

cudaError_t occupancy_clique(int k, bool list, int threads, size_t smem, int* blocks, int* regs) {
#define GPM_CASE(KK)                                                                   \
  case KK:                                                                             \
    return list ? occ_k<KK, true>(threads, smem, blocks, regs)                         \
                : occ_k<KK, false>(threads, smem, blocks, regs);
  switch (k) {
    GPM_CASE(3) GPM_CASE(4) GPM_CASE(5) GPM_CASE(6) GPM_CASE(7) GPM_CASE(8)
    default: return cudaErrorInvalidValue;
  }
#undef GPM_CASE
}

}  // namespace gpm
