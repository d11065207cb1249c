// enum_small.cu — plans for the non-clique patterns on the undirected CSR.
//
// Each plan is a matching order plus a symmetry order (Section 2.2) written
// as nested warp-cooperative set operations (Sections 5.1, 6.1).  Vertex-
// induced variants subtract the neighbour lists of pattern non-neighbours
// (set difference); edge-induced variants do not.  Counting-only forms
// (Section 5.4 (1)) replace the innermost enumeration by its size where the
// innermost set is a plain prefix or a C(n, 2) choice.
//
//  diamond          task (v1, v2), v1 > v2 = the chord; W = N(v1) ∩ N(v2);
//                   v3 > v4 in W (Algorithm 1).  Edge-induced counting uses
//                   C(|W|, 2) per task (Algorithm 3); vertex-induced keeps
//                   v4 in W[0, i) − N(v3) for v3 = W[i].
//  4-cycle          task (v1, v2), v1 > v2, v1 the largest vertex; v4 in
//                   N(v1) ∩ [0, v2); v3 in N(v2) ∩ N(v4) ∩ [0, v1).  Induced:
//                   v4 not in N(v2), v3 not in N(v1).
//  tailed-triangle  task (v1, v2) in both directions, v1 the degree-3 vertex;
//                   v3 in N(v1) ∩ N(v2) ∩ [0, v2); tail v4 in N(v1) − {v2, v3}
//                   (induced: v4 in N(v1) − N(v2) − N(v3)).
//  3-star           task (v1, v2) in both directions, v1 the centre, v2 the
//                   largest leaf; v3 > v4 in N(v1) ∩ [0, v2) (induced: the
//                   leaves pairwise non-adjacent).
//  4-path           task (v1, v2), v1 > v2 the middle edge; v3 in N(v1) − {v2},
//                   v4 in N(v2) − {v1, v3} (induced: v3 not in N(v2), v4 not in
//                   N(v1) ∪ N(v3)).
//  wedge            task (v1, v2) in both directions, v1 the centre; v3 in
//                   N(v1) ∩ [0, v2) (induced: v3 not in N(v2)).
#include "enum_common.cuh"

namespace gpm {

// Copy A[0, n) without x1 and x2 to out (may alias A: in-place compaction is
// safe because every lane reads its element before the ballot).
__device__ __forceinline__ uint32_t warp_copy_without(const uint32_t* A, uint32_t n, uint32_t x1,
                                                      uint32_t x2, uint32_t* out) {
  uint32_t total = 0;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane_id();
    const uint32_t x = (i < n) ? A[i] : kNone;
    const bool keep = i < n && x != x1 && x != x2;
    const unsigned m = __ballot_sync(kFull, keep);
    if (keep) out[total + __popc(m & lanemask_lt())] = x;
    total += __popc(m);
  }
  return total;
}

// Emit fixed[] with slot `slot` taking every x in R[0, n) except ex1, ex2.
template <int K>
__device__ __forceinline__ void emit_row_without(const EnumArgs& a, const uint32_t (&fixed)[K],
                                                 int slot, const uint32_t* R, uint32_t n,
                                                 uint32_t ex1, uint32_t ex2) {
  uint32_t c = 0;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane_id();
    const bool keep = i < n && R[i] != ex1 && R[i] != ex2;
    c += __popc(__ballot_sync(kFull, keep));
  }
  if (c == 0) return;
  const unsigned long long b0 = list_reserve(a, c);
  uint32_t w = 0;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane_id();
    const uint32_t x = (i < n) ? R[i] : kNone;
    const bool keep = i < n && x != ex1 && x != ex2;
    const unsigned m = __ballot_sync(kFull, keep);
    if (keep) {
      const unsigned long long slotidx = b0 + w + __popc(m & lanemask_lt());
      if (slotidx < a.list_cap) {
        uint32_t* o = a.list_out + slotidx * K;
#pragma unroll
        for (int q = 0; q < K; q++) o[q] = (q == slot) ? x : fixed[q];
      }
    }
    w += __popc(m);
  }
}

namespace {

__device__ __forceinline__ unsigned long long choose2(unsigned long long n) {
  return n ? n * (n - 1) / 2 : 0;
}

// ------------------------------------------------------------------ diamond
template <bool INDUCED, bool LIST, bool CO>
struct DiamondPlan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t *N1 = row_of(a.g, v1), *N2 = row_of(a.g, v2);
    const uint32_t d1 = deg_of(a.g, v1), d2 = deg_of(a.g, v2);
    if constexpr (CO && !INDUCED && !LIST) {
      // Algorithm 3: n = |N(v1) ∩ N(v2)| triangles on the edge, C(n, 2) diamonds
      return choose2(isect<kCountOnly>(a, N1, d1, N2, d2, nullptr));
    } else {
      const Bufs B = pick_bufs(a, sbuf, gbuf, max(d1, d2));
      uint32_t* W = B.level(0);
      const uint32_t s = isect<kWrite>(a, N1, d1, N2, d2, W);
      __syncwarp();
      unsigned long long total = 0;
      for (uint32_t i = 1; i < s; i++) {  // v3 = W[i], v4 in W[0, i)
        const uint32_t v3 = W[i];
        if constexpr (INDUCED) {
          const uint32_t *N3 = row_of(a.g, v3);
          const uint32_t d3 = deg_of(a.g, v3);
          if constexpr (LIST) {
            uint32_t* X = B.level(1);
            const uint32_t c = diff<kWrite>(a, W, i, N3, d3, X);
            __syncwarp();
            const uint32_t f[4] = {v1, v2, v3, 0};
            emit_set<4>(a, f, 3, X, c);
            __syncwarp();
            total += c;
          } else {
            total += diff<kCountOnly>(a, W, i, N3, d3, nullptr);
          }
        } else {
          // Algorithm 1: every v4 < v3 in W
          if constexpr (LIST) {
            const uint32_t f[4] = {v1, v2, v3, 0};
            emit_set<4>(a, f, 3, W, i);
          }
          total += i;
        }
      }
      __syncwarp();
      return total;
    }
  }
};

// ------------------------------------------------------------------ 4-cycle
template <bool INDUCED, bool LIST>
struct Cycle4Plan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t *N1 = row_of(a.g, v1), *N2 = row_of(a.g, v2);
    const uint32_t d1 = deg_of(a.g, v1), d2 = deg_of(a.g, v2);
    const uint32_t p4 = warp_count_less(N1, d1, v2);  // v4 in N(v1) ∩ [0, v2)
    const uint32_t b2 = warp_count_less(N2, d2, v1);  // v3 in N(v2) ∩ [0, v1)
    if (p4 == 0 || b2 == 0) return 0;
    const Bufs B = pick_bufs(a, sbuf, gbuf, max(d1, d2));
    const uint32_t* A4 = N1;
    uint32_t na4 = p4;
    const uint32_t* B2 = N2;
    uint32_t nb2 = b2;
    int lv = 0;
    if constexpr (INDUCED) {
      uint32_t* x = B.level(lv++);
      na4 = diff<kWrite>(a, N1, p4, N2, d2, x);  // v4 not adjacent to v2
      A4 = x;
      uint32_t* y = B.level(lv++);
      nb2 = diff<kWrite>(a, N2, b2, N1, d1, y);  // v3 not adjacent to v1
      B2 = y;
      __syncwarp();
    }
    unsigned long long total = 0;
    for (uint32_t i = 0; i < na4; i++) {
      const uint32_t v4 = A4[i];
      const uint32_t* N4 = row_of(a.g, v4);
      const uint32_t b4 = warp_count_less(N4, deg_of(a.g, v4), v1);
      if constexpr (LIST) {
        uint32_t* S = B.level(lv);
        const uint32_t c = isect<kWrite>(a, B2, nb2, N4, b4, S);
        __syncwarp();
        const uint32_t f[4] = {v1, v2, 0, v4};
        emit_set<4>(a, f, 2, S, c);
        __syncwarp();
        total += c;
      } else {
        total += isect<kCountOnly>(a, B2, nb2, N4, b4, nullptr);
      }
    }
    __syncwarp();
    return total;
  }
};

// ---------------------------------------------------------- tailed triangle
template <bool INDUCED, bool LIST>
struct TailedTrianglePlan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t *N1 = row_of(a.g, v1), *N2 = row_of(a.g, v2);
    const uint32_t d1 = deg_of(a.g, v1), d2 = deg_of(a.g, v2);
    if (d1 < 3) return 0;
    const uint32_t a1 = warp_count_less(N1, d1, v2);
    const uint32_t a2 = warp_count_less(N2, d2, v2);
    if constexpr (!INDUCED && !LIST) {
      // counting-only: each triangle (v1, v2, v3 < v2) has d(v1) - 2 tails
      const uint32_t t = isect<kCountOnly>(a, N1, a1, N2, a2, nullptr);
      return (unsigned long long)t * (d1 - 2);
    } else {
      const Bufs B = pick_bufs(a, sbuf, gbuf, max(d1, d2));
      uint32_t* W = B.level(0);
      const uint32_t s = isect<kWrite>(a, N1, a1, N2, a2, W);
      __syncwarp();
      if (s == 0) return 0;
      unsigned long long total = 0;
      if constexpr (!INDUCED) {
        for (uint32_t i = 0; i < s; i++) {
          const uint32_t v3 = W[i];
          const uint32_t f[4] = {v1, v2, v3, 0};
          emit_row_without<4>(a, f, 3, N1, d1, v2, v3);
          total += d1 - 2;
        }
      } else {
        // D = N(v1) − N(v2): v2 itself is removed by − N(v3) below (v3 ~ v2)
        uint32_t* D = B.level(1);
        const uint32_t nd = diff<kWrite>(a, N1, d1, N2, d2, D);
        __syncwarp();
        for (uint32_t i = 0; i < s; i++) {
          const uint32_t v3 = W[i];
          const uint32_t *N3 = row_of(a.g, v3);
          const uint32_t d3 = deg_of(a.g, v3);
          if constexpr (LIST) {
            uint32_t* X = B.level(2);
            const uint32_t c = diff<kWrite>(a, D, nd, N3, d3, X);
            __syncwarp();
            const uint32_t f[4] = {v1, v2, v3, 0};
            emit_set<4>(a, f, 3, X, c);
            __syncwarp();
            total += c;
          } else {
            total += diff<kCountOnly>(a, D, nd, N3, d3, nullptr);
          }
        }
      }
      __syncwarp();
      return total;
    }
  }
};

// ------------------------------------------------------------------- 3-star
template <bool INDUCED, bool LIST>
struct Star3Plan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t *N1 = row_of(a.g, v1), *N2 = row_of(a.g, v2);
    const uint32_t d1 = deg_of(a.g, v1), d2 = deg_of(a.g, v2);
    const uint32_t p = warp_count_less(N1, d1, v2);  // leaves below v2
    if (p < 2) return 0;
    if constexpr (!INDUCED) {
      if constexpr (LIST) {
        for (uint32_t i = 1; i < p; i++) {
          const uint32_t f[4] = {v1, v2, N1[i], 0};
          emit_set<4>(a, f, 3, N1, i);
        }
      }
      return choose2(p);
    } else {
      const Bufs B = pick_bufs(a, sbuf, gbuf, max(d1, d2));
      uint32_t* A = B.level(0);
      const uint32_t s = diff<kWrite>(a, N1, p, N2, d2, A);  // leaves ≁ v2
      __syncwarp();
      unsigned long long total = 0;
      for (uint32_t i = 1; i < s; i++) {
        const uint32_t v3 = A[i];
        const uint32_t *N3 = row_of(a.g, v3);
        const uint32_t d3 = deg_of(a.g, v3);
        if constexpr (LIST) {
          uint32_t* X = B.level(1);
          const uint32_t c = diff<kWrite>(a, A, i, N3, d3, X);
          __syncwarp();
          const uint32_t f[4] = {v1, v2, v3, 0};
          emit_set<4>(a, f, 3, X, c);
          __syncwarp();
          total += c;
        } else {
          total += diff<kCountOnly>(a, A, i, N3, d3, nullptr);
        }
      }
      __syncwarp();
      return total;
    }
  }
};

// ------------------------------------------------------------------- 4-path
template <bool INDUCED, bool LIST>
struct Path4Plan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t *N1 = row_of(a.g, v1), *N2 = row_of(a.g, v2);
    const uint32_t d1 = deg_of(a.g, v1), d2 = deg_of(a.g, v2);
    if constexpr (!INDUCED) {
      if constexpr (!LIST) {
        // counting-only: (d1-1)(d2-1) end pairs minus the triangles (v3 = v4)
        const uint32_t t = isect<kCountOnly>(a, N1, d1, N2, d2, nullptr);
        return (unsigned long long)(d1 - 1) * (d2 - 1) - t;
      } else {
        unsigned long long total = 0;
        for (uint32_t i = 0; i < d1; i++) {
          const uint32_t v3 = N1[i];
          if (v3 == v2) continue;
          const uint32_t f[4] = {v1, v2, v3, 0};
          emit_row_without<4>(a, f, 3, N2, d2, v1, v3);
          total += d2 - 1 - (lane_contains(N2, d2, v3) ? 1u : 0u);
        }
        return total;
      }
    } else {
      const Bufs B = pick_bufs(a, sbuf, gbuf, max(d1, d2));
      uint32_t* A = B.level(0);
      uint32_t na = diff<kWrite>(a, N1, d1, N2, d2, A);
      __syncwarp();
      na = warp_copy_without(A, na, v2, kNone, A);  // v3 ≠ v2
      uint32_t* D = B.level(1);
      uint32_t nd = diff<kWrite>(a, N2, d2, N1, d1, D);
      __syncwarp();
      nd = warp_copy_without(D, nd, v1, kNone, D);  // v4 ≠ v1
      __syncwarp();
      unsigned long long total = 0;
      for (uint32_t i = 0; i < na; i++) {
        const uint32_t v3 = A[i];
        const uint32_t *N3 = row_of(a.g, v3);
        const uint32_t d3 = deg_of(a.g, v3);
        if constexpr (LIST) {
          uint32_t* X = B.level(2);
          const uint32_t c = diff<kWrite>(a, D, nd, N3, d3, X);
          __syncwarp();
          const uint32_t f[4] = {v1, v2, v3, 0};
          emit_set<4>(a, f, 3, X, c);
          __syncwarp();
          total += c;
        } else {
          total += diff<kCountOnly>(a, D, nd, N3, d3, nullptr);
        }
      }
      __syncwarp();
      return total;
    }
  }
};

// -------------------------------------------------------------------- wedge
template <bool INDUCED, bool LIST>
struct WedgePlan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const uint32_t *N1 = row_of(a.g, v1), *N2 = row_of(a.g, v2);
    const uint32_t d1 = deg_of(a.g, v1), d2 = deg_of(a.g, v2);
    const uint32_t p = warp_count_less(N1, d1, v2);
    if (p == 0) return 0;
    if constexpr (!INDUCED) {
      if constexpr (LIST) {
        const uint32_t f[3] = {v1, v2, 0};
        emit_set<3>(a, f, 2, N1, p);
      }
      return p;
    } else {
      if constexpr (LIST) {
        const Bufs B = pick_bufs(a, sbuf, gbuf, max(d1, d2));
        uint32_t* X = B.level(0);
        const uint32_t c = diff<kWrite>(a, N1, p, N2, d2, X);
        __syncwarp();
        const uint32_t f[3] = {v1, v2, 0};
        emit_set<3>(a, f, 2, X, c);
        __syncwarp();
        return c;
      } else {
        return diff<kCountOnly>(a, N1, p, N2, d2, nullptr);
      }
    }
  }
};

template <class Plan>
__global__ void __launch_bounds__(256) k_enum(EnumArgs a) {
  task_loop<Plan>(a);
}

template <class Plan>
cudaError_t launch_plan(const EnumArgs& a, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
  auto kern = k_enum<Plan>;
  if (smem > 40 * 1024) {  // static smem adds to the dynamic slab
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

template <class Plan>
cudaError_t occ_plan(int threads, size_t smem, int* blocks, int* regs) {
  auto kern = k_enum<Plan>;
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

// Dispatch on (family, induced, list, count_only) to a Plan type and apply F.
template <template <class> class F, class... Args>
cudaError_t dispatch(int family, bool induced, bool list, bool co, Args... args) {
#define GPM_IL(PLAN)                                                               \
  if (induced) return list ? F<PLAN<true, true>>::go(args...) : F<PLAN<true, false>>::go(args...); \
  return list ? F<PLAN<false, true>>::go(args...) : F<PLAN<false, false>>::go(args...);
  switch (family) {
    case kDiamond:
      if (induced)
        return list ? F<DiamondPlan<true, true, false>>::go(args...)
                    : F<DiamondPlan<true, false, false>>::go(args...);
      if (list) return F<DiamondPlan<false, true, false>>::go(args...);
      return co ? F<DiamondPlan<false, false, true>>::go(args...)
                : F<DiamondPlan<false, false, false>>::go(args...);
    case kCycle4: { GPM_IL(Cycle4Plan) }
    case kTailedTriangle: { GPM_IL(TailedTrianglePlan) }
    case kStar3: { GPM_IL(Star3Plan) }
    case kPath4: { GPM_IL(Path4Plan) }
    case kWedge: { GPM_IL(WedgePlan) }
    default: return cudaErrorInvalidValue;
  }
#undef GPM_IL
}

template <class Plan>
struct LaunchF {
  static cudaError_t go(const EnumArgs* a, dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
    return launch_plan<Plan>(*a, grid, block, smem, s);
  }
};
template <class Plan>
struct OccF {
  static cudaError_t go(int threads, size_t smem, int* blocks, int* regs) {
    return occ_plan<Plan>(threads, smem, blocks, regs);
  }
};

}  // namespace

cudaError_t launch_small(int family, bool induced, bool list, bool co, const EnumArgs& a,
                         dim3 grid, dim3 block, size_t smem, cudaStream_t s) {
  return dispatch<LaunchF>(family, induced, list, co, &a, grid, block, smem, s);
}

cudaError_t occupancy_small(int family, bool induced, bool list, bool co, int threads, size_t smem,
                            int* blocks, int* regs) {
  return dispatch<OccF>(family, induced, list, co, threads, smem, blocks, regs);
}

}  // namespace gpm
