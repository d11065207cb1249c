// enum_generic.cu — the generic interpreter for any connected pattern of 3..8
// vertices (Sections 4.2, 5.1, 6.1): the search plan of a GenTable run as a
// warp-cooperative DFS over the root tasks.
//
// Positions 0 and 1 are the root task (an edge).  The candidates of a later
// position t are
//   C_t = ∩_{s in E[t]} N(v_s) ∩ [0, min_{s in U[t]} v_s)      (connectivity,
//         − ∪_{s in N[t]} N(v_s)   (vertex-induced only)        symmetry order)
//         − {v_s : s in N[t]}                                  (distinct vertices)
// The intersection starts from the shortest neighbour list, bounded by set
// bounding (Section 6.1); further lists are intersected, then (induced) the
// non-neighbours' lists subtracted, ping-ponging between two per-warp buffers
// so no operation writes its own input.  A set that needs no operation is the
// neighbour-list prefix itself (no copy).  Matched vertices that fall in a set
// are skipped while iterating, and subtracted after counting.  The last
// position is only counted (the last operation counts), or listed.
//
// Buffers: positions 2..k-1 each own one level, plus one scratch level; a
// set never exceeds the largest degree, so the levels live in shared memory
// when the maximum degree fits the slab and in the warp's HBM slice otherwise.
#include "enum_common.cuh"

namespace gpm {

namespace {

// Single-lane test: does y belong to the candidate set of position t?
__device__ __forceinline__ bool gen_member(const DevCsr& g, const GenTable& T, int t,
                                           const uint32_t* m, uint32_t ub, uint32_t y) {
  if (y >= ub) return false;
  for (int i = 0; i < T.nE[t]; i++) {
    const uint32_t v = m[T.E[t][i]];
    if (!lane_contains(row_of(g, v), deg_of(g, v), y)) return false;
  }
  if (T.induced)
    for (int i = 0; i < T.nN[t]; i++) {
      const uint32_t v = m[T.N[t][i]];
      if (lane_contains(row_of(g, v), deg_of(g, v), y)) return false;
    }
  return true;
}

__device__ __forceinline__ uint32_t gen_bound(const GenTable& T, int t, const uint32_t* m) {
  uint32_t ub = kNone;
  for (int i = 0; i < T.nU[t]; i++) ub = min(ub, m[T.U[t][i]]);
  return ub;
}

// The candidate set of position t (before removing matched vertices).
// COUNT: its size only.  Else *out = its elements (a neighbour-list prefix or
// dst), returns the size.
template <bool COUNT>
__device__ __forceinline__ uint32_t gen_set(const EnumArgs& a, const GenTable& T, int t,
                                            const uint32_t* m, uint32_t ub, uint32_t* dst,
                                            uint32_t* tmp, const uint32_t** out) {
  const DevCsr& g = a.g;
  const int nE = T.nE[t];
  int bi = 0;
  uint32_t bd = deg_of(g, m[T.E[t][0]]);
  for (int i = 1; i < nE; i++) {
    const uint32_t d = deg_of(g, m[T.E[t][i]]);
    if (d < bd) { bd = d; bi = i; }
  }
  const uint32_t* cur = row_of(g, m[T.E[t][bi]]);
  uint32_t n = (ub != kNone) ? warp_count_less(cur, bd, ub) : bd;
  const int ops = (nE - 1) + (T.induced ? (int)T.nN[t] : 0);
  if (ops == 0) {
    if (!COUNT) *out = cur;
    return n;
  }
  // the last written result must land in dst: the first write goes to dst
  // when the number of writes is odd
  const int writes = COUNT ? ops - 1 : ops;
  uint32_t* buf[2] = {(writes & 1) ? dst : tmp, (writes & 1) ? tmp : dst};
  int op = 0, wi = 0;
  for (int i = 0; i < nE; i++) {
    if (i == bi) continue;
    const uint32_t v = m[T.E[t][i]];
    if (COUNT && ++op == ops) return isect<kCountOnly>(a, cur, n, row_of(g, v), deg_of(g, v), nullptr);
    if (!COUNT) ++op;
    uint32_t* o = buf[wi++ & 1];
    n = isect<kWrite>(a, cur, n, row_of(g, v), deg_of(g, v), o);
    __syncwarp();
    cur = o;
  }
  if (T.induced)
    for (int i = 0; i < T.nN[t]; i++) {
      const uint32_t v = m[T.N[t][i]];
      if (COUNT && ++op == ops) return diff<kCountOnly>(a, cur, n, row_of(g, v), deg_of(g, v), nullptr);
      if (!COUNT) ++op;
      uint32_t* o = buf[wi++ & 1];
      n = diff<kWrite>(a, cur, n, row_of(g, v), deg_of(g, v), o);
      __syncwarp();
      cur = o;
    }
  if (!COUNT) *out = cur;
  return n;
}

// Is x one of the matched vertices position t must avoid?  (warp-uniform)
__device__ __forceinline__ bool gen_taken(const GenTable& T, int t, const uint32_t* m, uint32_t x) {
  bool hit = false;
  for (int i = 0; i < T.nN[t]; i++) hit |= m[T.N[t][i]] == x;
  return hit;
}

// Emit m[0, t) plus every x of C[0, n) not taken, in pattern-vertex order.
__device__ __forceinline__ void gen_emit(const EnumArgs& a, const GenTable& T, int t,
                                         const uint32_t* m, const uint32_t* C, uint32_t n) {
  uint32_t c = 0;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane_id();
    const bool keep = i < n && !gen_taken(T, t, m, C[i]);
    c += __popc(__ballot_sync(kFull, keep));
  }
  if (c == 0) return;
  const unsigned long long b0 = list_reserve(a, c);
  uint32_t w = 0;
  for (uint32_t base = 0; base < n; base += 32) {
    const uint32_t i = base + lane_id();
    const uint32_t x = (i < n) ? C[i] : kNone;
    const bool keep = i < n && !gen_taken(T, t, m, x);
    const unsigned msk = __ballot_sync(kFull, keep);
    if (keep) {
      const unsigned long long slot = b0 + w + __popc(msk & lanemask_lt());
      if (slot < a.list_cap) {
        uint32_t* o = a.list_out + slot * T.k;
        for (int q = 0; q < t; q++) o[T.order[q]] = m[q];
        o[T.order[t]] = x;
      }
    }
    w += __popc(msk);
  }
}

template <bool LIST>
struct GenericPlan {
  static __device__ __forceinline__ unsigned long long run(const EnumArgs& a, uint32_t v1,
                                                           uint32_t v2, uint32_t* sbuf,
                                                           uint32_t* gbuf) {
    const GenTable& T = *a.gen;
    const int k = (int)T.k, last = k - 1;
    const Bufs B = a.gcap ? Bufs{gbuf, a.gcap, a.gcap} : Bufs{sbuf, a.scap, a.scap};
    uint32_t* scratch = B.level(k - 2);
    uint32_t m[kGenMaxK];
    m[0] = v1;
    m[1] = v2;
    unsigned long long total = 0;
    const uint32_t* cp[kGenMaxK];
    uint32_t cn[kGenMaxK], ci[kGenMaxK];
    int t = 2;
    for (;;) {
      if (t == last) {
        // the last position: count (or list) its candidates
        const uint32_t ub = gen_bound(T, t, m);
        if constexpr (LIST) {
          const uint32_t* C = nullptr;
          const uint32_t n = gen_set<false>(a, T, t, m, ub, B.level(t - 2), scratch, &C);
          __syncwarp();
          gen_emit(a, T, t, m, C, n);
          uint32_t taken = 0;
          for (uint32_t i = lane_id(); i < n; i += 32) taken += gen_taken(T, t, m, C[i]) ? 1u : 0u;
          total += n - __reduce_add_sync(kFull, taken);
        } else {
          uint32_t c = gen_set<true>(a, T, t, m, ub, B.level(t - 2), scratch, nullptr);
          uint32_t taken = 0;
          if (lane_id() == 0)
            for (int i = 0; i < T.nN[t]; i++) taken += gen_member(a.g, T, t, m, ub, m[T.N[t][i]]) ? 1u : 0u;
          c -= __shfl_sync(kFull, taken, 0);
          total += c;
        }
        __syncwarp();
        t--;
        if (t < 2) break;
      } else {
        // a fresh position: materialise its candidates
        cn[t] = gen_set<false>(a, T, t, m, gen_bound(T, t, m), B.level(t - 2), scratch, &cp[t]);
        ci[t] = 0;
        __syncwarp();
      }
      // advance the deepest open position to its next candidate
      for (;;) {
        if (ci[t] < cn[t]) {
          const uint32_t x = cp[t][ci[t]++];
          if (gen_taken(T, t, m, x)) continue;
          m[t] = x;
          t++;
          break;
        }
        t--;
        if (t < 2) break;
      }
      if (t < 2) break;
    }
    return total;
  }
};

template <bool LIST>
__global__ void __launch_bounds__(256) k_generic(EnumArgs a) {
  task_loop<GenericPlan<LIST>>(a);
}

}  // namespace

cudaError_t launch_generic(bool list, const EnumArgs& a, dim3 grid, dim3 block, size_t smem,
                           cudaStream_t s) {
  auto kern = list ? k_generic<true> : k_generic<false>;
  if (smem > 40 * 1024) {  // static smem adds to the dynamic slab
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  kern<<<grid, block, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t occupancy_generic(bool list, int threads, size_t smem, int* blocks, int* regs) {
  auto kern = list ? k_generic<true> : k_generic<false>;
  if (smem > 40 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, kern);
  if (e != cudaSuccess) return e;
  *regs = at.numRegs;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, threads, smem);
}

}  // namespace gpm
