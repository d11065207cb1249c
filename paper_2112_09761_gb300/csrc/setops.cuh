// setops.cuh — warp-cooperative sorted-set primitives (Section 6.1).
//
// Every primitive is called by all 32 lanes of a warp with warp-uniform
// arguments and returns a warp-uniform result.  Sets are strictly ascending
// uint32 arrays in global or shared memory (generic pointers).  Vertex IDs are
// below 0xFFFFFFFF, which serves as the "past the end" sentinel.
//
// Intersection C = A ∩ B has two variants, picked by the length ratio:
//   * binary search (the paper's choice, after TriCore): each lane takes
//     elements of the shorter list and searches the longer one; the top five
//     levels of the search run on 32 evenly spaced pivots of the longer list
//     held one per lane and read with shuffles (the register analogue of the
//     paper's scratchpad-cached top of the search tree);
//   * chunked merge: both lists advance in 32-element chunks held in
//     registers; each A-lane finds its element in the current B chunk with a
//     5-step shuffle search; the chunk with the smaller last element advances
//     (merge path at chunk granularity).  Loads are fully coalesced.
// Outputs are compacted with __ballot_sync / __popc in ascending order.
// Set difference C = A − B and set bounding {x in A : x < y} follow the same
// scheme (Section 6.1).
#pragma once
#include <cstdint>

namespace gpm {

constexpr unsigned kFull = 0xffffffffu;
constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Number of elements of sorted A[0, n) that are < key (set bounding, Section
// 6.1).  32-ary search: each round probes 32 interior positions with one
// gathered load and narrows the range ~33x.
__device__ __forceinline__ uint32_t warp_count_less(const uint32_t* __restrict__ A, uint32_t n,
                                                    uint32_t key) {
  const uint32_t lane = lane_id();
  uint32_t lo = 0, hi = n;
  while (hi - lo > 32) {
    const uint64_t span = hi - lo;
    const uint32_t idx = lo + (uint32_t)((span * (lane + 1)) / 33);
    const unsigned m = __ballot_sync(kFull, A[idx] < key);
    const uint32_t c = __popc(m);  // probes below key form a prefix
    const uint32_t nlo = c ? lo + (uint32_t)((span * c) / 33) + 1 : lo;
    const uint32_t nhi = (c < 32) ? lo + (uint32_t)((span * (c + 1)) / 33) : hi;
    lo = nlo;
    hi = nhi;
  }
  const bool lt = (lo + lane < hi) && (A[lo + lane] < key);
  return lo + __popc(__ballot_sync(kFull, lt));
}

// Is `key` present in A[0, n)?  Single-lane sequential binary search.
__device__ __forceinline__ bool lane_contains(const uint32_t* __restrict__ A, uint32_t n,
                                              uint32_t key) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    const uint32_t x = A[mid];
    if (x == key) return true;
    if (x < key) lo = mid + 1; else hi = mid;
  }
  return false;
}

// Does the 32-element sorted chunk held one-per-lane in `b` (kNone-padded)
// contain `key`?  5 shuffles; every lane must call it.
__device__ __forceinline__ bool chunk_contains(uint32_t b, uint32_t key) {
  int j = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t p = __shfl_sync(kFull, b, j + step - 1);
    if (p < key) j += step;
  }
  return __shfl_sync(kFull, b, j) == key;
}

// Membership flags of a[lane] in B via binary search with a register-cached
// top level.  `piv` is B[(j*nb)>>5] for lane j (nb > 32).
__device__ __forceinline__ bool pivot_search(const uint32_t* __restrict__ B, uint32_t nb, uint32_t piv,
                                             uint32_t key) {
  // largest j with piv_j <= key (piv_0 = B[0]); 5 shuffles
  int j = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const uint32_t p = __shfl_sync(kFull, piv, j + step);
    if (j + step < 32 && p <= key) j += step;
  }
  const uint32_t s = (uint32_t)(((uint64_t)j * nb) >> 5);
  const uint32_t e = (uint32_t)(((uint64_t)(j + 1) * nb) >> 5);
  return lane_contains(B + s, e - s, key);
}

// Mode of a set operation's result.
enum SetOut { kCountOnly = 0, kWrite = 1 };
// Which elements of A to keep: those in B (intersection) or not (difference).
enum SetOp { kIntersect = 0, kDifference = 1 };

// Core A∘B where each lane owns A's elements (binary-search variant).  Keeps
// a in A iff (a in B) == (OP == kIntersect).  Writes kept elements to out in
// order when OUT == kWrite.  Returns the kept count.
template <SetOp OP, SetOut OUT>
__device__ __forceinline__ uint32_t warp_setop_bsearch(const uint32_t* __restrict__ A, uint32_t na,
                                                       const uint32_t* __restrict__ B, uint32_t nb,
                                                       uint32_t* __restrict__ out) {
  const uint32_t lane = lane_id();
  uint32_t piv = 0;
  const bool pivots = nb > 32;
  if (pivots) piv = B[(uint32_t)(((uint64_t)lane * nb) >> 5)];
  const uint32_t breg = (!pivots && lane < nb) ? B[lane] : kNone;
  uint32_t total = 0;
  for (uint32_t base = 0; base < na; base += 32) {
    const uint32_t i = base + lane;
    const bool valid = i < na;
    const uint32_t a = valid ? A[i] : kNone;
    bool in;
    if (pivots) in = pivot_search(B, nb, piv, a) && valid;  // all lanes shuffle
    else in = chunk_contains(breg, a) && valid;
    const bool keep = valid && (OP == kIntersect ? in : !in);
    const unsigned m = __ballot_sync(kFull, keep);
    if (OUT == kWrite && keep) out[total + __popc(m & lanemask_lt())] = a;
    total += __popc(m);
  }
  return total;
}

// Core A∘B by chunked merge (balanced lengths).  Same contract as above.
template <SetOp OP, SetOut OUT>
__device__ __forceinline__ uint32_t warp_setop_merge(const uint32_t* __restrict__ A, uint32_t na,
                                                     const uint32_t* __restrict__ B, uint32_t nb,
                                                     uint32_t* __restrict__ out) {
  const uint32_t lane = lane_id();
  uint32_t total = 0;
  uint32_t ia = 0, ib = 0;
  uint32_t a = (lane < na) ? A[lane] : kNone;
  uint32_t b = (lane < nb) ? B[lane] : kNone;
  // per A chunk: lanes whose element was found in some B chunk so far
  bool found = false;
  while (ia < na) {
    if (ib >= nb) break;  // remaining A chunks see no more B elements
    found |= chunk_contains(b, a);
    const uint32_t la = min(31u, na - ia - 1), lb = min(31u, nb - ib - 1);
    const uint32_t a_last = __shfl_sync(kFull, a, la);
    const uint32_t b_last = __shfl_sync(kFull, b, lb);
    if (a_last <= b_last) {
      // A chunk complete: emit it
      const bool valid = ia + lane < na;
      const bool keep = valid && (OP == kIntersect ? found : !found);
      const unsigned m = __ballot_sync(kFull, keep);
      if (OUT == kWrite && keep) out[total + __popc(m & lanemask_lt())] = a;
      total += __popc(m);
      found = false;
      ia += 32;
      a = (ia + lane < na) ? A[ia + lane] : kNone;
    }
    if (b_last <= a_last) {
      ib += 32;
      b = (ib + lane < nb) ? B[ib + lane] : kNone;
    }
  }
  // A chunks never closed against B (B exhausted): intersection keeps the
  // found flags of the current chunk only; difference keeps everything else.
  while (ia < na) {
    const bool valid = ia + lane < na;
    const bool keep = valid && (OP == kIntersect ? found : !found);
    const unsigned m = __ballot_sync(kFull, keep);
    if (OUT == kWrite && keep) out[total + __popc(m & lanemask_lt())] = a;
    total += __popc(m);
    found = false;
    ia += 32;
    a = (ia + lane < na) ? A[ia + lane] : kNone;
  }
  return total;
}

// |A ∩ B| or A ∩ B (written to out in ascending order), choosing binary
// search when the longer list is at least `ratio` times the shorter one.
template <SetOut OUT>
__device__ __forceinline__ uint32_t warp_intersect(const uint32_t* __restrict__ A, uint32_t na,
                                                   const uint32_t* __restrict__ B, uint32_t nb,
                                                   uint32_t* __restrict__ out, uint32_t ratio) {
  if (na > nb) {
    const uint32_t* t = A; A = B; B = t;
    const uint32_t tn = na; na = nb; nb = tn;
  }
  if (na == 0) return 0;
  if ((uint64_t)nb >= (uint64_t)ratio * na)
    return warp_setop_bsearch<kIntersect, OUT>(A, na, B, nb, out);
  return warp_setop_merge<kIntersect, OUT>(A, na, B, nb, out);
}

// |A − B| or A − B (ascending), same variant choice on the length ratio.
template <SetOut OUT>
__device__ __forceinline__ uint32_t warp_difference(const uint32_t* __restrict__ A, uint32_t na,
                                                    const uint32_t* __restrict__ B, uint32_t nb,
                                                    uint32_t* __restrict__ out, uint32_t ratio) {
  if (na == 0) return 0;
  if (nb == 0) {
    if (OUT == kWrite)
      for (uint32_t i = lane_id(); i < na; i += 32) out[i] = A[i];
    return na;
  }
  if ((uint64_t)nb >= (uint64_t)ratio * na)
    return warp_setop_bsearch<kDifference, OUT>(A, na, B, nb, out);
  return warp_setop_merge<kDifference, OUT>(A, na, B, nb, out);
}

// Warp sum of a per-lane uint64.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

}  // namespace gpm
