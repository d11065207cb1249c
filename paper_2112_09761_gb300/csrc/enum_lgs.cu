// enum_lgs.cu — k-clique counting by local graph search (Section 5.4 (2)) with
// bitmap vertex sets (Section 6.2).
//
// A clique is a hub pattern: once its first (lowest-rank) vertex u is fixed,
// every other vertex lies in N+(u).  So each root vertex u gets a local graph:
// the DAG induced on A = N+(u), stored as one bitmap row per member,
//   row_i bit j  <=>  A[j] in N+(A[i])            (renaming A[j] -> j),
// built with one warp-cooperative set operation per member (Section 6.1).
// The deeper DFS levels then become AND + popc over rows of ceil(|A|/32)
// words instead of sorted-list intersections:
//   candidates after arc (u, A[i])          m = row_i
//   after the next vertex A[j], j in m      m' = m & row_j
//   last level                              count popc(m ...)
// Every clique is counted once: its topological order in the DAG fixes u,
// the arc (u, A[i]) and each later vertex.
//
// Three size classes of d = |N+(u)|, each its own launch:
//   d <= 64           one warp per vertex, rows are uint64 in shared memory,
//                     one lane per root arc for the bitmap DFS;
//   64 < d <= 1024    one CTA per vertex, members sorted by DAG rank so rows
//                     are upper-triangular, rows of d/32 words in shared
//                     memory; warps over root arcs, lanes over words for the
//                     upper levels and over members for the last one;
//   d > 1024          arcs go to the sorted-set kernel (enum_clique.cu).
// Root arcs outside the requested task range [lo, hi) are not counted, so
// gpm_count_range keeps its meaning.
#include "enum_common.cuh"

namespace gpm {

namespace {

constexpr int kWarpMaxD = 64;

// Bits j (0 <= j < d) with A[j] in L, for the warp-held A (lane l owns A[l]
// in a0 and A[32 + l] in a1; padding kNone).
__device__ __forceinline__ unsigned long long row_bits64(const uint32_t* __restrict__ L, uint32_t dl,
                                                         uint32_t a0, uint32_t a1, uint32_t d) {
  const uint32_t lane = lane_id();
  bool f0 = false, f1 = false;
  const bool two = d > 32;
  if (dl == 0) return 0ull;
  if (dl <= 64) {
    for (uint32_t base = 0; base < dl; base += 32) {
      const uint32_t c = (base + lane < dl) ? L[base + lane] : kNone;
      f0 |= chunk_contains(c, a0);
      if (two) f1 |= chunk_contains(c, a1);
    }
  } else {
    const uint32_t piv = L[(uint32_t)(((uint64_t)lane * dl) >> 5)];
    f0 = pivot_search(L, dl, piv, a0);
    if (two) f1 = pivot_search(L, dl, piv, a1);
  }
  const unsigned lo = __ballot_sync(kFull, f0 && lane < d);
  const unsigned hi = __ballot_sync(kFull, f1 && lane + 32 < d);
  return (unsigned long long)lo | ((unsigned long long)hi << 32);
}

// Number of L-level extensions of candidate set m (uint64 rows), per lane.
template <int L, bool ST>
__device__ __forceinline__ unsigned long long count64(const unsigned long long* rows,
                                                      unsigned long long m,
                                                      unsigned long long& wop) {
  if constexpr (L == 0) {
    return (unsigned long long)__popcll(m);
  } else {
    // A[j] for j in m in turn; the next candidates are m ∩ N+(A[j]) over the
    // whole of m (local indices follow vertex IDs, not DAG rank, so rows are
    // not triangular)
    unsigned long long t = 0, rem = m;
    while (rem) {
      const int j = __ffsll((long long)rem) - 1;
      rem &= rem - 1;
      if constexpr (ST) wop += 2;  // one 64-bit AND (+ POPC below) = two word-ops
      t += count64<L - 1, ST>(rows, m & rows[j], wop);
    }
    return t;
  }
}

template <int K, bool ST, bool BATCH>
__global__ void __launch_bounds__(256) k_lgs_warp(LgsArgs a) {
  __shared__ unsigned long long s_rows[8][kWarpMaxD];
  __shared__ unsigned long long s_acc;
  const uint32_t lane = lane_id(), wib = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_acc = 0;
  __syncthreads();
  unsigned long long* rows = s_rows[wib];
  unsigned long long acc = 0, stat_b = 0, wop = 0;
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(a.next, 4ull);
    start = __shfl_sync(kFull, start, 0);
    if (start >= a.nverts) break;
    const uint64_t end = min((uint64_t)start + 4, a.nverts);
    for (uint64_t q = start; q < end; q++) {
      DevCsr dag = a.dag;
      uint32_t u;
      uint64_t lo = a.lo, hi = a.hi;
      unsigned long long* gout = nullptr;
      if constexpr (BATCH) {
        const uint64_t r = a.broots[q];
        const LgsGraph& G = a.graphs[r >> 32];
        dag = G.dag;
        u = (uint32_t)r;
        lo = 0;
        hi = ~0ull;
        gout = a.gsums + (r >> 32) * a.gstride + a.gslot;
      } else {
        u = a.verts[q];
      }
      const int64_t o0 = dag.off[u], o1 = dag.off[u + 1];
      const uint32_t d = (uint32_t)(o1 - o0);
      const int64_t ia = max(o0, (int64_t)lo) - o0, ib = min(o1, (int64_t)min(hi, (uint64_t)o1)) - o0;
      if (ia >= ib) continue;
      const uint32_t* A = dag.nbr + o0;
      const uint32_t a0 = (lane < d) ? A[lane] : kNone;
      const uint32_t a1 = (lane + 32 < d) ? A[lane + 32] : kNone;
      // local graph rows (only rows reachable from the root arcs in range are
      // needed; for a full range that is all of them)
      for (uint32_t i = (K == 3 ? (uint32_t)ia : 0); i < (K == 3 ? (uint32_t)ib : d); i++) {
        const uint32_t v = (i < 32) ? __shfl_sync(kFull, a0, i) : __shfl_sync(kFull, a1, i - 32);
        const int64_t vs = dag.off[v];
        const uint32_t dl = (uint32_t)(dag.off[v + 1] - vs);
        const unsigned long long bits = row_bits64(dag.nbr + vs, dl, a0, a1, d);
        if (lane == 0) rows[i] = bits;
        if (a.stats) {
          const uint32_t lo2 = min(d, dl), hi2 = max(d, dl);
          stat_b += 4ull * (lo2 + min((unsigned long long)hi2,
                                      (unsigned long long)lo2 * (32 - __clz(hi2)))) + 16ull + 8ull;
        }
      }
      __syncwarp();
      unsigned long long root = 0;
      for (uint32_t i = (uint32_t)ia + lane; i < (uint32_t)ib; i += 32)
        root += count64<K - 3, ST>(rows, rows[i], wop);
      if constexpr (BATCH) {
        root = warp_sum_u64(root);
        if (lane == 0 && root) atomicAdd(gout, root);
      } else {
        acc += root;
      }
      __syncwarp();
    }
  }
  acc = warp_sum_u64(acc);
  if (lane == 0 && acc) atomicAdd(&s_acc, acc);
  if (a.stats && lane == 0 && stat_b) atomicAdd(&a.stats[0], stat_b);
  if constexpr (ST) {
    wop = warp_sum_u64(wop);
    if (lane == 0 && wop) atomicAdd(&a.stats[2], wop);
  }
  __syncthreads();
  if (!BATCH && threadIdx.x == 0 && s_acc) atomicAdd(a.result, s_acc);
}

// ---------------------------------------------------------------- CTA class
//
// One CTA per root with a local graph of 64 < d <= 32*NW members.  Members
// are laid out in DAG-rank order (sorted by the orientation key (degree, id)),
// so row_i only holds members after i: rows are upper-triangular.  Rows have
// a padded stride of NW+2 words: every row starts 8-byte aligned, so the
// innermost word loops load word pairs (64-bit shared-memory loads), and the
// padding words stay zero.  Lane l of a warp holds word l of a candidate set.
//
// Roots are vertices u (members N+(u), a root arc per member), or, for roots
// too large for shared memory, arcs (u, v) with members N+(u) ∩ N+(v).
//
// f_L(S) = number of L-cliques of the local DAG inside candidate set S:
//   f_1(S) = |S|,  f_L(S) = sum over x in S of f_{L-1}(S ∩ row_x).
// Above the last two levels, a set with at most 64 members is first
// compressed to its own 64x64 bitmap (one uint64 row per member, in shared
// memory) and finished lane-parallel, one lane per member; larger sets iterate
// their members warp-cooperatively.  The last two levels (edges inside a set)
// always run lane-parallel over members, word by word.

// CTA shape per class: NW words per row (members <= 32*NW); 512 threads for
// the 8-word class (four CTAs per SM), 1024 for the 16-word class (two CTAs
// per SM fit in shared memory: 64 warps), 31 warps for the 32-word class (one
// CTA fills the shared memory, so it brings all the warps it can: its rows
// and per-warp scratch leave room for 31 warps' scratch, not 32).
template <int NW>
struct BlockShape {
  static constexpr int THREADS = NW >= 32 ? 992 : (NW >= 16 ? 1024 : 512);
  static constexpr int WARPS = THREADS / 32;
};

template <int NW>
struct BlockSmem {
  static constexpr int MAXD = 32 * NW;
  static constexpr int STRIDE = NW + 2;
  static constexpr int WARPS = BlockShape<NW>::WARPS;
  static constexpr size_t rows = 0;                                           // u32 [MAXD*STRIDE]
  static constexpr size_t aid = rows + sizeof(uint32_t) * MAXD * STRIDE;      // u32 [MAXD] ids (id order)
  static constexpr size_t ridx = aid + sizeof(uint32_t) * MAXD;               // u16 [MAXD] id pos of rank pos
  static constexpr size_t rpos = ridx + sizeof(uint16_t) * MAXD;              // u16 [MAXD] rank pos of id pos
  // per-warp scratch; the rank-sort keys (u64 [MAXD]) reuse this area before
  // the counting phase starts
  static constexpr size_t scratch = rpos + sizeof(uint16_t) * MAXD;
  static constexpr size_t cmp = scratch;                                       // u64 [warps][64]
  static constexpr size_t sbuf = cmp + sizeof(unsigned long long) * 64 * WARPS;  // u32 [warps][32]
  static constexpr size_t list = sbuf + sizeof(uint32_t) * 32 * WARPS;        // u16 [warps][MAXD]
  static constexpr size_t scratch_end = list + sizeof(uint16_t) * MAXD * WARPS;
  static constexpr size_t key = scratch;                                       // u64 [MAXD] (aliases)
  static constexpr size_t bytes =
      scratch_end > key + sizeof(unsigned long long) * MAXD ? scratch_end
                                                            : key + sizeof(unsigned long long) * MAXD;
};

struct WarpScratch {
  uint32_t* sb;            // [32] words of the current set
  uint16_t* list;          // [MAXD] member positions of the current set
  unsigned long long* cmp;  // [64] compressed rows
};

// Positions of the members of S (ascending) into list; returns |S|.
__device__ __forceinline__ uint32_t compact_set(uint32_t S, uint16_t* list) {
  const uint32_t lane = lane_id();
  const uint32_t c = __popc(S);
  uint32_t inc = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFull, inc, o);
    if ((int)lane >= o) inc += y;
  }
  const uint32_t total = __shfl_sync(kFull, inc, 31);
  uint32_t p = inc - c, bits = S;
  while (bits) {
    const uint32_t b = __ffs(bits) - 1;
    bits &= bits - 1;
    list[p++] = (uint16_t)(lane * 32 + b);
  }
  __syncwarp();
  return total;
}

template <int L, int NW, bool ST>
__device__ __forceinline__ unsigned long long f_set(uint32_t S, const uint32_t* rows, uint32_t nw,
                                                    const WarpScratch& ws, unsigned long long& wop);

// f_L(S) for |S| = s <= 64 after compact_set: compressed rows, lane-parallel.
template <int L, int NW, bool ST>
__device__ __forceinline__ unsigned long long f_small(uint32_t s, const uint32_t* rows,
                                                      const WarpScratch& ws,
                                                      unsigned long long& wop) {
  constexpr int STRIDE = NW + 2;
  const uint32_t lane = lane_id();
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const uint32_t j = lane + 32 * h;
    if (j < s) {
      const uint32_t* rj = rows + (uint32_t)ws.list[j] * STRIDE;
      unsigned long long b = 0;
      for (uint32_t y = j + 1; y < s; y++) {  // rows are upper-triangular
        const uint32_t py = ws.list[y];
        b |= (unsigned long long)((rj[py >> 5] >> (py & 31)) & 1u) << y;
      }
      if constexpr (ST) wop += (s > j + 1) ? s - j - 1 : 0;  // bit tests
      ws.cmp[j] = b;
    }
  }
  __syncwarp();
  unsigned long long t = 0;
#pragma unroll
  for (int h = 0; h < 2; h++) {
    const uint32_t j = lane + 32 * h;
    if (j < s) t += count64<L - 2, ST>(ws.cmp, ws.cmp[j], wop);
  }
  __syncwarp();
  return t;
}

// f_3(S), the triangles inside S, lane-parallel over the members x of S:
// each lane walks the members y of S ∩ row_x and adds |S ∩ row_x ∩ row_y|
// word by word.  S is compacted once; the sets S ∩ row_x are never
// materialised (rows are triangular, so words start after x and after y).
// Members are handed to lanes in ascending order through a per-warp counter,
// so a lane that finishes early takes the next member (the first members
// carry the most work).  The count fits 32 bits (at most C(1024, 3)).
template <int NW, bool ST>
__device__ __forceinline__ unsigned long long f3_lanes(uint32_t S, uint32_t s, const uint32_t* rows,
                                                       uint32_t nw, const WarpScratch& ws,
                                                       unsigned long long& wop) {
  constexpr int STRIDE = NW + 2;
  const uint32_t lane = lane_id();
  compact_set(S, ws.list);
  ws.sb[lane] = S;
  uint32_t* next = reinterpret_cast<uint32_t*>(ws.cmp);  // unused by this level
  if (lane == 0) *next = 32;
  __syncwarp();
  uint32_t acc = 0;
  for (uint32_t k = lane; k < s;) {
    const uint32_t x = ws.list[k];
    const uint32_t* rx = rows + x * STRIDE;
#pragma unroll 2
    for (uint32_t w = (x + 1) >> 5; w < nw; w++) {
      uint32_t t = ws.sb[w] & rx[w];
      if constexpr (ST) wop += 1;
      while (t) {
        const uint32_t y = w * 32 + __ffs(t) - 1;
        t &= t - 1;
        const uint32_t* ry = rows + y * STRIDE;
        // word pairs (rows and the set are 8-byte aligned; the word before
        // an odd start holds no bit after y, words past nw are zero)
        const uint2* sb2 = reinterpret_cast<const uint2*>(ws.sb);
        const uint2* rx2 = reinterpret_cast<const uint2*>(rx);
        const uint2* ry2 = reinterpret_cast<const uint2*>(ry);
        for (uint32_t p = (y + 1) >> 6; 2 * p < nw; p++) {
          const uint2 a = sb2[p], b = rx2[p], c = ry2[p];
          acc += __popc(a.x & b.x & c.x) + __popc(a.y & b.y & c.y);
        }
        if constexpr (ST) wop += nw - ((y + 1) >> 5);
      }
    }
    k = atomicAdd(next, 1u);
  }
  __syncwarp();
  return acc;
}

template <int L, int NW, bool ST>
__device__ __forceinline__ unsigned long long f_set(uint32_t S, const uint32_t* rows, uint32_t nw,
                                                    const WarpScratch& ws, unsigned long long& wop) {
  if constexpr (L == 1) {
    return (unsigned long long)__popc(S);
  } else {
    constexpr int STRIDE = NW + 2;
    const uint32_t lane = lane_id();
    const uint32_t s = __reduce_add_sync(kFull, __popc(S));
    if (s < (uint32_t)L) return 0;
    // compress small sets only where deeper levels reuse the compressed rows
    // (L >= 3); for the last two vertices (L = 2) each row is read once, and
    // the word loop below is cheaper than building the compressed rows
    if (L >= 3 && s <= 64) {
      compact_set(S, ws.list);
      return f_small<L, NW, ST>(s, rows, ws, wop);
    }
    if constexpr (L == 3) return f3_lanes<NW, ST>(S, s, rows, nw, ws, wop);
    if constexpr (L == 2) {
      // edges inside S: lanes take members x, |S ∩ row_x| word by word
      // (at most C(1024, 2) edges: 32 bits)
      compact_set(S, ws.list);
      ws.sb[lane] = S;
      __syncwarp();
      uint32_t acc = 0;
      for (uint32_t k = lane; k < s; k += 32) {
        const uint32_t x = ws.list[k];
        const uint32_t* rx = rows + x * STRIDE;
        const uint2* sb2 = reinterpret_cast<const uint2*>(ws.sb);
        const uint2* rx2 = reinterpret_cast<const uint2*>(rx);
        for (uint32_t p = (x + 1) >> 6; 2 * p < nw; p++) {
          const uint2 a = sb2[p], b = rx2[p];
          acc += __popc(a.x & b.x) + __popc(a.y & b.y);
        }
        if constexpr (ST) wop += nw - ((x + 1) >> 5);
      }
      __syncwarp();
      return acc;
    } else {
      unsigned long long t = 0;
      uint32_t rem = S;
      for (;;) {
        const unsigned nz = __ballot_sync(kFull, rem != 0);
        if (!nz) break;
        const int wl = __ffs(nz) - 1;
        const uint32_t word = __shfl_sync(kFull, rem, wl);
        const int x = wl * 32 + __ffs(word) - 1;
        if ((int)lane == wl) rem &= rem - 1;
        const uint32_t rx = (lane < (uint32_t)NW) ? rows[x * STRIDE + lane] : 0u;
        if constexpr (ST) wop += (lane < nw) ? 1u : 0u;
        t += f_set<L - 1, NW, ST>(S & rx, rows, nw, ws, wop);
      }
      return t;
    }
  }
}

// ARC = false: roots are vertices u of a.verts; ARC = true: roots are the
// arcs a.idx[q] (members N+(u) ∩ N+(v)); roots whose member set exceeds
// 32*NW are appended to a.overflow for the sorted-set kernel.
template <int K, int NW, bool ARC, bool ST, bool BATCH>
__global__ void __launch_bounds__(BlockShape<NW>::THREADS) k_lgs_block(LgsArgs a) {
  using SM = BlockSmem<NW>;
  constexpr int kWarps = BlockShape<NW>::WARPS;
  constexpr int MAXD = SM::MAXD, STRIDE = SM::STRIDE;
  extern __shared__ __align__(16) unsigned char s_raw[];
  uint32_t* rows = reinterpret_cast<uint32_t*>(s_raw + SM::rows);
  unsigned long long* key = reinterpret_cast<unsigned long long*>(s_raw + SM::key);
  uint32_t* aid = reinterpret_cast<uint32_t*>(s_raw + SM::aid);
  uint16_t* ridx = reinterpret_cast<uint16_t*>(s_raw + SM::ridx);
  uint16_t* rpos = reinterpret_cast<uint16_t*>(s_raw + SM::rpos);
  __shared__ unsigned long long s_q;
  __shared__ unsigned int s_arc, s_d;
  __shared__ unsigned long long s_acc;
  const uint32_t lane = lane_id(), wib = threadIdx.x >> 5;
  WarpScratch ws;
  ws.sb = reinterpret_cast<uint32_t*>(s_raw + SM::sbuf) + wib * 32;
  ws.list = reinterpret_cast<uint16_t*>(s_raw + SM::list) + wib * MAXD;
  ws.cmp = reinterpret_cast<unsigned long long*>(s_raw + SM::cmp) + wib * 64;
  if (threadIdx.x == 0) s_acc = 0;
  unsigned long long acc = 0, stat_b = 0, wop = 0;
  const uint64_t nroots = ARC ? a.nidx : a.nverts;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_q = atomicAdd(a.next, 1ull);
      s_arc = 0;
    }
    __syncthreads();
    const uint64_t q = s_q;
    if (q >= nroots) break;
    // the root's graph: the plan's, or (batch) the one packed into the root
    DevCsr dag = a.dag;
    const int64_t* uoff = a.uoff;
    const uint32_t* src = a.src;
    uint64_t lo = a.lo, hi = a.hi, rootv = 0;
    unsigned long long* gout = nullptr;
    if constexpr (BATCH) {
      const uint64_t r = a.broots[q];
      const uint64_t g = ARC ? (r >> 40) : (r >> 32);
      const LgsGraph& G = a.graphs[g];
      dag = G.dag;
      uoff = G.uoff;
      src = G.src;
      lo = 0;
      hi = ~0ull;
      rootv = ARC ? (r & ((1ull << 40) - 1)) : (r & 0xffffffffull);
      gout = a.gsums + g * a.gstride + a.gslot;
    } else {
      rootv = ARC ? a.idx[q] : a.verts[q];
    }
    uint32_t d = 0;
    int64_t ia = 0, ib = 0;  // root arcs (member positions, id order) to count
    if constexpr (!ARC) {
      const uint32_t u = (uint32_t)rootv;
      const int64_t o0 = dag.off[u], o1 = dag.off[u + 1];
      d = (uint32_t)(o1 - o0);
      ia = max(o0, (int64_t)lo) - o0;
      ib = min(o1, (int64_t)min(hi, (uint64_t)o1)) - o0;
      if (ia >= ib || d > (uint32_t)MAXD) continue;  // block-uniform
      for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) aid[t] = dag.nbr[o0 + t];
    } else {
      const uint64_t e = rootv;
      if (e < lo || e >= hi) continue;
      const uint32_t u = src[e], v = dag.nbr[e];
      const int64_t u0 = dag.off[u], v0 = dag.off[v];
      const uint32_t du = (uint32_t)(dag.off[u + 1] - u0), dv = (uint32_t)(dag.off[v + 1] - v0);
      if (min(du, dv) > (uint32_t)MAXD) {
        if (threadIdx.x == 0) a.overflow[atomicAdd(a.overflow_count, 1ull)] = BATCH ? a.broots[q] : e;
        continue;
      }
      if (wib == 0) {
        const uint32_t c = warp_intersect<kWrite>(dag.nbr + u0, du, dag.nbr + v0, dv, aid, 8);
        if (lane == 0) s_d = c;
      }
      __syncthreads();
      d = s_d;
      if (d < (uint32_t)(K - 2)) continue;
    }
    const uint32_t nw = (d + 31) >> 5;
    uint32_t P = 1;
    while (P < d) P <<= 1;
    for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
      if (t < d) {
        const uint32_t v = aid[t];
        key[t] = ((unsigned long long)(uoff[v + 1] - uoff[v]) << 32) | v;  // orientation key
      } else {
        key[t] = ~0ull;
      }
      ridx[t] = (uint16_t)t;
    }
    for (uint32_t t = threadIdx.x; t < d * STRIDE; t += blockDim.x) rows[t] = 0u;
    __syncthreads();
    // bitonic sort of (key, ridx) by the orientation key (undirected degree,
    // id): every out-neighbour of a member ranks after it, so rows built in
    // this order are upper-triangular
    for (uint32_t k = 2; k <= P; k <<= 1) {
      for (uint32_t j = k >> 1; j > 0; j >>= 1) {
        for (uint32_t t = threadIdx.x; t < P; t += blockDim.x) {
          const uint32_t x = t ^ j;
          if (x > t) {
            const bool up = (t & k) == 0;
            const unsigned long long kt = key[t], kx = key[x];
            if ((kt > kx) == up) {
              key[t] = kx; key[x] = kt;
              const uint16_t r = ridx[t]; ridx[t] = ridx[x]; ridx[x] = r;
            }
          }
        }
        __syncthreads();
      }
    }
    for (uint32_t t = threadIdx.x; t < d; t += blockDim.x) rpos[ridx[t]] = (uint16_t)t;
    __syncthreads();
    // rows in rank order: one warp per member
    for (uint32_t i = wib; i < d; i += kWarps) {
      const uint32_t v = aid[ridx[i]];
      const int64_t vs = dag.off[v];
      const uint32_t dl = (uint32_t)(dag.off[v + 1] - vs);
      const uint32_t* Lv = dag.nbr + vs;
      if (dl == 0) continue;
      if (dl >= 2 * d) {
        const uint32_t piv = Lv[(uint32_t)(((uint64_t)lane * dl) >> 5)];
        for (uint32_t c = (i + 1) >> 5; c < nw; c++) {  // triangular: members after i
          const uint32_t pos = 32 * c + lane;
          const uint32_t x = (pos < d) ? aid[ridx[pos]] : kNone;
          const bool f = pivot_search(Lv, dl, piv, x) && pos < d;
          const unsigned w = __ballot_sync(kFull, f);
          if (lane == 0) rows[i * STRIDE + c] = w;
        }
      } else {
        for (uint32_t base = 0; base < dl; base += 32) {
          if (base + lane < dl) {
            const uint32_t x = Lv[base + lane];
            uint32_t lo = 0, hi = d;
            while (lo < hi) {
              const uint32_t mid = (lo + hi) >> 1;
              if (aid[mid] < x) lo = mid + 1; else hi = mid;
            }
            if (lo < d && aid[lo] == x) {
              const uint32_t r = rpos[lo];
              atomicOr(&rows[i * STRIDE + (r >> 5)], 1u << (r & 31));
            }
          }
        }
      }
      if (a.stats && lane == 0) {
        const uint32_t lo2 = min(d, dl), hi2 = max(d, dl);
        stat_b += 4ull * (lo2 + min((unsigned long long)hi2,
                                    (unsigned long long)lo2 * (32 - __clz(hi2)))) + 16ull + 4ull * nw;
      }
    }
    __syncthreads();
    // bitmap DFS: warps take member rows dynamically
    for (;;) {
      unsigned int r = 0;
      if (lane == 0) r = atomicAdd(&s_arc, 1u);
      r = __shfl_sync(kFull, r, 0);
      if (r >= d) break;
      const uint32_t m = (lane < nw) ? rows[r * STRIDE + lane] : 0u;
      unsigned long long c;
      if constexpr (!ARC) {
        // root arc (u, member r): K-cliques = (K-2)-cliques inside row_r
        const int64_t id_pos = ridx[r];
        if (id_pos < ia || id_pos >= ib) continue;
        c = f_set<K - 2, NW, ST>(m, rows, nw, ws, wop);
      } else {
        // root arc (u, v), third vertex = member r: (K-3)-cliques inside row_r
        c = f_set<K - 3, NW, ST>(m, rows, nw, ws, wop);
      }
      if constexpr (BATCH) {
        c = warp_sum_u64(c);
        if (lane == 0 && c) atomicAdd(gout, c);
      } else {
        acc += c;
      }
    }
  }
  acc = warp_sum_u64(acc);
  if (lane == 0 && acc) atomicAdd(&s_acc, acc);
  if (a.stats && lane == 0 && stat_b) atomicAdd(&a.stats[0], stat_b);
  if constexpr (ST) {
    wop = warp_sum_u64(wop);
    if (lane == 0 && wop) atomicAdd(&a.stats[2], wop);
  }
  __syncthreads();
  if (!BATCH && threadIdx.x == 0 && s_acc) atomicAdd(a.result, s_acc);
}

// Batch roots (a.graphs set) are only instantiated for 4-cliques, the size
// the batched motif counts need.
template <int K>
cudaError_t launch_warp_k(const LgsArgs& a, unsigned blocks, cudaStream_t s) {
  if (a.graphs) {
    if constexpr (K == 4) k_lgs_warp<K, false, true><<<blocks, 256, 0, s>>>(a);
    else return cudaErrorInvalidValue;
  } else if (a.stats) {
    k_lgs_warp<K, true, false><<<blocks, 256, 0, s>>>(a);
  } else {
    k_lgs_warp<K, false, false><<<blocks, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <int K, int NW, bool ARC>
cudaError_t launch_block_k(const LgsArgs& a, unsigned blocks, cudaStream_t s) {
  const size_t smem = BlockSmem<NW>::bytes;
  void (*kern)(LgsArgs) = a.stats ? k_lgs_block<K, NW, ARC, true, false>
                                  : k_lgs_block<K, NW, ARC, false, false>;
  if (a.graphs) {
    if constexpr (K == 4) kern = k_lgs_block<K, NW, ARC, false, true>;
    else return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<blocks, BlockShape<NW>::THREADS, smem, s>>>(a);
  return cudaGetLastError();
}

template <int K, int NW>
int occ_block_k() {
  const size_t smem = BlockSmem<NW>::bytes;
  auto kern = k_lgs_block<K, NW, false, false, false>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 1;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, BlockShape<NW>::THREADS, smem) !=
      cudaSuccess)
    return 1;
  return b > 0 ? b : 1;
}

}  // namespace

// Size classes handled by the bitmap kernels.
uint32_t lgs_warp_max_degree() { return kWarpMaxD; }
uint32_t lgs_block_max_degree() { return 1024; }

// Launch the warp kernel (d <= 64) for clique size k.
cudaError_t lgs_launch_warp(int k, const LgsArgs& a, unsigned blocks, cudaStream_t s) {
  switch (k) {
    case 4: return launch_warp_k<4>(a, blocks, s);
    case 5: return launch_warp_k<5>(a, blocks, s);
    case 6: return launch_warp_k<6>(a, blocks, s);
    case 7: return launch_warp_k<7>(a, blocks, s);
    case 8: return launch_warp_k<8>(a, blocks, s);
    default: return cudaErrorInvalidValue;
  }
}

// Launch the block kernel with rows of nw words (8: d <= 256, 16: d <= 512,
// 32: d <= 1024); `arc` roots at the arcs of a.idx (32-word rows).
cudaError_t lgs_launch_block(int k, int nw, bool arc, const LgsArgs& a, unsigned blocks_per_sm,
                             unsigned sms, cudaStream_t s) {
#define GPM_B(KK)                                                                            \
  case KK:                                                                                   \
    if (arc) return launch_block_k<KK, 32, true>(a, blocks_per_sm * sms, s);                 \
    if (nw == 8) return launch_block_k<KK, 8, false>(a, blocks_per_sm * sms, s);             \
    if (nw == 16) return launch_block_k<KK, 16, false>(a, blocks_per_sm * sms, s);           \
    return launch_block_k<KK, 32, false>(a, blocks_per_sm * sms, s);
  switch (k) {
    GPM_B(4) GPM_B(5) GPM_B(6) GPM_B(7) GPM_B(8)
    default: return cudaErrorInvalidValue;
  }
#undef GPM_B
}

int lgs_block_occupancy(int k, int nw) {
#define GPM_O(KK) \
  case KK: return nw == 8 ? occ_block_k<KK, 8>() : nw == 16 ? occ_block_k<KK, 16>() : occ_block_k<KK, 32>();
  switch (k) {
    GPM_O(4) GPM_O(5) GPM_O(6) GPM_O(7) GPM_O(8)
    default: return 1;
  }
#undef GPM_O
}

}  // namespace gpm
