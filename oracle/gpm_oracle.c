/*
 * gpm_oracle.c — plain, slow, obviously-correct CPU oracle for pattern-aware
 * subgraph enumeration (G2Miner, arXiv 2112.09761).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path: it has its own set operations,
 * its own orientation and its own task lists.  Its only common ground with
 * the CUDA path is the input CSR (built by the seeded generators) and the
 * documented definitions of the root-task order (below).
 *
 * Three tiers:
 *   O1  og_brute       - the definition written out (Section 2.1): every
 *                        k-subset S, every bijection; vertex-induced counts
 *                        S with G[S] ~= P, edge-induced counts edge subsets
 *                        F of G[S] with (S,F) ~= P.  Tiny graphs only.
 *   O2  og_count/list  - nested-loop matcher: the plans' matching orders and
 *                        symmetry orders as plain loops with merge-based set
 *                        intersection / difference (Algorithm 1, Sections 2.2,
 *                        5.4, 6.1).  Per root task, so a sub-range of the task
 *                        list can be compared at full size.
 *   O1b og_injhom      - any pattern: injective homomorphisms P -> G by plain
 *                        backtracking (no symmetry breaking), divided by
 *                        |Aut(P)| (og_automorphisms) gives the count of
 *                        Section 2.1; mid-size graphs.
 *   O3  og_identities  - closed forms / pattern decompositions (Section 5.4
 *                        counting-only pruning generalised): degrees,
 *                        per-edge triangle counts, wedge co-degrees, and the
 *                        edge-induced -> vertex-induced 4-motif inversion.
 *
 * Root task list Omega (Sections 5.1, 7.2).  Index t of:
 *   CLIQUE     the t-th arc of the degree-oriented DAG: u->v iff
 *              (deg u, u) < (deg v, v); arcs listed by source ascending, then
 *              destination ascending (Section 4.2 orientation).
 *   LOWER      the t-th pair (v1, v2), v2 in N(v1), v2 < v1, listed by v1
 *              ascending then v2 ascending (edgelist reduction, Section 7.2).
 *   ALL        the t-th directed edge of the CSR (v1 = row, v2 = column).
 *
 * Counts are uint64; all arithmetic is integer.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* pattern families (the oracle's own codes) */
enum {
  OG_CLIQUE = 1,          /* k = 3..8; k = 3 is the triangle */
  OG_DIAMOND = 2,         /* K4 minus one edge */
  OG_CYCLE4 = 3,          /* 4-cycle */
  OG_TAILED_TRIANGLE = 4, /* triangle plus a pendant edge */
  OG_STAR3 = 5,           /* claw K_{1,3} */
  OG_PATH4 = 6,           /* path on 4 vertices */
  OG_WEDGE = 7            /* path on 3 vertices */
};

enum { OG_TASKS_CLIQUE = 1, OG_TASKS_LOWER = 2, OG_TASKS_ALL = 3 };

typedef struct {
  uint32_t n;
  const int64_t* off;
  const uint32_t* nbr;
} og_g;

/* ------------------------------------------------------ set operations --- */

/* C = A ∩ B by a plain two-pointer merge (out may be NULL: count only). */
static uint64_t og_intersect(const uint32_t* a, uint64_t na, const uint32_t* b, uint64_t nb,
                             uint32_t* out) {
  uint64_t i = 0, j = 0, k = 0;
  while (i < na && j < nb) {
    if (a[i] < b[j]) i++;
    else if (a[i] > b[j]) j++;
    else { if (out) out[k] = a[i]; k++; i++; j++; }
  }
  return k;
}

/* Set bounding {x in A : x < y}: the length of that prefix of sorted A. */
static uint64_t og_bound(const uint32_t* a, uint64_t na, uint32_t y) {
  uint64_t k = 0;
  while (k < na && a[k] < y) k++;
  return k;
}

static int og_adjacent(const og_g* g, uint32_t u, uint32_t v) {
  const uint32_t* a = g->nbr + g->off[u];
  int64_t lo = 0, hi = g->off[u + 1] - g->off[u] - 1;
  while (lo <= hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] == v) return 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid - 1;
  }
  return 0;
}

#define DEG(g, v) ((uint64_t)((g)->off[(v) + 1] - (g)->off[(v)]))
#define ROW(g, v) ((g)->nbr + (g)->off[(v)])

/* ------------------------------------------------------- orientation --- */

/* Degree-oriented DAG (Section 4.2): u->v iff (deg u, u) < (deg v, v).
 * Out-lists keep ascending ID order.  Returns 0 or -1 (allocation). */
static int og_orient(const og_g* g, int64_t** doff_out, uint32_t** dnbr_out) {
  uint32_t n = g->n;
  int64_t* doff = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!doff) return -1;
  doff[0] = 0;
  for (uint32_t u = 0; u < n; u++) {
    uint64_t du = DEG(g, u), c = 0;
    for (uint64_t i = 0; i < du; i++) {
      uint32_t v = ROW(g, u)[i];
      uint64_t dv = DEG(g, v);
      if (du < dv || (du == dv && u < v)) c++;
    }
    doff[u + 1] = doff[u] + (int64_t)c;
  }
  uint32_t* dnbr = (uint32_t*)malloc(((size_t)doff[n] + 1) * sizeof(uint32_t));
  if (!dnbr) { free(doff); return -1; }
  for (uint32_t u = 0; u < n; u++) {
    uint64_t du = DEG(g, u);
    int64_t w = doff[u];
    for (uint64_t i = 0; i < du; i++) {
      uint32_t v = ROW(g, u)[i];
      uint64_t dv = DEG(g, v);
      if (du < dv || (du == dv && u < v)) dnbr[w++] = v;
    }
  }
  *doff_out = doff;
  *dnbr_out = dnbr;
  return 0;
}

/* --------------------------------------------------------- task lists --- */

static int og_task_kind(int family) {
  switch (family) {
    case OG_CLIQUE: return OG_TASKS_CLIQUE;
    case OG_DIAMOND: case OG_CYCLE4: case OG_PATH4: return OG_TASKS_LOWER;
    case OG_TAILED_TRIANGLE: case OG_STAR3: case OG_WEDGE: return OG_TASKS_ALL;
    default: return 0;
  }
}

/* Build Omega as (src, dst) arrays.  For CLIQUE, g is the DAG. */
static int og_tasks(const og_g* g, int kind, uint32_t** src_out, uint32_t** dst_out,
                    uint64_t* ntasks) {
  uint64_t cnt = 0;
  for (uint32_t v = 0; v < g->n; v++) {
    if (kind == OG_TASKS_LOWER) cnt += og_bound(ROW(g, v), DEG(g, v), v);
    else cnt += DEG(g, v);
  }
  uint32_t* s = (uint32_t*)malloc((cnt + 1) * sizeof(uint32_t));
  uint32_t* d = (uint32_t*)malloc((cnt + 1) * sizeof(uint32_t));
  if (!s || !d) { free(s); free(d); return -1; }
  uint64_t t = 0;
  for (uint32_t v = 0; v < g->n; v++) {
    uint64_t len = (kind == OG_TASKS_LOWER) ? og_bound(ROW(g, v), DEG(g, v), v) : DEG(g, v);
    for (uint64_t i = 0; i < len; i++) { s[t] = v; d[t] = ROW(g, v)[i]; t++; }
  }
  *src_out = s; *dst_out = d; *ntasks = cnt;
  return 0;
}

/* ------------------------------------------------------- the matcher --- */

typedef struct {
  uint32_t* out;     /* listing buffer (k uint32 per match) or NULL */
  uint64_t cap;      /* capacity in matches */
  uint64_t written;  /* matches written */
  uint32_t k;
} og_sink;

static inline void og_emit(og_sink* s, const uint32_t* m) {
  if (s && s->out && s->written < s->cap)
    memcpy(s->out + s->written * s->k, m, s->k * sizeof(uint32_t));
  if (s) s->written++;
}

/* k-clique on the DAG: C holds the candidates for vertex `depth` (0-based)
 * given m[0..depth-1]; each level intersects with the out-list of the vertex
 * just matched (Section 4.2 orientation + Algorithm 1 style nesting). */
static uint64_t og_clique_rec(const og_g* dag, uint32_t k, uint32_t depth, const uint32_t* C,
                              uint64_t nC, uint32_t** bufs, uint32_t* m, og_sink* sink) {
  if (depth + 1 == k) {
    if (sink)
      for (uint64_t i = 0; i < nC; i++) { m[depth] = C[i]; og_emit(sink, m); }
    return nC;
  }
  uint64_t total = 0;
  for (uint64_t i = 0; i < nC; i++) {
    uint32_t w = C[i];
    m[depth] = w;
    uint64_t n2 = og_intersect(C, nC, ROW(dag, w), DEG(dag, w), bufs[depth]);
    total += og_clique_rec(dag, k, depth + 1, bufs[depth], n2, bufs, m, sink);
  }
  return total;
}

/* One root task (v1, v2) of the given plan.  `bufs` are scratch lists of at
 * least max-degree entries.  Returns the number of matches under the task. */
static uint64_t og_task(const og_g* g, const og_g* dag, int family, uint32_t k, int induced,
                        uint32_t v1, uint32_t v2, uint32_t** bufs, og_sink* sink) {
  uint32_t m[8];
  uint64_t count = 0;
  m[0] = v1; m[1] = v2;
  switch (family) {
    case OG_CLIQUE: {
      /* u->v arc; candidates N+(v1) ∩ N+(v2); deeper levels intersect */
      uint64_t n1 = og_intersect(ROW(dag, v1), DEG(dag, v1), ROW(dag, v2), DEG(dag, v2), bufs[7]);
      return og_clique_rec(dag, k, 2, bufs[7], n1, bufs, m, sink);
    }
    case OG_DIAMOND: {
      /* Algorithm 1: W = N(v1) ∩ N(v2); v3, v4 in W with v4 < v3 */
      uint32_t* W = bufs[0];
      uint64_t nW = og_intersect(ROW(g, v1), DEG(g, v1), ROW(g, v2), DEG(g, v2), W);
      for (uint64_t i = 0; i < nW; i++) {
        uint32_t v3 = W[i];
        for (uint64_t j = 0; j < nW; j++) {
          uint32_t v4 = W[j];
          if (v4 >= v3) break;
          if (induced && og_adjacent(g, v3, v4)) continue;
          m[2] = v3; m[3] = v4;
          og_emit(sink, m);
          count++;
        }
      }
      return count;
    }
    case OG_CYCLE4: {
      /* v1 = max vertex; v2 > v4 its cycle neighbours; v3 opposite, v3 < v1 */
      uint64_t n4 = og_bound(ROW(g, v1), DEG(g, v1), v2);
      for (uint64_t i = 0; i < n4; i++) {
        uint32_t v4 = ROW(g, v1)[i];
        if (induced && og_adjacent(g, v2, v4)) continue;
        uint32_t* S = bufs[0];
        uint64_t nS = og_intersect(ROW(g, v2), og_bound(ROW(g, v2), DEG(g, v2), v1),
                                   ROW(g, v4), og_bound(ROW(g, v4), DEG(g, v4), v1), S);
        for (uint64_t j = 0; j < nS; j++) {
          uint32_t v3 = S[j];
          if (induced && og_adjacent(g, v1, v3)) continue;
          m[2] = v3; m[3] = v4;
          og_emit(sink, m);
          count++;
        }
      }
      return count;
    }
    case OG_TAILED_TRIANGLE: {
      /* v1 = degree-3 vertex, (v1,v2) any direction, v3 in N(v1)∩N(v2), v3<v2,
       * tail v4 in N(v1) \ {v2, v3} (vertex-induced: v4 not adjacent to v2, v3) */
      uint32_t* W = bufs[0];
      uint64_t nW = og_intersect(ROW(g, v1), DEG(g, v1), ROW(g, v2), DEG(g, v2), W);
      for (uint64_t i = 0; i < nW; i++) {
        uint32_t v3 = W[i];
        if (v3 >= v2) break;
        for (uint64_t j = 0; j < DEG(g, v1); j++) {
          uint32_t v4 = ROW(g, v1)[j];
          if (v4 == v2 || v4 == v3) continue;
          if (induced && (og_adjacent(g, v2, v4) || og_adjacent(g, v3, v4))) continue;
          m[2] = v3; m[3] = v4;
          og_emit(sink, m);
          count++;
        }
      }
      return count;
    }
    case OG_STAR3: {
      /* centre v1, leaves v2 > v3 > v4 */
      for (uint64_t i = 0; i < DEG(g, v1); i++) {
        uint32_t v3 = ROW(g, v1)[i];
        if (v3 >= v2) break;
        if (induced && og_adjacent(g, v2, v3)) continue;
        for (uint64_t j = 0; j < DEG(g, v1); j++) {
          uint32_t v4 = ROW(g, v1)[j];
          if (v4 >= v3) break;
          if (induced && (og_adjacent(g, v2, v4) || og_adjacent(g, v3, v4))) continue;
          m[2] = v3; m[3] = v4;
          og_emit(sink, m);
          count++;
        }
      }
      return count;
    }
    case OG_PATH4: {
      /* path a-b-c-d with root middle edge (b, c) = (v1, v2), v1 > v2;
       * a = v3 in N(b) \ {c}, d = v4 in N(c) \ {b, a} */
      for (uint64_t i = 0; i < DEG(g, v1); i++) {
        uint32_t a = ROW(g, v1)[i];
        if (a == v2) continue;
        if (induced && og_adjacent(g, a, v2)) continue;
        for (uint64_t j = 0; j < DEG(g, v2); j++) {
          uint32_t d = ROW(g, v2)[j];
          if (d == v1 || d == a) continue;
          if (induced && (og_adjacent(g, d, v1) || og_adjacent(g, d, a))) continue;
          m[2] = a; m[3] = d;
          og_emit(sink, m);
          count++;
        }
      }
      return count;
    }
    case OG_WEDGE: {
      /* centre v1, ends v2 > v3 */
      for (uint64_t i = 0; i < DEG(g, v1); i++) {
        uint32_t v3 = ROW(g, v1)[i];
        if (v3 >= v2) break;
        if (induced && og_adjacent(g, v2, v3)) continue;
        m[2] = v3;
        og_emit(sink, m);
        count++;
      }
      return count;
    }
    default:
      return 0;
  }
}

static uint32_t og_family_k(int family, uint32_t k) {
  switch (family) {
    case OG_CLIQUE: return k;
    case OG_WEDGE: return 3;
    default: return 4;
  }
}

/* Common setup: validate family, orient if needed, build Omega. */
typedef struct {
  og_g g, dag;
  int64_t* doff;
  uint32_t* dnbr;
  uint32_t *src, *dst;
  uint64_t ntasks;
  uint64_t maxdeg;
} og_ctx;

static void og_ctx_free(og_ctx* c) {
  free(c->doff); free(c->dnbr); free(c->src); free(c->dst);
}

static int og_ctx_init(og_ctx* c, const int64_t* off, const uint32_t* nbr, uint32_t n, int family,
                       uint32_t k) {
  memset(c, 0, sizeof(*c));
  c->g.n = n; c->g.off = off; c->g.nbr = nbr;
  int kind = og_task_kind(family);
  if (!kind) return -2;
  if (family == OG_CLIQUE && (k < 3 || k > 8)) return -2;
  for (uint32_t v = 0; v < n; v++) if (DEG(&c->g, v) > c->maxdeg) c->maxdeg = DEG(&c->g, v);
  if (family == OG_CLIQUE) {
    if (og_orient(&c->g, &c->doff, &c->dnbr)) return -1;
    c->dag.n = n; c->dag.off = c->doff; c->dag.nbr = c->dnbr;
    if (og_tasks(&c->dag, kind, &c->src, &c->dst, &c->ntasks)) { og_ctx_free(c); return -1; }
  } else {
    c->dag = c->g;
    if (og_tasks(&c->g, kind, &c->src, &c->dst, &c->ntasks)) { og_ctx_free(c); return -1; }
  }
  return 0;
}

/* |Omega| for the family (DAG arcs, lower pairs, or directed edges). */
int64_t og_num_tasks(const int64_t* off, const uint32_t* nbr, uint32_t n, int family, uint32_t k) {
  og_ctx c;
  int rc = og_ctx_init(&c, off, nbr, n, family, k);
  if (rc) return rc;
  int64_t t = (int64_t)c.ntasks;
  og_ctx_free(&c);
  return t;
}

/*
 * O2 count over root tasks [task_lo, task_hi) (clamped to |Omega|), with
 * `nthreads` OpenMP threads (1 = single-thread; integer sums make the result
 * independent of the thread count).  Returns 0, -1 (allocation) or -2 (bad
 * family / k).
 */
int og_count(const int64_t* off, const uint32_t* nbr, uint32_t n, int family, uint32_t k,
             int induced, uint64_t task_lo, uint64_t task_hi, int nthreads, uint64_t* out) {
  og_ctx c;
  int rc = og_ctx_init(&c, off, nbr, n, family, k);
  if (rc) return rc;
  if (task_hi > c.ntasks) task_hi = c.ntasks;
  if (task_lo > task_hi) task_lo = task_hi;
  uint64_t total = 0;
  int failed = 0;
  if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads) reduction(+ : total)
  {
    uint32_t* bufs[8];
    int ok = 1;
    for (int i = 0; i < 8; i++) {
      bufs[i] = (uint32_t*)malloc((c.maxdeg + 1) * sizeof(uint32_t));
      if (!bufs[i]) ok = 0;
    }
    if (!ok) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t t = (int64_t)task_lo; t < (int64_t)task_hi; t++)
        total += og_task(&c.g, &c.dag, family, k, induced, c.src[t], c.dst[t], bufs, NULL);
    }
    for (int i = 0; i < 8; i++) free(bufs[i]);
  }
  og_ctx_free(&c);
  if (failed) return -1;
  *out = total;
  return 0;
}

/*
 * O2 counts of several task ranges [ranges[2i], ranges[2i+1]) with one shared
 * setup (orientation, task list).  per_range[i] (if not NULL) receives range
 * i's count and *out their sum; *seconds the wall time of the counting phase
 * only (setup excluded, as preprocessing is excluded from the paper's
 * timings, Section 8).  Returns 0, -1 or -2.
 */
int og_count_ranges(const int64_t* off, const uint32_t* nbr, uint32_t n, int family, uint32_t k,
                    int induced, const uint64_t* ranges, uint64_t nranges, int nthreads,
                    uint64_t* per_range, uint64_t* out, double* seconds) {
  og_ctx c;
  int rc = og_ctx_init(&c, off, nbr, n, family, k);
  if (rc) return rc;
  if (nthreads < 1) nthreads = 1;
  struct timespec t0, t1;
  clock_gettime(CLOCK_MONOTONIC, &t0);
  uint64_t grand = 0;
  int failed = 0;
  for (uint64_t r = 0; r < nranges && !failed; r++) {
    uint64_t lo = ranges[2 * r], hi = ranges[2 * r + 1];
    if (hi > c.ntasks) hi = c.ntasks;
    if (lo > hi) lo = hi;
    uint64_t total = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : total)
    {
      uint32_t* bufs[8];
      int ok = 1;
      for (int i = 0; i < 8; i++) {
        bufs[i] = (uint32_t*)malloc((c.maxdeg + 1) * sizeof(uint32_t));
        if (!bufs[i]) ok = 0;
      }
      if (!ok) {
#pragma omp atomic write
        failed = 1;
      } else {
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = (int64_t)lo; t < (int64_t)hi; t++)
          total += og_task(&c.g, &c.dag, family, k, induced, c.src[t], c.dst[t], bufs, NULL);
      }
      for (int i = 0; i < 8; i++) free(bufs[i]);
    }
    if (per_range) per_range[r] = total;
    grand += total;
  }
  clock_gettime(CLOCK_MONOTONIC, &t1);
  og_ctx_free(&c);
  if (failed) return -1;
  *out = grand;
  *seconds = (double)(t1.tv_sec - t0.tv_sec) + 1e-9 * (double)(t1.tv_nsec - t0.tv_nsec);
  return 0;
}

/*
 * O2 listing over root tasks [task_lo, task_hi): writes up to `cap` matches of
 * k vertex IDs each (matching order) into `out`, in task order; *total gets the
 * number of matches.  Single-threaded.  Returns 0, -1 or -2.
 */
int og_list(const int64_t* off, const uint32_t* nbr, uint32_t n, int family, uint32_t k,
            int induced, uint64_t task_lo, uint64_t task_hi, uint32_t* out, uint64_t cap,
            uint64_t* total) {
  og_ctx c;
  int rc = og_ctx_init(&c, off, nbr, n, family, k);
  if (rc) return rc;
  if (task_hi > c.ntasks) task_hi = c.ntasks;
  if (task_lo > task_hi) task_lo = task_hi;
  uint32_t* bufs[8];
  for (int i = 0; i < 8; i++) bufs[i] = (uint32_t*)malloc((c.maxdeg + 1) * sizeof(uint32_t));
  og_sink sink = {out, cap, 0, og_family_k(family, k)};
  for (uint64_t t = task_lo; t < task_hi; t++)
    og_task(&c.g, &c.dag, family, k, induced, c.src[t], c.dst[t], bufs, &sink);
  for (int i = 0; i < 8; i++) free(bufs[i]);
  og_ctx_free(&c);
  *total = sink.written;
  return 0;
}

/* ------------------------------------------------------- O1 brute force --- */

/* Is (vertex set S of size k with adjacency bits `adj`) isomorphic to the
 * pattern (k vertices, adjacency bits `padj`)?  Tries all k! bijections.
 * adj bit (i*8+j) set iff i~j. */
static int og_iso(uint32_t k, uint64_t padj, uint64_t adj) {
  uint32_t perm[8];
  for (uint32_t i = 0; i < k; i++) perm[i] = i;
  for (;;) {
    int ok = 1;
    for (uint32_t i = 0; i < k && ok; i++)
      for (uint32_t j = i + 1; j < k; j++) {
        int pe = (int)((padj >> (i * 8 + j)) & 1);
        int ge = (int)((adj >> (perm[i] * 8 + perm[j])) & 1);
        if (pe != ge) { ok = 0; break; }
      }
    if (ok) return 1;
    /* next permutation (lexicographic) */
    int i = (int)k - 2;
    while (i >= 0 && perm[i] > perm[i + 1]) i--;
    if (i < 0) return 0;
    int j = (int)k - 1;
    while (perm[j] < perm[i]) j--;
    uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    for (int a = i + 1, b = (int)k - 1; a < b; a++, b--) { t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
  }
}

/*
 * O1: count subgraphs of G isomorphic to the pattern P (k <= 8 vertices,
 * edges pe[2*i], pe[2*i+1]) by the definitions of Section 2.1:
 *   induced = 1: #{S : |S| = k, G[S] ~= P}
 *   induced = 0: #{(S, F) : |S| = k, F ⊆ E(G[S]), (S, F) ~= P}
 * Exponential; intended for n <= ~14.  Returns the count.
 */
uint64_t og_brute(const int64_t* off, const uint32_t* nbr, uint32_t n, uint32_t k,
                  const uint8_t* pe, uint32_t npe, int induced) {
  og_g g = {n, off, nbr};
  if (k < 1 || k > 8 || n < k) return 0;
  uint64_t padj = 0;
  for (uint32_t i = 0; i < npe; i++) {
    uint32_t a = pe[2 * i], b = pe[2 * i + 1];
    padj |= 1ULL << (a * 8 + b);
    padj |= 1ULL << (b * 8 + a);
  }
  uint32_t S[8];
  for (uint32_t i = 0; i < k; i++) S[i] = i;
  uint64_t count = 0;
  for (;;) {
    /* edges of G[S] */
    uint32_t ei[28], ej[28], ne = 0;
    for (uint32_t i = 0; i < k; i++)
      for (uint32_t j = i + 1; j < k; j++)
        if (og_adjacent(&g, S[i], S[j])) { ei[ne] = i; ej[ne] = j; ne++; }
    if (induced) {
      uint64_t adj = 0;
      for (uint32_t e = 0; e < ne; e++)
        adj |= (1ULL << (ei[e] * 8 + ej[e])) | (1ULL << (ej[e] * 8 + ei[e]));
      if (ne == npe && og_iso(k, padj, adj)) count++;
    } else if (ne >= npe) {
      /* every subset F of E(G[S]) with |F| = |E(P)| */
      for (uint64_t mask = 0; mask < (1ULL << ne); mask++) {
        if ((uint32_t)__builtin_popcountll(mask) != npe) continue;
        uint64_t adj = 0;
        for (uint32_t e = 0; e < ne; e++)
          if (mask >> e & 1) adj |= (1ULL << (ei[e] * 8 + ej[e])) | (1ULL << (ej[e] * 8 + ei[e]));
        if (og_iso(k, padj, adj)) count++;
      }
    }
    /* next k-combination of 0..n-1 */
    int i = (int)k - 1;
    while (i >= 0 && S[i] == n - k + (uint32_t)i) i--;
    if (i < 0) break;
    S[i]++;
    for (uint32_t j = (uint32_t)i + 1; j < k; j++) S[j] = S[j - 1] + 1;
  }
  return count;
}

/* Number of connected k-vertex subsets (k <= 8), by brute force. */
uint64_t og_connected_subsets(const int64_t* off, const uint32_t* nbr, uint32_t n, uint32_t k) {
  og_g g = {n, off, nbr};
  if (k < 1 || k > 8 || n < k) return 0;
  uint32_t S[8];
  for (uint32_t i = 0; i < k; i++) S[i] = i;
  uint64_t count = 0;
  for (;;) {
    uint32_t seen = 1, frontier = 1;
    while (frontier) {
      uint32_t next = 0;
      for (uint32_t i = 0; i < k; i++)
        if (frontier >> i & 1)
          for (uint32_t j = 0; j < k; j++)
            if (!(seen >> j & 1) && og_adjacent(&g, S[i], S[j])) next |= 1u << j;
      seen |= next;
      frontier = next;
    }
    if (seen == (1u << k) - 1) count++;
    int i = (int)k - 1;
    while (i >= 0 && S[i] == n - k + (uint32_t)i) i--;
    if (i < 0) break;
    S[i]++;
    for (uint32_t j = (uint32_t)i + 1; j < k; j++) S[j] = S[j - 1] + 1;
  }
  return count;
}

/* --------------------------------------- O1b injective homomorphisms --- */

/* |Aut(P)|: permutations of the k pattern vertices that map edges to edges
 * (padj bit i*8+j set iff i~j). */
uint64_t og_automorphisms(uint32_t k, const uint8_t* pe, uint32_t npe) {
  if (k < 1 || k > 8) return 0;
  uint64_t padj = 0;
  for (uint32_t i = 0; i < npe; i++) {
    uint32_t a = pe[2 * i], b = pe[2 * i + 1];
    padj |= 1ULL << (a * 8 + b);
    padj |= 1ULL << (b * 8 + a);
  }
  uint32_t perm[8];
  for (uint32_t i = 0; i < k; i++) perm[i] = i;
  uint64_t count = 0;
  for (;;) {
    int ok = 1;
    for (uint32_t i = 0; i < k && ok; i++)
      for (uint32_t j = i + 1; j < k; j++)
        if (((padj >> (i * 8 + j)) & 1) != ((padj >> (perm[i] * 8 + perm[j])) & 1)) { ok = 0; break; }
    count += (uint64_t)ok;
    int i = (int)k - 2;
    while (i >= 0 && perm[i] > perm[i + 1]) i--;
    if (i < 0) break;
    int j = (int)k - 1;
    while (perm[j] < perm[i]) j--;
    uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    for (int a = i + 1, b = (int)k - 1; a < b; a++, b--) { t = perm[a]; perm[a] = perm[b]; perm[b] = t; }
  }
  return count;
}

typedef struct {
  const og_g* g;
  uint32_t k;
  uint64_t padj;
  int induced;
  uint32_t ord[8];    /* pattern vertices in visiting order */
  int anchor[8];      /* a visited pattern neighbour of ord[i] (-1: none) */
} og_hom;

/* Extend the partial map phi (pattern vertex -> data vertex) of the first i
 * visited pattern vertices; returns the number of complete injective maps. */
static uint64_t og_hom_extend(const og_hom* h, uint32_t i, uint32_t* phi) {
  if (i == h->k) return 1;
  const uint32_t u = h->ord[i];
  const uint32_t* cand;
  uint64_t nc;
  if (h->anchor[i] >= 0) {
    cand = ROW(h->g, phi[h->anchor[i]]);
    nc = DEG(h->g, phi[h->anchor[i]]);
  } else {
    cand = NULL;
    nc = h->g->n;
  }
  uint64_t total = 0;
  for (uint64_t c = 0; c < nc; c++) {
    const uint32_t x = cand ? cand[c] : (uint32_t)c;
    int ok = 1;
    for (uint32_t j = 0; j < i && ok; j++) {
      const uint32_t w = h->ord[j];
      if (phi[w] == x) { ok = 0; break; }
      const int pe = (int)((h->padj >> (u * 8 + w)) & 1);
      if (pe || h->induced) {
        const int ge = og_adjacent(h->g, x, phi[w]);
        if (pe != ge) ok = 0;
      }
    }
    if (!ok) continue;
    phi[u] = x;
    total += og_hom_extend(h, i + 1, phi);
  }
  return total;
}

/*
 * Number of injective maps phi: V(P) -> V(G) with u~w in P => phi(u)~phi(w)
 * in G (and, if induced, u!~w => phi(u)!~phi(w)): the embeddings of Section
 * 2.1 before symmetry breaking.  Pattern vertices are visited in BFS order
 * from vertex 0, each drawing its candidates from the neighbours of an
 * already mapped pattern neighbour (any vertex when it has none).  The first
 * vertex's images are split over `nthreads` OpenMP threads.
 */
uint64_t og_injhom(const int64_t* off, const uint32_t* nbr, uint32_t n, uint32_t k,
                   const uint8_t* pe, uint32_t npe, int induced, int nthreads) {
  og_g g = {n, off, nbr};
  if (k < 1 || k > 8 || n < k) return 0;
  og_hom h;
  h.g = &g;
  h.k = k;
  h.padj = 0;
  h.induced = induced;
  for (uint32_t i = 0; i < npe; i++) {
    uint32_t a = pe[2 * i], b = pe[2 * i + 1];
    h.padj |= 1ULL << (a * 8 + b);
    h.padj |= 1ULL << (b * 8 + a);
  }
  /* BFS order over pattern vertices (restarting at the lowest unvisited) */
  uint32_t seen = 0, cnt = 0;
  while (cnt < k) {
    uint32_t r = 0;
    while (seen >> r & 1) r++;
    seen |= 1u << r;
    h.ord[cnt] = r;
    h.anchor[cnt] = -1;
    uint32_t head = cnt++;
    while (head < cnt) {
      const uint32_t u = h.ord[head++];
      for (uint32_t w = 0; w < k; w++)
        if (!(seen >> w & 1) && ((h.padj >> (u * 8 + w)) & 1)) {
          seen |= 1u << w;
          h.ord[cnt] = w;
          h.anchor[cnt] = (int)u;
          cnt++;
        }
    }
  }
  uint64_t total = 0;
  const uint32_t r0 = h.ord[0];
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 16) reduction(+ : total)
  for (int64_t x = 0; x < (int64_t)n; x++) {
    uint32_t phi[8];
    phi[r0] = (uint32_t)x;
    total += og_hom_extend(&h, 1, phi);
  }
  return total;
}

/* ------------------------------------------------ O3 closed forms --- */

/*
 * Pattern-decomposition identities (Section 5.4 counting-only pruning,
 * generalised).  With d_v the degree, t_e the triangles on edge e, t_v the
 * triangles at v, T the triangle count and c_xy = |N(x) ∩ N(y)|:
 *   out[0]  T                                  (sum t_e / 3)
 *   out[1]  wedge, edge-induced = sum_v C(d_v, 2)
 *   out[2]  3-star, edge-induced = sum_v C(d_v, 3)
 *   out[3]  4-path, edge-induced = sum_{uv in E} (d_u-1)(d_v-1) - 3T
 *   out[4]  tailed-triangle, edge-induced = sum_v t_v (d_v - 2)
 *   out[5]  diamond, edge-induced = sum_e C(t_e, 2)
 *   out[6]  4-cycle, edge-induced = (1/2) sum_{x<y} C(c_xy, 2)
 *   out[7]  wedge, vertex-induced = out[1] - 3T
 * (4-clique counts need enumeration; the caller combines them with these via
 * og_motif4_inversion.)  Uses `nthreads` OpenMP threads.  Returns 0 or -1.
 */
int og_identities(const int64_t* off, const uint32_t* nbr, uint32_t n, int nthreads, uint64_t* out) {
  og_g g = {n, off, nbr};
  if (nthreads < 1) nthreads = 1;
  uint64_t* tv = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t)); /* 2 t_v */
  if (!tv) return -1;
  uint64_t sum_te = 0, dia = 0, p4 = 0, w = 0, s3 = 0, c4x2 = 0;
  int failed = 0;
#pragma omp parallel num_threads(nthreads) reduction(+ : sum_te, dia, p4)
  {
#pragma omp for schedule(dynamic, 256)
    for (int64_t u = 0; u < (int64_t)n; u++) {
      for (uint64_t i = 0; i < DEG(&g, u); i++) {
        uint32_t v = ROW(&g, u)[i];
        if (v >= u) break; /* each undirected edge once (v < u) */
        uint64_t te = og_intersect(ROW(&g, u), DEG(&g, u), ROW(&g, v), DEG(&g, v), NULL);
        sum_te += te;
        dia += te ? te * (te - 1) / 2 : 0; /* C(t_e, 2) */
        p4 += (DEG(&g, u) - 1) * (DEG(&g, v) - 1);
#pragma omp atomic
        tv[u] += te;
#pragma omp atomic
        tv[v] += te;
      }
    }
  }
  uint64_t T = sum_te / 3, tt = 0;
  for (uint32_t v = 0; v < n; v++) {
    uint64_t d = DEG(&g, v);
    w += d ? d * (d - 1) / 2 : 0;
    if (d >= 3) s3 += d * (d - 1) * (d - 2) / 6;
    if (d >= 2) tt += (tv[v] / 2) * (d - 2);
  }
  /* 4-cycles via co-degrees: for each x, count c_xy over wedges x-w-y, y<x */
#pragma omp parallel num_threads(nthreads) reduction(+ : c4x2)
  {
    uint32_t* cnt = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
    uint32_t* touched = (uint32_t*)malloc(((size_t)n + 1) * sizeof(uint32_t));
    if (!cnt || !touched) {
#pragma omp atomic write
      failed = 1;
    } else {
#pragma omp for schedule(dynamic, 64)
      for (int64_t x = 0; x < (int64_t)n; x++) {
        uint64_t nt = 0;
        for (uint64_t i = 0; i < DEG(&g, x); i++) {
          uint32_t wv = ROW(&g, x)[i];
          for (uint64_t j = 0; j < DEG(&g, wv); j++) {
            uint32_t y = ROW(&g, wv)[j];
            if (y >= (uint32_t)x) break;
            if (cnt[y]++ == 0) touched[nt++] = y;
          }
        }
        for (uint64_t i = 0; i < nt; i++) {
          uint64_t c = cnt[touched[i]];
          c4x2 += c * (c - 1) / 2;
          cnt[touched[i]] = 0;
        }
      }
    }
    free(cnt); free(touched);
  }
  free(tv);
  if (failed) return -1;
  out[0] = T;
  out[1] = w;
  out[2] = s3;
  out[3] = p4 - 3 * T;
  out[4] = tt;
  out[5] = dia;
  out[6] = c4x2 / 2;
  out[7] = w - 3 * T;
  return 0;
}

/*
 * Edge-induced -> vertex-induced inversion for the six connected 4-vertex
 * patterns.  in[] = edge-induced counts {4-path, 3-star, 4-cycle,
 * tailed-triangle, diamond, 4-clique}; out[] = vertex-induced counts in the
 * same order.  Each coefficient is the number of edge-induced copies of one
 * pattern inside the vertex-induced other (e.g. a 4-clique holds 6 diamonds,
 * 3 four-cycles, 12 tailed triangles, 4 three-stars and 12 four-paths).
 */
void og_motif4_inversion(const uint64_t* in, uint64_t* out) {
  uint64_t P4 = in[0], S3 = in[1], C4 = in[2], TT = in[3], DI = in[4], K4 = in[5];
  uint64_t k4 = K4;
  uint64_t di = DI - 6 * k4;
  uint64_t c4 = C4 - di - 3 * k4;
  uint64_t tt = TT - 4 * di - 12 * k4;
  uint64_t s3 = S3 - tt - 2 * di - 4 * k4;
  uint64_t p4 = P4 - 2 * tt - 4 * c4 - 6 * di - 12 * k4;
  out[0] = p4; out[1] = s3; out[2] = c4; out[3] = tt; out[4] = di; out[5] = k4;
}
