/*
 * graphgen.c — seeded synthetic data graphs for the enumeration library, its
 * oracle and its benchmark.
 *
 * This module only MAKES INPUTS.  It contains none of the pattern-matching
 * arithmetic: no set operations, no orientation, no counting.  Both the CUDA
 * path and the CPU oracle consume the CSR arrays produced here, and neither
 * shares any other code.
 *
 * Random numbers.  Every random draw is a pure function of (seed, stream,
 * index): the SplitMix64 finaliser (Steele, Lea & Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to a Weyl sequence
 * position.  Draw i therefore does not depend on how many threads produced
 * draws 0..i-1, and the same seed gives the same graph on x86-64 and AArch64.
 * Probabilities are compared as 32-bit fixed-point integers, never as floats,
 * so no rounding mode or FMA contraction can change a decision.  The one
 * floating-point step (Chung-Lu weights) is quantised to integers before use.
 *
 * Output format.  A simple undirected graph in CSR: int64 offsets[n+1],
 * uint32 nbrs[offsets[n]], each row sorted ascending, both directions of every
 * edge present, no self-loops, no duplicates.  (The paper's loader produces
 * the same shape: CSR with ascending neighbour lists, Section 4.2.)
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- RNG --- */

static inline uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Draw `idx` of stream `stream` under `seed`. */
uint64_t gg_rand(uint64_t seed, uint64_t stream, uint64_t idx) {
  uint64_t base = gg_mix64(seed ^ gg_mix64(stream + 0x632BE59BD9B4E019ULL));
  return gg_mix64(base + (idx + 1) * 0x9E3779B97F4A7C15ULL);
}

/* Uniform integer in [0, bound) by 64x64->128 multiply-high (Lemire). The
 * tiny bias (< bound / 2^64) is irrelevant here and identical on all hosts. */
static inline uint64_t gg_below(uint64_t r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)r * (unsigned __int128)bound) >> 64);
}

enum { GG_STREAM_ER = 1, GG_STREAM_RMAT = 2, GG_STREAM_PERM = 3, GG_STREAM_CL = 4,
       GG_STREAM_SMALL = 5 };

/* ------------------------------------------------------ small helpers --- */

static void gg_sort_u32(uint32_t* a, int64_t n);

static void gg_insertion(uint32_t* a, int64_t n) {
  for (int64_t i = 1; i < n; i++) {
    uint32_t x = a[i];
    int64_t j = i - 1;
    while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; j--; }
    a[j + 1] = x;
  }
}

/* Three-way quicksort (robust to the many duplicates of R-MAT hub rows). */
static void gg_sort_u32(uint32_t* a, int64_t n) {
  while (n > 24) {
    uint32_t x = a[0], y = a[n / 2], z = a[n - 1];
    uint32_t p = (x < y) ? ((y < z) ? y : ((x < z) ? z : x)) : ((x < z) ? x : ((y < z) ? z : y));
    int64_t lt = 0, i = 0, gt = n - 1;
    while (i <= gt) {
      if (a[i] < p) { uint32_t t = a[lt]; a[lt] = a[i]; a[i] = t; lt++; i++; }
      else if (a[i] > p) { uint32_t t = a[gt]; a[gt] = a[i]; a[i] = t; gt--; }
      else i++;
    }
    /* recurse on the smaller side, loop on the larger */
    int64_t nl = lt, nr = n - (gt + 1);
    if (nl < nr) { gg_sort_u32(a, nl); a += gt + 1; n = nr; }
    else { gg_sort_u32(a + gt + 1, nr); n = nl; }
  }
  gg_insertion(a, n);
}

void gg_free(void* p) { free(p); }

/* -------------------------------------------------------- CSR builder --- */

/*
 * Build a simple undirected CSR from `npairs` endpoint pairs (us[i], vs[i]).
 * Self-loops are dropped, both directions are inserted, rows are sorted and
 * duplicates removed.  On success *nbr_out is a malloc'ed array of *nnz_out
 * entries (free with gg_free) and off_out[0..n] is filled.  Returns 0, or -1
 * on allocation failure / out-of-range endpoint.
 */
int gg_build_csr(uint32_t n, const uint32_t* us, const uint32_t* vs, uint64_t npairs,
                 int64_t* off_out, uint32_t** nbr_out, uint64_t* nnz_out) {
  int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) return -1;
  for (uint64_t i = 0; i < npairs; i++) {
    uint32_t u = us[i], v = vs[i];
    if (u >= n || v >= n) { free(deg); return -1; }
    if (u == v) continue;
    deg[u]++; deg[v]++;
  }
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) { free(deg); return -1; }
  off[0] = 0;
  for (uint32_t v = 0; v < n; v++) off[v + 1] = off[v] + deg[v];
  uint64_t total = (uint64_t)off[n];
  uint32_t* tmp = (uint32_t*)malloc((total ? total : 1) * sizeof(uint32_t));
  if (!tmp) { free(deg); free(off); return -1; }
  memcpy(deg, off, (size_t)n * sizeof(int64_t)); /* deg reused as cursor */
  for (uint64_t i = 0; i < npairs; i++) {
    uint32_t u = us[i], v = vs[i];
    if (u == v) continue;
    tmp[deg[u]++] = v;
    tmp[deg[v]++] = u;
  }
  /* sort + dedup each row in place; new degree in deg[] */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t v = 0; v < (int64_t)n; v++) {
    uint32_t* row = tmp + off[v];
    int64_t len = off[v + 1] - off[v];
    gg_sort_u32(row, len);
    int64_t w = 0;
    for (int64_t i = 0; i < len; i++)
      if (w == 0 || row[i] != row[w - 1]) row[w++] = row[i];
    deg[v] = w;
  }
  off_out[0] = 0;
  for (uint32_t v = 0; v < n; v++) off_out[v + 1] = off_out[v] + deg[v];
  uint64_t nnz = (uint64_t)off_out[n];
  uint32_t* nbr = (uint32_t*)malloc((nnz ? nnz : 1) * sizeof(uint32_t));
  if (!nbr) { free(deg); free(off); free(tmp); return -1; }
#pragma omp parallel for schedule(dynamic, 4096)
  for (int64_t v = 0; v < (int64_t)n; v++)
    memcpy(nbr + off_out[v], tmp + off[v], (size_t)deg[v] * sizeof(uint32_t));
  free(deg); free(off); free(tmp);
  *nbr_out = nbr;
  *nnz_out = nnz;
  return 0;
}

/* ------------------------------------------------- ID permutation --- */

/* Seeded Fisher-Yates permutation of 0..n-1 (Graph500-style relabelling). */
void gg_permutation(uint32_t n, uint64_t seed, uint32_t* perm) {
  for (uint32_t i = 0; i < n; i++) perm[i] = i;
  for (uint32_t i = n; i > 1; i--) {
    uint64_t j = gg_below(gg_rand(seed, GG_STREAM_PERM, i), i);
    uint32_t t = perm[i - 1]; perm[i - 1] = perm[j]; perm[j] = t;
  }
}

void gg_apply_perm(const uint32_t* perm, uint32_t* xs, uint64_t count) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)count; i++) xs[i] = perm[xs[i]];
}

/* --------------------------------------------------- Erdős–Rényi G(n,m) --- */

/*
 * Exactly m distinct unordered pairs {u,v}, u != v, uniform without
 * replacement: draw candidate pairs in a fixed index order and keep the first
 * m distinct ones (an open-addressing set on the 64-bit key).  Requires
 * m <= n(n-1)/2.  Writes us[0..m), vs[0..m).  Returns 0 or -1.
 */
int gg_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t* us, uint32_t* vs) {
  if (n < 2 || m > (uint64_t)n * (n - 1) / 2) return -1;
  uint64_t cap = 16;
  while (cap < 2 * m + 16) cap <<= 1;
  uint64_t* table = (uint64_t*)malloc(cap * sizeof(uint64_t));
  if (!table) return -1;
  memset(table, 0xFF, cap * sizeof(uint64_t));
  uint64_t have = 0, draw = 0;
  while (have < m) {
    uint64_t r = gg_rand(seed, GG_STREAM_ER, draw++);
    uint32_t u = (uint32_t)gg_below(r, n);
    uint32_t v = (uint32_t)gg_below(gg_rand(seed, GG_STREAM_ER + 100, draw), n);
    if (u == v) continue;
    if (u > v) { uint32_t t = u; u = v; v = t; }
    uint64_t key = ((uint64_t)u << 32) | v;
    uint64_t h = gg_mix64(key) & (cap - 1);
    while (table[h] != UINT64_MAX && table[h] != key) h = (h + 1) & (cap - 1);
    if (table[h] == key) continue;
    table[h] = key;
    us[have] = u; vs[have] = v; have++;
  }
  free(table);
  return 0;
}

/* ------------------------------------------------------------- R-MAT --- */

/*
 * R-MAT (Chakrabarti, Zhan & Faloutsos 2004) edge draws at `scale` levels with
 * quadrant probabilities (a, b, c, 1-a-b-c) given as 32-bit fixed-point
 * thresholds ta <= tb <= tc (= round(a*2^32), round((a+b)*2^32),
 * round((a+b+c)*2^32)).  Quadrant a keeps both bits 0, b sets the column bit,
 * c the row bit, d both.  Endpoints >= n_limit are rejected and the whole
 * draw is repeated with the next attempt counter (n_limit = 2^scale accepts
 * all).  Writes ndraws pairs; no dedup here.
 */
void gg_rmat(uint32_t scale, uint64_t ndraws, uint32_t ta, uint32_t tb, uint32_t tc,
             uint32_t n_limit, uint64_t seed, uint32_t* us, uint32_t* vs) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < (int64_t)ndraws; i++) {
    for (uint64_t attempt = 0;; attempt++) {
      uint32_t u = 0, v = 0;
      uint64_t r = 0;
      for (uint32_t l = 0; l < scale; l++) {
        if ((l & 1) == 0)
          r = gg_rand(seed ^ (attempt * 0x2545F4914F6CDD1DULL), GG_STREAM_RMAT,
                      (uint64_t)i * 64 + (l >> 1));
        uint32_t x = (uint32_t)(r >> ((l & 1) ? 32 : 0));
        uint32_t ubit = 0, vbit = 0;
        if (x < ta) { }
        else if (x < tb) { vbit = 1; }
        else if (x < tc) { ubit = 1; }
        else { ubit = 1; vbit = 1; }
        u = (u << 1) | ubit;
        v = (v << 1) | vbit;
      }
      if (u < n_limit && v < n_limit) { us[i] = u; vs[i] = v; break; }
    }
  }
}

/* --------------------------------------------------------- Chung–Lu --- */

/*
 * Chung–Lu power-law endpoint pairs.  Vertex i has weight
 *   w_i = wmax * (1 + i/i0)^(-1/(gamma-1)),
 * quantised to the integer q_i = floor(16 w_i + 1/2) (so that an ULP of
 * difference in pow() between hosts cannot change a draw), and each endpoint
 * is drawn independently with probability proportional to q_i by inverse CDF
 * over the integer prefix sums.  Writes npairs pairs (loops and duplicates
 * are removed later by the CSR builder).  Returns 0 or -1.
 */
int gg_chung_lu(uint32_t n, uint64_t npairs, double wmax, double i0, double gamma,
                uint64_t seed, uint32_t* us, uint32_t* vs) {
  uint64_t* cdf = (uint64_t*)malloc((size_t)n * sizeof(uint64_t));
  if (!cdf) return -1;
  double expo = -1.0 / (gamma - 1.0);
  uint64_t acc = 0;
  for (uint32_t i = 0; i < n; i++) {
    double w = wmax * pow(1.0 + (double)i / i0, expo);
    uint64_t q = (uint64_t)(w * 16.0 + 0.5);
    if (q == 0) q = 1;
    acc += q;
    cdf[i] = acc; /* inclusive prefix */
  }
  uint64_t total = acc;
#pragma omp parallel for schedule(static)
  for (int64_t p = 0; p < (int64_t)npairs; p++) {
    for (int side = 0; side < 2; side++) {
      uint64_t x = gg_below(gg_rand(seed, GG_STREAM_CL, 2 * (uint64_t)p + side), total);
      /* smallest i with cdf[i] > x */
      uint32_t lo = 0, hi = n - 1;
      while (lo < hi) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (cdf[mid] > x) hi = mid; else lo = mid + 1;
      }
      if (side == 0) us[p] = lo; else vs[p] = lo;
    }
  }
  free(cdf);
  return 0;
}

/* ----------------------------------------- small random graphs (tests) --- */

/* G(n,p) with p = p_num/2^32 as a fixed-point threshold; writes pairs u<v,
 * returns the count.  Caller provides room for n(n-1)/2 pairs. */
uint64_t gg_gnp(uint32_t n, uint32_t p_fixed, uint64_t seed, uint32_t* us, uint32_t* vs) {
  uint64_t k = 0, idx = 0;
  for (uint32_t u = 0; u < n; u++)
    for (uint32_t v = u + 1; v < n; v++) {
      uint32_t x = (uint32_t)gg_rand(seed, GG_STREAM_SMALL, idx++);
      if (x < p_fixed) { us[k] = u; vs[k] = v; k++; }
    }
  return k;
}

/* FNV-1a over a byte range, used to check that two hosts built the same graph. */
uint64_t gg_fnv1a(const void* data, uint64_t nbytes, uint64_t h) {
  const unsigned char* p = (const unsigned char*)data;
  if (h == 0) h = 0xCBF29CE484222325ULL;
  for (uint64_t i = 0; i < nbytes; i++) { h ^= p[i]; h *= 0x100000001B3ULL; }
  return h;
}
