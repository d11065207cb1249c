// analyzer.cu — the pattern analyzer for patterns outside the plan families
// (Section 4.2): a matching order picked by a cost model over all valid
// orders, and a symmetry order generated along that matching order.
//
// Matching order.  A valid order starts with an edge (the root task) and
// adds, at every later position, a pattern vertex adjacent to an earlier one,
// so its candidates come from intersecting neighbour lists.  The cost model
// is the usual random-graph estimate: with n vertices, average degree d and
// edge probability p = d / n, a position joined to c earlier positions reads
// c neighbour lists (c * d entries) per partial match and multiplies the
// number of partial matches by d * p^(c-1).  The order with the least total
// list reading wins (ties: a highest-degree first vertex, then the
// lexicographically smallest order).
//
// Symmetry order.  Walking the matching order, each pattern vertex u is made
// the largest of its orbit under the automorphisms that fix every earlier
// vertex (data vertex of u > data vertex of every other orbit member), and the
// group shrinks to the stabiliser of u.  Every orbit member lies later in the
// order (earlier vertices are fixed points), so each constraint is an upper
// bound on a later position, and each subgraph is matched exactly once: the
// embeddings of one subgraph form one orbit of Aut(P), and the constraints
// select one representative of it.  For the diamond with the chord matched
// first this gives v1 > v2 and v3 > v4, the order of Section 2.2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gpm_internal.cuh"

namespace gpm {

namespace {

using Perm = std::vector<int>;

bool adjacent(const uint32_t* adj, int a, int b) { return (adj[a] >> b) & 1u; }

bool connected_pattern(uint32_t k, const uint32_t* adj) {
  uint32_t seen = 1, frontier = 1;
  while (frontier) {
    uint32_t next = 0;
    for (uint32_t i = 0; i < k; i++)
      if ((frontier >> i) & 1u) next |= adj[i] & ~seen;
    seen |= next;
    frontier = next;
  }
  return seen == (1u << k) - 1;
}

std::vector<Perm> automorphisms(uint32_t k, const uint32_t* adj) {
  std::vector<Perm> out;
  Perm p(k);
  for (uint32_t i = 0; i < k; i++) p[i] = (int)i;
  do {
    bool ok = true;
    for (uint32_t i = 0; i < k && ok; i++)
      for (uint32_t j = i + 1; j < k; j++)
        if (adjacent(adj, (int)i, (int)j) != adjacent(adj, p[i], p[j])) { ok = false; break; }
    if (ok) out.push_back(p);
  } while (std::next_permutation(p.begin(), p.end()));
  return out;
}

// Estimated neighbour-list entries read by the nested loops of an order.
double order_cost(uint32_t k, const uint32_t* adj, const Perm& ord, double n, double d) {
  const double p = n > 0 ? std::min(1.0, d / n) : 1.0;
  double partial = n * d;  // matches of the root edge
  double cost = 0;
  for (uint32_t t = 2; t < k; t++) {
    int c = 0;
    for (uint32_t s = 0; s < t; s++) c += adjacent(adj, ord[t], ord[s]) ? 1 : 0;
    cost += partial * c * d;
    partial *= d * std::pow(p, c - 1);
  }
  return cost;
}

bool valid_order(uint32_t k, const uint32_t* adj, const Perm& ord) {
  if (!adjacent(adj, ord[0], ord[1])) return false;
  for (uint32_t t = 2; t < k; t++) {
    bool ok = false;
    for (uint32_t s = 0; s < t && !ok; s++) ok = adjacent(adj, ord[t], ord[s]);
    if (!ok) return false;
  }
  return true;
}

}  // namespace

bool analyze_pattern(uint32_t k, const std::vector<std::pair<int, int>>& edges, int induced,
                     double n, double avg_degree, GenTable* T, std::string* why) {
  if (k < 3 || k > (uint32_t)kGenMaxK) {
    *why = "the generic plan needs 3 to 8 pattern vertices";
    return false;
  }
  uint32_t adj[kGenMaxK] = {};
  for (auto& e : edges) {
    if (e.first < 0 || e.second < 0 || e.first >= (int)k || e.second >= (int)k || e.first == e.second) {
      *why = "pattern edge out of range or a self-loop";
      return false;
    }
    adj[e.first] |= 1u << e.second;
    adj[e.second] |= 1u << e.first;
  }
  if (!connected_pattern(k, adj)) {
    *why = "the pattern is not connected";
    return false;
  }
  // matching order: every valid order, least estimated cost
  Perm ord(k), best;
  for (uint32_t i = 0; i < k; i++) ord[i] = (int)i;
  double best_cost = 0;
  int best_deg = -1;
  do {
    if (!valid_order(k, adj, ord)) continue;
    const double c = order_cost(k, adj, ord, n, avg_degree);
    const int d0 = __builtin_popcount(adj[ord[0]]);
    if (best.empty() || c < best_cost * (1 - 1e-12) ||
        (c <= best_cost * (1 + 1e-12) && d0 > best_deg)) {
      best = ord;
      best_cost = c;
      best_deg = d0;
    }
  } while (std::next_permutation(ord.begin(), ord.end()));
  // symmetry order along the matching order (stabiliser chain of Aut(P))
  std::vector<Perm> group = automorphisms(k, adj);
  int pos[kGenMaxK];
  for (uint32_t t = 0; t < k; t++) pos[best[t]] = (int)t;
  memset(T, 0, sizeof(*T));
  T->k = k;
  T->induced = induced ? 1u : 0u;
  for (uint32_t t = 0; t < k; t++) {
    const int u = best[t];
    uint32_t orbit = 0;
    for (auto& g : group) orbit |= 1u << g[u];
    for (int w = 0; w < (int)k; w++) {
      if (w == u || !((orbit >> w) & 1u)) continue;
      const int pw = pos[w];  // later than t: earlier vertices are fixed points
      T->U[pw][T->nU[pw]++] = (uint8_t)t;
    }
    std::vector<Perm> stab;
    for (auto& g : group)
      if (g[u] == u) stab.push_back(g);
    group.swap(stab);
  }
  for (uint32_t t = 0; t < k; t++) {
    T->order[t] = (uint8_t)best[t];
    for (uint32_t s = 0; s < t; s++) {
      if (adjacent(adj, best[t], best[s])) T->E[t][T->nE[t]++] = (uint8_t)s;
      else T->N[t][T->nN[t]++] = (uint8_t)s;
    }
  }
  T->root_lower = (T->nU[1] == 1 && T->U[1][0] == 0) ? 1u : 0u;
  return true;
}

// "order: u0 u2 u1 u3; symmetry: v0>v1 v2>v3; tasks: v0>v1" (positions are
// numbered in matching order, u are pattern vertices).
std::string describe_gen(const GenTable& T) {
  std::string s = "order:";
  for (uint32_t t = 0; t < T.k; t++) s += " u" + std::to_string(T.order[t]);
  s += "; symmetry:";
  bool any = false;
  for (uint32_t t = 0; t < T.k; t++)
    for (uint32_t i = 0; i < T.nU[t]; i++) {
      s += " v" + std::to_string(T.U[t][i]) + ">v" + std::to_string(t);
      any = true;
    }
  if (!any) s += " none";
  s += T.root_lower ? "; tasks: pairs v0>v1" : "; tasks: every directed edge";
  s += T.induced ? "; vertex-induced" : "; edge-induced";
  return s;
}

}  // namespace gpm
