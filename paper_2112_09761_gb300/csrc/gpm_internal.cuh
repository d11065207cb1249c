// gpm_internal.cuh — internal types shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/gpm.h"

namespace gpm {

// Plan families (Section 2.1 problem set; Section 4.2 pattern analyzer).
enum Family : int {
  kClique = 1,          // k-clique on the degree-oriented DAG (k = 3..8)
  kDiamond = 2,         // chord (v1,v2), v3 > v4 in N(v1) ∩ N(v2)
  kCycle4 = 3,          // v1 max, v2 > v4 in N(v1), v3 in N(v2) ∩ N(v4)
  kTailedTriangle = 4,  // triangle v1 v2 v3 (v3 < v2) + tail v4 on v1
  kStar3 = 5,           // centre v1, leaves v2 > v3 > v4
  kPath4 = 6,           // v3 - v1 - v2 - v4 with v1 > v2
  kWedge = 7,           // centre v1, ends v2 > v3
  kGeneric = 8          // any connected pattern: the generic interpreter (GenTable)
};

// Search plan of the generic interpreter (Section 4.2 pattern analyzer): the
// matching order and the symmetry order of a connected pattern with 3..8
// vertices, as per-position lists of earlier positions.  Position t's
// candidates are the common neighbours of the matches of E[t], below the
// matches of U[t], distinct from the matches of N[t] and, vertex-induced,
// adjacent to none of them.
constexpr int kGenMaxK = 8;
struct GenTable {
  uint32_t k;
  uint32_t induced;
  uint32_t root_lower;             // symmetry order holds v0 > v1: root tasks are pairs v1 < v0
  uint8_t order[kGenMaxK];         // pattern vertex matched at each position
  uint8_t nE[kGenMaxK], E[kGenMaxK][kGenMaxK];  // earlier positions adjacent in the pattern
  uint8_t nN[kGenMaxK], N[kGenMaxK][kGenMaxK];  // earlier positions not adjacent
  uint8_t nU[kGenMaxK], U[kGenMaxK][kGenMaxK];  // earlier positions s with v_t < v_s
};

// Root task lists (Section 7.2 (2) edgelist reduction).
enum TaskKind : int {
  kTasksDag = 1,    // arcs of the degree-oriented DAG
  kTasksLower = 2,  // (v1, v2) with v2 < v1
  kTasksAll = 3     // every directed CSR entry
};

// Device-side view of a CSR (int64 offsets, uint32 neighbours).
struct DevCsr {
  const int64_t* off = nullptr;
  const uint32_t* nbr = nullptr;
  uint32_t n = 0;
  uint64_t nnz = 0;
};

// A root task list: task t is (src[t], dst[t]).
struct DevTasks {
  const uint32_t* src = nullptr;
  const uint32_t* dst = nullptr;
  uint64_t count = 0;
};

// Per-launch control block in device memory (scratch owned by the plan).
struct Control {
  unsigned long long next;       // dynamic task queue head (relative to task_lo)
  unsigned long long result;     // match count accumulator
  unsigned long long list_head;  // listing cursor (matches reserved so far)
  unsigned long long stats[3];   // algorithmic bytes, set operations, bitmap word-ops
  unsigned long long overflow;   // arcs appended to the plan's overflow list
  unsigned int error;            // nonzero: a device-side check failed
  unsigned int pad;
};

// Kernel launch parameters common to the enumeration kernels.
struct LaunchCfg {
  uint32_t blocks = 0;
  uint32_t warps_per_block = 0;
  uint32_t chunk = 0;
  uint32_t ratio = 0;
  uint32_t smem_cap = 0;     // per-warp, per-level shared-memory buffer (entries)
  uint32_t levels = 0;       // buffered DFS levels X
  uint32_t gstack_cap = 0;   // per-warp, per-level global buffer (entries)
  uint32_t stats = 0;        // accumulate algorithmic bytes / set operations
};

// Error word bits set by kernels.
constexpr unsigned kErrStack = 1u;     // DFS buffer overflow (plan mis-sized)
constexpr unsigned kErrListCap = 2u;   // (not an error) listing truncated

}  // namespace gpm

struct gpm_graph {
  gpm::DevCsr g;
  int64_t* off_d = nullptr;  // owned unless borrowed
  uint32_t* nbr_d = nullptr;
  bool borrowed = false;
  uint32_t max_degree = 0;
  // degree-oriented DAG (lazily built)
  int64_t* doff_d = nullptr;
  uint32_t* dnbr_d = nullptr;
  uint32_t* dsrc_d = nullptr;  // source vertex of each arc (task list)
  uint64_t dag_arcs = 0;
  uint32_t max_out_degree = 0;
  // CSR row index of every entry (ALL task list sources)
  uint32_t* row_d = nullptr;
  // reduced (v1 > v2) task list
  uint32_t* lsrc_d = nullptr;
  uint32_t* ldst_d = nullptr;
  uint64_t lower_count = 0;
  uint32_t* deg32_d = nullptr;  // undirected degree of every vertex (lazily built)
  uint32_t* perm_d = nullptr;   // renamed graphs: the caller's ID of every vertex
  int device = 0;
  int num_sms = 0;
};

struct gpm_plan_s {
  gpm_graph* graph = nullptr;
  int family = 0;
  uint32_t k = 0;
  int induced = 0;
  int mode = 0;
  int count_only = 1;
  gpm::TaskKind task_kind = gpm::kTasksDag;
  gpm::DevTasks tasks;
  gpm::DevCsr csr;  // the CSR the kernel walks (DAG for cliques)
  gpm::LaunchCfg cfg;
  gpm::Control* ctl_d = nullptr;       // device control block
  uint32_t* gstack_d = nullptr;        // per-warp global DFS buffers
  size_t gstack_bytes = 0;
  gpm::Control* host_pinned = nullptr;  // pinned staging for results
  gpm::Control last{};                  // control block of the last launch
  // local graph search (cliques, counting): root vertices by out-degree class
  bool lgs = false;
  // root classes by DAG out-degree: <= 64 (warp), <= 256, <= 512, <= 1024 (CTA)
  uint32_t* lgs_verts[4] = {nullptr, nullptr, nullptr, nullptr};
  uint64_t lgs_count[4] = {0, 0, 0, 0};
  uint64_t* heavy_idx = nullptr;  // arcs of roots with d > 1024 (arc-rooted local graphs)
  uint64_t heavy_count = 0;
  uint64_t* overflow_d = nullptr;  // heavy arcs whose local graph exceeds 1024 members
  // counting-only 4-cycles (full counts): per-CTA dense wedge counters
  bool wedge = false;
  uint32_t* wedge_cnt = nullptr;
  unsigned wedge_blocks = 0;
  unsigned lgs_warp_blocks = 0;
  unsigned lgs_bps[4] = {1, 1, 1, 1};  // resident CTAs per SM of each CTA class
  // generic plans: the search plan (host copy and device copy)
  gpm::GenTable gen{};
  gpm::GenTable* gen_d = nullptr;
  // vertex parallelism: root tasks are vertices (no task list built)
  bool vertex_tasks = false;
};

namespace gpm {

// Thread-local last error message.
void set_error(const std::string& msg);
const std::string& get_error();

// Preprocessing (prep.cu).  All run on `stream`; return a CUDA error code.
// Offsets, ranges, order and self-loops are always checked (they guard the
// kernels' memory accesses); the symmetry check runs only when `full`.
cudaError_t validate_csr(const DevCsr& g, bool full, cudaStream_t stream, unsigned* flags_out,
                         uint32_t* max_degree_out);
cudaError_t build_dag(gpm_graph* G, cudaStream_t stream);
cudaError_t build_rows(gpm_graph* G, cudaStream_t stream);
cudaError_t build_lower(gpm_graph* G, cudaStream_t stream);
// Root vertices of the local graph search by DAG out-degree class c:
// out-degree in (bounds[c-1], bounds[c]] (bounds[-1] = 0) and >= kmin, for
// c < nclass; and the arcs of roots with out-degree > bounds[nclass-1].
cudaError_t build_lgs_classes(gpm_graph* G, uint32_t kmin, const uint32_t* bounds, int nclass,
                              uint32_t** verts, uint64_t* counts, uint64_t** heavy,
                              uint64_t* heavy_count, cudaStream_t stream);

// Enumeration launch (enum.cu).  Runs tasks [lo, hi) of plan p on `stream`.
cudaError_t launch_enum(gpm_plan_t* p, uint64_t lo, uint64_t hi, uint32_t* list_out,
                        uint64_t list_cap, cudaStream_t stream);
// Required dynamic shared memory for a plan's configuration.
size_t enum_smem_bytes(const gpm_plan_t* p);
// Max resident blocks per SM of the plan's kernel at its configuration.
int enum_occupancy(const gpm_plan_t* p, int* regs_per_thread);

// Validation flag bits (prep.cu -> api.cu).
constexpr unsigned kBadUnsorted = 1u, kBadSelfLoop = 2u, kBadDuplicate = 4u,
                   kBadAsymmetric = 8u, kBadRange = 16u, kBadOffsets = 32u;

}  // namespace gpm
