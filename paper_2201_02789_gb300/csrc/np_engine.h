// Host engine shared by the single-solve, batched and serving entry points.
//
// A Workspace is the device state of one running level loop: its LevelState
// (level base, frontier counts, per-level slots, counters, error word), the
// frontier buffers and the aggregation scratch, plus the CUDA graphs captured
// against those pointers. An Engine is what one device needs once: its SM
// count, a capture stream, pinned read-back words, the occupancy cache and the
// execution-time breakdown. The single-solve context owns one Engine and one
// Workspace; a batch owns one Workspace per instance group and a server one
// per pool, all driven by the same functions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <map>
#include <string>

#include "nestpar.h"
#include "np_device.cuh"
#include "np_kernels.h"

namespace nestpar {

np_status from_cuda(cudaError_t e);
np_status status_from_bits(unsigned bits);

#define NP_CK(x)                                              \
  do {                                                        \
    cudaError_t e_ = (x);                                     \
    if (e_ != cudaSuccess) return ::nestpar::from_cuda(e_);   \
  } while (0)

#define NP_TRY(x)                          \
  do {                                     \
    np_status s_ = (x);                    \
    if (s_ != NP_OK) return s_;            \
  } while (0)

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

enum Mode : int { M_NODP = 0, M_GRID_HOST = 1, M_DEVICE_LAUNCH = 2 };

struct Plan {
  const void* parent = nullptr;
  const void* child = nullptr;  // persistent child grid (grid-host form)
  const void* loop = nullptr;   // persistent level loop (NODP and grid-host forms)
  const void* small = nullptr;  // one-CTA small-level loop before the while loop and at each body's end (grid-host)
  const void* sweep = nullptr;  // swept frontier: the kernel that rebuilds the next frontier after each level
  // grid-host form that can give its child grid no work (threshold INT32_MAX,
  // serialised children in the parent kernel): no child grid is launched (a
  // fixed pass, or each level of a level loop)
  bool child_idle = false;
  int mode = M_NODP;
  int gran = G_NODP;
};

struct Layout {
  size_t off_fr0, off_fr1, off_stamp, off_rec, off_boff, off_lb_flag, off_lb_agg, off_lb_incl, off_ob_flag,
      off_ob_agg, off_ob_incl, off_grp_ctr, off_grp_acc, off_grp_total, off_prec, off_pfirst, total;
  int64_t P2, T;
};

// Frontier buffers, stamps, records and block offsets for up to `parents`
// entries; look-back tile states for ceil(parents / 32) tiles.
Layout layout_for(int64_t parents);

struct Grids {
  int pgrid, pblock, cgrid, cblock, cthreads;
};

struct Engine {
  int device = 0;
  int sms = 0;
  cudaStream_t cap_stream = nullptr;
  int* pin = nullptr;                 // pinned read-back of the level header
  LevelState* pin_state = nullptr;    // pinned read-back of the whole state
  std::map<std::pair<const void*, int>, int> occ;
  // execution-time breakdown (np_profile_*)
  bool profile = false;
  np_profile prof{};
  int prof_next_parents = 0;          // frontier size of the level about to be profiled
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
};

struct Workspace {
  LevelState* st = nullptr;
  unsigned char* ws = nullptr;
  Layout lay{};
  int64_t cap_parents = 0;
  std::map<std::string, GraphEntry> graphs;
};

np_status engine_init(Engine& e, int device);
void engine_release(Engine& e);

np_status ws_init(Workspace& w);
void ws_release(Workspace& w);
void ws_drop_graphs(Workspace& w);
// Grows the buffers to hold `parents` (at least 4096); drops cached graphs when it does.
np_status ws_ensure(Workspace& w, int64_t parents);
template <class T>
T* wsp(const Workspace& w, size_t off) {
  return reinterpret_cast<T*>(w.ws + off);
}

int occupancy(Engine& e, const void* fn, int block);
np_status check_config(const np_config* cfg);
// Where the children below the threshold run under cfg (NP_SERIAL_*): the
// configured place for grid-host aggregation (PACKED needs threshold <= 1024,
// else BLOCK), SPREAD-or-serial-in-thread (the warp-tiled kernels) otherwise.
int serial_form(const np_config& cfg);
// The CTA-tiled forms count a tile's or a level's items in 32 bits: a level
// loop over `copies` traversals of a graph with m edges at once, which could
// meet 2^31 items or more, takes the warp-tiled parent (SPREAD) instead.
np_config serial_for(const np_config& cfg, int64_t copies, int64_t m);
// The swept frontier under cfg: requested, grid-host aggregation with the
// warp-tiled parent, not the persistent loop (np_bfs / np_sssp only; other
// entry points run the appended frontier).
bool sweeps(const np_config& cfg);
Plan make_plan(const BodyKernels& K, const np_config& cfg);
// Args of one level loop / pass over workspace `w` (vmask all ones).
void base_args(const Workspace& w, const np_config& cfg, Args& a);
Grids grids_for(Engine& e, const Plan& p, const np_config& cfg, int64_t max_parents);
// AUTO resolved: chunks for the device-launch forms, a conditional while loop otherwise.
int resolve_driver(const Plan& p, const np_config& cfg);

np_status enqueue_pass(const Plan& p, Args a, const Grids& g, bool level_mode, int k, cudaStream_t s);
np_status enqueue_advance(LevelState* st, int K, cudaStream_t s, bool after_launch_free = false);
np_status profiled_pass(Engine& e, const Workspace& w, const Plan& p, Args a, const Grids& g, bool level_mode,
                        cudaStream_t s);

// K levels plus the base advance, captured into a plain graph (cached in w).
np_status chunk_graph(Engine& e, Workspace& w, const Plan& p, const Args& a, const Grids& g, int K,
                      cudaGraphExec_t* out);
// Adds `while (frontier not empty) { K levels; set condition }` to `graph` after `deps`.
np_status add_while_node(Engine& e, LevelState* st, cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                         const Plan& p, const Args& a, const Grids& g, int K, cudaGraphNode_t* node);
// The while loop alone as a cached executable graph.
np_status while_graph(Engine& e, Workspace& w, const Plan& p, const Args& a, const Grids& g, int K,
                      cudaGraphExec_t* out);
np_status instantiate(cudaGraph_t graph, cudaGraphExec_t* exec);
std::string graph_key(const char* tag, const Plan& p, const Args& a, const Grids& g, int unroll);
// Instantiates `graph` and keeps it in w's cache under `key` (w owns both afterwards).
np_status cache_graph(Workspace& w, const std::string& key, cudaGraph_t graph, cudaGraphExec_t* out);

np_status read_header(Engine& e, const Workspace& w, cudaStream_t s, int* level, int* count);
// Synchronises `s`, fills `stats` from the workspace counters, clears the error word.
np_status finish(Engine& e, const Workspace& w, cudaStream_t s, np_stats* stats);
// The level loop from the current base until the frontier is empty (or max_levels).
np_status run_levels(Engine& e, Workspace& w, const Plan& p, const Args& a, const np_config& cfg, int64_t parents,
                     int max_levels, cudaStream_t s);
np_status check_csr(const np_csr* g, bool need_w);
// The persistent level loop (NP_DRIVER_PERSISTENT) as one cooperative launch on s.
np_status launch_level_loop(Engine& e, const Plan& p, const Args& a, const np_config& cfg, int max_levels,
                            cudaStream_t s);

// ---- device-side initialisation kernels (np_engine.cu)
__global__ void init_solve_kernel(LevelState* st, int kind, int n, int src, int* level, unsigned* dist, int* stamp,
                                  int* fr0, int max_levels);
__global__ void init_fixed_kernel(LevelState* st);
// Multi-source start: every element of level/dist/stamp[0, total) to its unreached value.
__global__ void fill_unreached_kernel(int kind, long long total, int* level, unsigned* dist, int* stamp);
// Then the sources (ids into those arrays) become level 0 / distance 0 and the first frontier.
__global__ void seed_sources_kernel(LevelState* st, int kind, const int* ids, int nsrc, int* level, unsigned* dist,
                                    int* fr0, int max_levels);
__global__ void advance_base_kernel(LevelState* st, int K);
// Bounded-wait checks of np_selftest_wait (each waits on a flag nothing sets).
__global__ void selftest_lookback_kernel(Args a);
__global__ void selftest_barrier_kernel(LevelState* st, unsigned long long limit_ns);
// Packed SSSP state: dtag[0, total) = unreached (all ones << 32), then the
// sources (ids) at distance 0 become the first frontier; finally dist = dtag >> 32.
__global__ void init_dtag_kernel(long long total, unsigned long long* dtag);
__global__ void seed_dtag_kernel(LevelState* st, const int* ids, int nsrc, unsigned long long* dtag, int* fr0,
                                 int max_levels);
__global__ void dtag_to_dist_kernel(long long total, const unsigned long long* dtag, unsigned* dist);
// Single-source start of the packed form in one kernel (as init_solve_kernel).
__global__ void init_dtag_solve_kernel(LevelState* st, int n, int src, unsigned long long* dtag, int* fr0,
                                       int max_levels);
// *out (+)= the sum of part[0, n) (one block)
__global__ void sum_u64_kernel(const unsigned long long* part, int n, unsigned long long* out, int accumulate);
// Sets *bad when a CSR breaks its contract: row_ptr[0] != 0, row_ptr[n] != m,
// a decreasing row_ptr, or a column index outside [0, n).
__global__ void csr_check_kernel(const int* row_ptr, const int* col, int n, long long m, int* bad);
// Runs csr_check_kernel over each graph on stream s and waits: NP_ERR_INVALID
// if any breaks the contract. `scratch` is one device int.
np_status check_csr_device(const np_csr* graphs, int count, int* scratch, cudaStream_t s);

inline int blocks_for(long long n, int per = 256, int cap = 4096) {
  long long b = (n + per - 1) / per;
  if (b < 1) b = 1;
  return (int)(b < cap ? b : cap);
}

}  // namespace nestpar
