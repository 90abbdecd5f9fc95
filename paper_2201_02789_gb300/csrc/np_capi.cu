// Host engine and C ABI (include/nestpar.h).
//
// Level loop. A level is one parent grid (persistent CTAs over the frontier,
// which lives in device memory) plus, for grid-host aggregation, one
// stream-ordered persistent child grid whose size is read from device memory.
// Forms without a device launch site (NODP, grid-host aggregation) run the
// whole loop inside a conditional-while CUDA graph: `unroll` levels per body
// iteration, a one-thread kernel setting the condition, no host round trip.
// Kernels containing device launches cannot sit in a conditional body, so the
// device-launch forms replay a graph of `unroll` levels from the host and read
// the frontier size back after each replay. NP_DRIVER_HOST is the paper's own
// form: one host launch per level and a read-back after each.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "nestpar.h"
#include "np_device.cuh"
#include "np_kernels.h"

using namespace nestpar;

namespace {

constexpr int kVersion = 10000;  // 1.0.0
constexpr size_t kAlign = 256;


__device__ __forceinline__ void reset_slots(LevelState* st) {
  for (int k = 0; k < 4; k++) {
    st->ticket[k] = 0;
    st->agg_records[k] = 0;
    st->agg_blocks[k] = 0;
    st->agg_acc[k] = 0ull;
  }
  for (int k = 0; k < S_N; k++) st->s[k] = 0ull;
  st->body_iters = 0;
  st->solve_id += 1;
}

__global__ void init_solve_kernel(LevelState* st, int kind, int n, int src, int* level, unsigned* dist,
                                  int* stamp, int* fr0, int max_levels) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (kind == 0) {
      level[v] = v == src ? 0 : -1;
    } else {
      dist[v] = v == src ? 0u : 0xffffffffu;
      stamp[v] = -1;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    fr0[0] = src;
    st->base = 0;
    st->count[0] = 1;
    st->count[1] = 0;
    st->count[2] = 0;
    st->max_levels = max_levels;
    reset_slots(st);
  }
}

__global__ void init_fixed_kernel(LevelState* st) { reset_slots(st); }

// Between graph bodies or chunks: the next body position 0 is level base + K.
__global__ void advance_base_kernel(LevelState* st, int K) { st->base += K; }

// End of a conditional-while body of K levels: move base on and continue while
// the next level has parents. The iteration cap turns a level loop that failed
// to terminate into an error instead of an endless loop.
__global__ void set_cond_kernel(LevelState* st, cudaGraphConditionalHandle h, int K) {
  const int L = st->base + K;
  st->base = L;
  const int c = st->count[L % 3];
  const int it = ++st->body_iters;
  bool more = c > 0 && L < st->max_levels;
  if (more && it > st->max_levels + 16) {
    st->error |= kErrTimeout;
    more = false;
  }
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

enum Mode : int { M_NODP = 0, M_GRID_HOST = 1, M_DEVICE_LAUNCH = 2 };

struct Plan {
  const void* parent = nullptr;
  const void* child = nullptr;  // persistent child grid (grid-host form)
  int mode = M_NODP;
  int gran = G_NODP;
};

struct Layout {
  size_t off_fr0, off_fr1, off_stamp, off_rec, off_boff, off_lb_flag, off_lb_agg, off_lb_incl, off_ob_flag,
      off_ob_agg, off_ob_incl, off_grp_ctr, off_grp_acc, off_grp_total, total;
  int64_t P2, T;
};

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Frontier buffers hold up to `parents` appends (exact appends: no padding).
Layout layout_for(int64_t parents, int sms) {
  (void)sms;
  Layout L{};
  L.P2 = ((parents + 1023) / 1024) * 1024 + 1024;
  L.T = L.P2 / 32 + 64;
  const int64_t fr = L.P2;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = align_up(o + bytes);
    return r;
  };
  L.off_fr0 = take(sizeof(int) * fr);
  L.off_fr1 = take(sizeof(int) * fr);
  L.off_stamp = take(sizeof(int) * L.P2);
  L.off_rec = take(sizeof(int4) * L.P2);
  L.off_boff = take(sizeof(int) * L.P2);
  L.off_lb_flag = take(sizeof(unsigned long long) * L.T);
  L.off_lb_agg = take(sizeof(uint4) * L.T);
  L.off_lb_incl = take(sizeof(uint4) * L.T);
  L.off_ob_flag = take(sizeof(unsigned long long) * L.T);
  L.off_ob_agg = take(sizeof(uint4) * L.T);
  L.off_ob_incl = take(sizeof(uint4) * L.T);
  L.off_grp_ctr = take(sizeof(int) * L.T);
  L.off_grp_acc = take(sizeof(unsigned long long) * L.T);
  L.off_grp_total = take(sizeof(uint2) * L.T);
  L.total = o;
  return L;
}

np_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return NP_OK;
  if (e == cudaErrorMemoryAllocation) return NP_ERR_NOMEM;
  return NP_ERR_CUDA;
}

#define NP_CK(x)                                   \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return from_cuda(e_);   \
  } while (0)

np_status status_from_bits(unsigned bits) {
  if (bits & kErrTimeout) return NP_ERR_TIMEOUT;
  if (bits & kErrCapacity) return NP_ERR_CAPACITY;
  if (bits & kErrLaunch) return NP_ERR_LAUNCH;
  return NP_OK;
}

}  // namespace

struct np_ctx {
  int device = 0;
  int sms = 0;
  LevelState* st = nullptr;
  unsigned char* ws = nullptr;
  Layout lay{};
  int64_t cap_parents = 0;
  int* pin = nullptr;                 // pinned read-back of the level header
  LevelState* pin_state = nullptr;    // pinned read-back of the whole state
  cudaStream_t cap_stream = nullptr;
  std::map<std::string, GraphEntry> graphs;
  std::map<std::pair<const void*, int>, int> occ;
  // device staging for the *_host entry points
  unsigned char* stage = nullptr;
  size_t stage_bytes = 0;
  // execution-time breakdown (np_profile_*)
  bool profile = false;
  np_profile prof{};
  int prof_next_parents = 0;   // frontier size of the level about to be profiled
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  std::mutex mu;
};

namespace {

void drop_graphs(np_ctx* c) {
  for (auto& kv : c->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  c->graphs.clear();
}

np_status ensure_workspace(np_ctx* c, int64_t parents) {
  if (parents <= c->cap_parents && c->ws) return NP_OK;
  int64_t want = parents < 4096 ? 4096 : parents;
  Layout L = layout_for(want, c->sms);
  drop_graphs(c);
  if (c->ws) {
    NP_CK(cudaDeviceSynchronize());
    cudaFree(c->ws);
    c->ws = nullptr;
    c->cap_parents = 0;
  }
  unsigned char* p = nullptr;
  NP_CK(cudaMalloc(&p, L.total));
  NP_CK(cudaMemset(p, 0, L.total));
  c->ws = p;
  c->lay = L;
  c->cap_parents = want;
  return NP_OK;
}

template <class T>
T* wsp(np_ctx* c, size_t off) {
  return reinterpret_cast<T*>(c->ws + off);
}

int occupancy(np_ctx* c, const void* fn, int block) {
  auto key = std::make_pair(fn, block);
  auto it = c->occ.find(key);
  if (it != c->occ.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0) != cudaSuccess || n < 1) n = 1;
  c->occ[key] = n;
  return n;
}

np_status check_config(const np_config* cfg) {
  if (!cfg) return NP_ERR_INVALID;
  if (cfg->variant != NP_VARIANT_NODP && cfg->variant != NP_VARIANT_CDP) return NP_ERR_INVALID;
  if (cf_index(cfg->cfactor) < 0) return NP_ERR_INVALID;
  if (cfg->granularity < NP_GRAN_NONE || cfg->granularity > NP_GRAN_GRID_HOST) return NP_ERR_INVALID;
  if (cfg->granularity == NP_GRAN_MULTIBLOCK && cfg->group_blocks < 1) return NP_ERR_INVALID;
  if (cfg->agg_threshold < 0) return NP_ERR_INVALID;
  if (cfg->child_block < 32 || cfg->child_block > 1024 || cfg->child_block % 32) return NP_ERR_INVALID;
  if (cfg->parent_block < 64 || cfg->parent_block > kMaxParentBlock || cfg->parent_block % 32) return NP_ERR_INVALID;
  if (cfg->scan != NP_SCAN_LOOKBACK && cfg->scan != NP_SCAN_ATOMIC) return NP_ERR_INVALID;
  if (cfg->driver < NP_DRIVER_AUTO || cfg->driver > NP_DRIVER_WHILE) return NP_ERR_INVALID;
  if (cfg->unroll < 1 || cfg->unroll > 16) return NP_ERR_INVALID;
  if (cfg->parent_grid < 0) return NP_ERR_INVALID;
  for (int k = 0; k < 4; k++)
    if (cfg->reserved[k] != 0) return NP_ERR_INVALID;
  return NP_OK;
}

Plan make_plan(const BodyKernels& K, const np_config& cfg) {
  Plan p;
  const int cfi = cf_index(cfg.cfactor);
  if (cfg.variant == NP_VARIANT_NODP) {
    // warp tiles; with granularity NONE the CTA-tiled kernel of the
    // device-launch forms without its launch code (dead-launch-code baseline)
    p.parent = cfg.granularity == NP_GRAN_NONE ? K.parent_nodp_cta : K.parent_nodp;
    p.mode = M_NODP;
    p.gran = G_NODP;
  } else if (cfg.granularity == NP_GRAN_GRID_HOST) {
    p.parent = K.parent_grid_host;
    p.child = K.child_agg[cfi];
    p.mode = M_GRID_HOST;
    p.gran = G_GRID_HOST;
  } else {
    int row = 0;
    switch (cfg.granularity) {
      case NP_GRAN_NONE: row = 0; break;
      case NP_GRAN_WARP: row = 1; break;
      case NP_GRAN_BLOCK: row = 2; break;
      default: row = 3; break;  // multi-block and grid-device share one kernel
    }
    p.parent = K.parent[row][cfi];
    p.mode = M_DEVICE_LAUNCH;
    p.gran = cfg.granularity;
  }
  return p;
}

void base_args(np_ctx* c, const np_config& cfg, Args& a) {
  std::memset(&a, 0, sizeof(a));
  a.st = c->st;
  a.fr0 = wsp<int>(c, c->lay.off_fr0);
  a.fr1 = wsp<int>(c, c->lay.off_fr1);
  a.rec = wsp<int4>(c, c->lay.off_rec);
  a.boff = wsp<int>(c, c->lay.off_boff);
  a.lb_flag = wsp<unsigned long long>(c, c->lay.off_lb_flag);
  a.lb_agg = wsp<uint4>(c, c->lay.off_lb_agg);
  a.lb_incl = wsp<uint4>(c, c->lay.off_lb_incl);
  a.ob_flag = wsp<unsigned long long>(c, c->lay.off_ob_flag);
  a.ob_agg = wsp<uint4>(c, c->lay.off_ob_agg);
  a.ob_incl = wsp<uint4>(c, c->lay.off_ob_incl);
  a.grp_ctr = wsp<int>(c, c->lay.off_grp_ctr);
  a.grp_acc = wsp<unsigned long long>(c, c->lay.off_grp_acc);
  a.grp_total = wsp<uint2>(c, c->lay.off_grp_total);
  a.threshold = cfg.threshold;
  a.cfactor = cfg.cfactor;
  a.child_block = cfg.child_block;
  a.group_blocks = cfg.granularity == NP_GRAN_MULTIBLOCK ? cfg.group_blocks : 0;
  a.agg_threshold = (cfg.granularity == NP_GRAN_WARP || cfg.granularity == NP_GRAN_BLOCK) ? cfg.agg_threshold : 0;
  a.scan = cfg.scan;
  a.b.st = c->st;
  a.count_fixed = -1;
}

struct Grids {
  int pgrid, pblock, cgrid, cblock, cthreads;
};

Grids grids_for(np_ctx* c, const Plan& p, const np_config& cfg, int64_t max_parents) {
  Grids g{};
  g.pblock = cfg.parent_block;
  g.cblock = cfg.child_block;
  int64_t tiles = (max_parents + g.pblock - 1) / g.pblock;
  if (tiles < 1) tiles = 1;
  int64_t pg = cfg.parent_grid > 0 ? cfg.parent_grid : (int64_t)occupancy(c, p.parent, g.pblock) * c->sms;
  if (pg > tiles) pg = tiles;
  g.pgrid = (int)pg;
  // the persistent child grid hosts cb-thread child blocks in CTAs of at least 256 threads
  g.cthreads = g.cblock < 256 ? 256 : g.cblock;
  g.cgrid = p.child ? occupancy(c, p.child, g.cthreads) * c->sms : 0;
  return g;
}

// Enqueues the grids of one level (level mode, at body position k) or of one
// fixed pass.
np_status enqueue_pass(np_ctx* c, const Plan& p, Args a, const Grids& g, bool level_mode, int k, cudaStream_t s) {
  a.k = level_mode ? k : 0;
  void* pargs[] = {&a};
  NP_CK(cudaLaunchKernel(p.parent, dim3(g.pgrid), dim3(g.pblock), pargs, 0, s));
  if (p.mode == M_GRID_HOST) {
    AggSeg seg{};
    seg.rec = a.rec;
    seg.boff = a.boff;
    seg.mode = a.scan == 0 ? 1 : 2;
    seg.k = a.k;
    seg.level_mode = level_mode ? 1 : 0;
    seg.fr0 = a.fr0;
    seg.fr1 = a.fr1;
    seg.cb = g.cblock;
    BodyArgs b = a.b;
    if (!level_mode) {
      b.L = a.L_fixed;
      b.next = a.next_ovr;
      b.next_count = a.next_count_ovr;
    }
    void* cargs[] = {&b, &seg};
    NP_CK(cudaLaunchKernel(p.child, dim3(g.cgrid), dim3(g.cthreads), cargs, 0, s));
  }
  return NP_OK;
}

np_status enqueue_advance(np_ctx* c, int K, cudaStream_t s) {
  advance_base_kernel<<<1, 1, 0, s>>>(c->st, K);
  NP_CK(cudaGetLastError());
  return NP_OK;
}

// Profile mode: the grids of one level (or pass) launched one by one between
// CUDA events, then waited for; times go to the context's breakdown.
np_status profiled_pass(np_ctx* c, const Plan& p, Args a, const Grids& g, bool level_mode, cudaStream_t s) {
  a.k = 0;
  void* pargs[] = {&a};
  NP_CK(cudaEventRecord(c->ev[0], s));
  NP_CK(cudaLaunchKernel(p.parent, dim3(g.pgrid), dim3(g.pblock), pargs, 0, s));
  NP_CK(cudaEventRecord(c->ev[1], s));
  bool child = false, other = false;
  cudaEvent_t child_end = c->ev[2];
  if (p.mode == M_GRID_HOST) {
    AggSeg seg{};
    seg.rec = a.rec;
    seg.boff = a.boff;
    seg.mode = a.scan == 0 ? 1 : 2;
    seg.k = 0;
    seg.level_mode = level_mode ? 1 : 0;
    seg.fr0 = a.fr0;
    seg.fr1 = a.fr1;
    seg.cb = g.cblock;
    BodyArgs b = a.b;
    if (!level_mode) {
      b.L = a.L_fixed;
      b.next = a.next_ovr;
      b.next_count = a.next_count_ovr;
    }
    void* cargs[] = {&b, &seg};
    NP_CK(cudaLaunchKernel(p.child, dim3(g.cgrid), dim3(g.cthreads), cargs, 0, s));
    child = true;
  }
  NP_CK(cudaEventRecord(child_end, s));
  if (level_mode) {
    advance_base_kernel<<<1, 1, 0, s>>>(c->st, 1);
    NP_CK(cudaGetLastError());
    other = true;
  }
  NP_CK(cudaEventRecord(c->ev[3], s));
  NP_CK(cudaEventSynchronize(c->ev[3]));
  float t01 = 0.f, t12 = 0.f, t23 = 0.f;
  NP_CK(cudaEventElapsedTime(&t01, c->ev[0], c->ev[1]));
  NP_CK(cudaEventElapsedTime(&t12, c->ev[1], c->ev[2]));
  NP_CK(cudaEventElapsedTime(&t23, c->ev[2], c->ev[3]));
  c->prof.parent_ms += t01;
  c->prof.parent_launches += 1;
  if (child) {
    c->prof.child_ms += t12;
    c->prof.child_launches += 1;
  }
  if (other) {
    c->prof.other_ms += t23;
    c->prof.other_launches += 1;
  }
  if (level_mode) {
    const int k = c->prof.levels;
    const double lvl = (double)t01 + (child ? (double)t12 : 0.0);
    if (lvl > c->prof.longest_level_ms) c->prof.longest_level_ms = lvl;
    if (k < NP_PROFILE_LEVELS) {
      c->prof.level_parents[k] = c->prof_next_parents;
      c->prof.level_parent_ms[k] = t01;
      c->prof.level_child_ms[k] = child ? t12 : 0.0;
      c->prof.levels = k + 1;
    }
  }
  return NP_OK;
}

std::string graph_key(const char* tag, const Plan& p, const Args& a, const Grids& g, int unroll) {
  std::string k(tag);
  k.append(reinterpret_cast<const char*>(&p), sizeof(p));
  k.append(reinterpret_cast<const char*>(&a), sizeof(a));
  k.append(reinterpret_cast<const char*>(&g), sizeof(g));
  k.append(reinterpret_cast<const char*>(&unroll), sizeof(unroll));
  return k;
}

np_status cache_graph(np_ctx* c, const std::string& key, cudaGraph_t graph, cudaGraphExec_t* out) {
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    cudaGetLastError();
    return e == cudaErrorInvalidValue ? NP_ERR_UNSUPPORTED : from_cuda(e);
  }
  if (c->graphs.size() >= 64) drop_graphs(c);
  c->graphs[key] = GraphEntry{graph, exec};
  *out = exec;
  return NP_OK;
}

// K levels captured on the context's capture stream into a plain graph.
np_status chunk_graph(np_ctx* c, const Plan& p, const Args& a, const Grids& g, int K, cudaGraphExec_t* out) {
  std::string key = graph_key("chunk", p, a, g, K);
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    *out = it->second.exec;
    return NP_OK;
  }
  NP_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  np_status st = NP_OK;
  for (int k = 0; k < K && st == NP_OK; k++) st = enqueue_pass(c, p, a, g, true, k, c->cap_stream);
  if (st == NP_OK) st = enqueue_advance(c, K, c->cap_stream);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (st != NP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  NP_CK(e);
  return cache_graph(c, key, graph, out);
}

// while (frontier not empty) { K levels; set condition } as a conditional graph.
np_status while_graph(np_ctx* c, const Plan& p, const Args& a, const Grids& g, int K, cudaGraphExec_t* out) {
  std::string key = graph_key("while", p, a, g, K);
  auto it = c->graphs.find(key);
  if (it != c->graphs.end()) {
    *out = it->second.exec;
    return NP_OK;
  }
  cudaGraph_t graph = nullptr;
  NP_CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return from_cuda(e);
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return from_cuda(e);
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return from_cuda(e);
  }
  np_status st = NP_OK;
  for (int k = 0; k < K && st == NP_OK; k++) st = enqueue_pass(c, p, a, g, true, k, c->cap_stream);
  set_cond_kernel<<<1, 1, 0, c->cap_stream>>>(c->st, h, K);
  cudaError_t le = cudaGetLastError();
  e = cudaStreamEndCapture(c->cap_stream, &body);
  if (st != NP_OK || le != cudaSuccess || e != cudaSuccess) {
    cudaGraphDestroy(graph);
    if (st != NP_OK) return st;
    return from_cuda(le != cudaSuccess ? le : e);
  }
  return cache_graph(c, key, graph, out);
}

np_status read_header(np_ctx* c, cudaStream_t s, int* level, int* count) {
  NP_CK(cudaMemcpyAsync(c->pin, c->st, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));   // base, count[3]
  NP_CK(cudaStreamSynchronize(s));
  *level = c->pin[0];
  *count = c->pin[1 + c->pin[0] % 3];
  return NP_OK;
}

np_status finish(np_ctx* c, cudaStream_t s, np_stats* stats) {
  if (!stats) return NP_OK;
  NP_CK(cudaMemcpyAsync(c->pin_state, c->st, sizeof(LevelState), cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  const LevelState& h = *c->pin_state;
  std::memset(stats, 0, sizeof(*stats));
  stats->levels = h.s[S_LEVELS];
  stats->parents = h.s[S_PARENTS];
  stats->serial_parents = h.s[S_SERIAL];
  stats->launch_parents = h.s[S_LAUNCHP];
  stats->device_launches = h.s[S_DEVLAUNCH];
  stats->aggregated_grids = h.s[S_AGGGRID];
  stats->child_blocks = h.s[S_CBLOCKS];
  stats->items = h.s[S_ITEMS];
  stats->pushes = h.s[S_PUSHES];
  stats->launch_failures = h.s[S_LFAIL];
  stats->timeouts = h.s[S_TIMEOUT];
  stats->child_items = h.s[S_CITEMS];
  stats->graph_iterations = (uint64_t)h.body_iters;
  stats->error = h.error;
  if (h.error) {
    NP_CK(cudaMemsetAsync(&c->st->error, 0, sizeof(unsigned), s));
    NP_CK(cudaStreamSynchronize(s));
  }
  return status_from_bits(h.error);
}

// The level loop of np_bfs / np_sssp.
np_status run_levels(np_ctx* c, const Plan& p, const Args& a, const np_config& cfg, int n, cudaStream_t s) {
  Grids g = grids_for(c, p, cfg, n);
  int driver = cfg.driver;
  if (driver == NP_DRIVER_AUTO) driver = p.mode == M_DEVICE_LAUNCH ? NP_DRIVER_CHUNK : NP_DRIVER_WHILE;
  if (driver == NP_DRIVER_WHILE && p.mode == M_DEVICE_LAUNCH) return NP_ERR_UNSUPPORTED;
  const int max_levels = n + 2;
  if (c->profile) {
    // per-level records describe this call only
    c->prof.levels = 0;
    c->prof.longest_level_ms = 0.0;
    c->prof_next_parents = 1;
    for (int iter = 0;; iter++) {
      if (iter > max_levels + 16) return NP_ERR_TIMEOUT;
      np_status st = profiled_pass(c, p, a, g, true, s);
      if (st != NP_OK) return st;
      int level = 0, count = 0;
      st = read_header(c, s, &level, &count);
      if (st != NP_OK) return st;
      c->prof_next_parents = count;
      if (count <= 0 || level >= max_levels) break;
    }
    return NP_OK;
  }
  if (driver == NP_DRIVER_WHILE) {
    cudaGraphExec_t exec;
    np_status st = while_graph(c, p, a, g, cfg.unroll, &exec);
    if (st != NP_OK) return st;
    NP_CK(cudaGraphLaunch(exec, s));
    return NP_OK;
  }
  cudaGraphExec_t exec = nullptr;
  if (driver == NP_DRIVER_CHUNK) {
    np_status st = chunk_graph(c, p, a, g, cfg.unroll, &exec);
    if (st != NP_OK) return st;
  }
  for (int iter = 0;; iter++) {
    if (iter > max_levels + 16) return NP_ERR_TIMEOUT;   // a level failed to advance
    if (exec) {
      NP_CK(cudaGraphLaunch(exec, s));
    } else {
      np_status st = enqueue_pass(c, p, a, g, true, 0, s);
      if (st == NP_OK) st = enqueue_advance(c, 1, s);
      if (st != NP_OK) return st;
    }
    int level = 0, count = 0;
    np_status st = read_header(c, s, &level, &count);
    if (st != NP_OK) return st;
    if (count <= 0 || level >= max_levels) break;
  }
  return NP_OK;
}

np_status check_csr(const np_csr* g, bool need_w) {
  if (!g || !g->row_ptr || (!g->col_idx && g->m > 0) || g->n < 1 || g->m < 0 || g->m >= INT_MAX) return NP_ERR_INVALID;
  if (need_w && !g->weights && g->m > 0) return NP_ERR_INVALID;
  return NP_OK;
}

// One graph solve (kind 0 BFS, 1 SSSP) on device arrays.
np_status solve(np_ctx* c, int kind, const np_csr* g, int src, int* level, unsigned* dist,
                const np_config* cfg, cudaStream_t s, np_stats* stats) {
  if (!c) return NP_ERR_INVALID;
  np_status st = check_config(cfg);
  if (st != NP_OK) return st;
  st = check_csr(g, kind == 1);
  if (st != NP_OK) return st;
  if (src < 0 || src >= g->n) return NP_ERR_INVALID;
  if ((kind == 0 && !level) || (kind == 1 && !dist)) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->device));
  st = ensure_workspace(c, g->n);
  if (st != NP_OK) return st;
  const BodyKernels& K = kind == 0 ? bfs_kernels() : sssp_kernels();
  Plan p = make_plan(K, *cfg);
  Args a;
  base_args(c, *cfg, a);
  a.row_ptr = g->row_ptr;
  a.b.col = g->col_idx;
  a.b.w = g->weights;
  a.b.level = level;
  a.b.dist = dist;
  a.b.stamp = wsp<int>(c, c->lay.off_stamp);
  const int blocks = (int)((g->n + 255) / 256 < 4096 ? (g->n + 255) / 256 : 4096);
  if (c->profile) NP_CK(cudaEventRecord(c->ev[0], s));
  init_solve_kernel<<<blocks, 256, 0, s>>>(c->st, kind, g->n, src, level, dist, a.b.stamp, a.fr0, g->n + 2);
  NP_CK(cudaGetLastError());
  if (c->profile) {
    NP_CK(cudaEventRecord(c->ev[3], s));
    NP_CK(cudaEventSynchronize(c->ev[3]));
    float t = 0.f;
    NP_CK(cudaEventElapsedTime(&t, c->ev[0], c->ev[3]));
    c->prof.other_ms += t;
    c->prof.other_launches += 1;
  }
  st = run_levels(c, p, a, *cfg, g->n, s);
  if (st != NP_OK) return st;
  return finish(c, s, stats);
}

// One fixed pass over an explicit parent set.
np_status fixed_pass(np_ctx* c, const Args& a0, const np_config& cfg, const BodyKernels& K, int count,
                     cudaStream_t s) {
  Plan p = make_plan(K, cfg);
  Args a = a0;
  Grids g = grids_for(c, p, cfg, count);
  if (c->profile) {
    NP_CK(cudaEventRecord(c->ev[0], s));
    init_fixed_kernel<<<1, 1, 0, s>>>(c->st);
    NP_CK(cudaGetLastError());
    NP_CK(cudaEventRecord(c->ev[3], s));
    NP_CK(cudaEventSynchronize(c->ev[3]));
    float t = 0.f;
    NP_CK(cudaEventElapsedTime(&t, c->ev[0], c->ev[3]));
    c->prof.other_ms += t;
    c->prof.other_launches += 1;
    return profiled_pass(c, p, a, g, false, s);
  }
  std::string key = graph_key("fixed", p, a, g, 1);
  auto it = c->graphs.find(key);
  cudaGraphExec_t exec = nullptr;
  if (it != c->graphs.end()) {
    exec = it->second.exec;
  } else {
    NP_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    init_fixed_kernel<<<1, 1, 0, c->cap_stream>>>(c->st);
    cudaError_t le = cudaGetLastError();
    np_status st = le == cudaSuccess ? enqueue_pass(c, p, a, g, false, 0, c->cap_stream) : from_cuda(le);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (st != NP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    NP_CK(e);
    st = cache_graph(c, key, graph, &exec);
    if (st != NP_OK) return st;
  }
  NP_CK(cudaGraphLaunch(exec, s));
  return NP_OK;
}

np_status stage_bytes(np_ctx* c, size_t bytes) {
  if (bytes <= c->stage_bytes) return NP_OK;
  if (c->stage) {
    NP_CK(cudaDeviceSynchronize());
    cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_bytes = 0;
  }
  NP_CK(cudaMalloc(&c->stage, bytes));
  c->stage_bytes = bytes;
  return NP_OK;
}

}  // namespace

// ======================================================================= C ABI

extern "C" {

np_status np_config_default(np_config* cfg) {
  if (!cfg) return NP_ERR_INVALID;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->variant = NP_VARIANT_CDP;
  cfg->threshold = 32;
  cfg->cfactor = 8;
  cfg->granularity = NP_GRAN_GRID_HOST;
  cfg->group_blocks = 8;
  cfg->agg_threshold = 0;
  cfg->child_block = 32;
  cfg->parent_block = 256;
  cfg->scan = NP_SCAN_ATOMIC;
  cfg->driver = NP_DRIVER_AUTO;
  cfg->unroll = 4;
  cfg->parent_grid = 0;
  return NP_OK;
}

np_status np_create(np_ctx** out, int32_t device) {
  if (!out) return NP_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  NP_CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return NP_ERR_INVALID;
  NP_CK(cudaSetDevice(device));
  cudaDeviceProp prop;
  NP_CK(cudaGetDeviceProperties(&prop, device));
  // plain CDP issues one device launch per parent: raise the pending-launch pool
  // (the driver caps the request; refused launches fall back to serial work)
  size_t cur = 0;
  if (cudaDeviceGetLimit(&cur, cudaLimitDevRuntimePendingLaunchCount) == cudaSuccess && cur < (1u << 20))
    cudaDeviceSetLimit(cudaLimitDevRuntimePendingLaunchCount, 1u << 20);
  cudaGetLastError();
  np_ctx* c = new np_ctx();
  c->device = device;
  c->sms = prop.multiProcessorCount;
  cudaError_t e = cudaMalloc(&c->st, sizeof(LevelState));
  if (e == cudaSuccess) e = cudaMemset(c->st, 0, sizeof(LevelState));
  if (e == cudaSuccess) e = cudaMallocHost(&c->pin, 64);
  if (e == cudaSuccess) e = cudaMallocHost(&c->pin_state, sizeof(LevelState));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  for (int k = 0; k < 4 && e == cudaSuccess; k++) e = cudaEventCreate(&c->ev[k]);
  if (e != cudaSuccess) {
    np_destroy(c);
    return from_cuda(e);
  }
  *out = c;
  return NP_OK;
}

np_status np_destroy(np_ctx* c) {
  if (!c) return NP_ERR_INVALID;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  drop_graphs(c);
  if (c->ws) cudaFree(c->ws);
  if (c->stage) cudaFree(c->stage);
  if (c->st) cudaFree(c->st);
  if (c->pin) cudaFreeHost(c->pin);
  if (c->pin_state) cudaFreeHost(c->pin_state);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  for (int k = 0; k < 4; k++)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  delete c;
  return NP_OK;
}

np_status np_workspace_size(int64_t max_parents, const np_config* cfg, size_t* bytes) {
  if (!bytes || max_parents < 0) return NP_ERR_INVALID;
  if (cfg && check_config(cfg) != NP_OK) return NP_ERR_INVALID;
  *bytes = layout_for(max_parents < 4096 ? 4096 : max_parents, 0).total + sizeof(LevelState);
  return NP_OK;
}

np_status np_sync(np_ctx* c, void* stream, np_stats* stats) {
  if (!c) return NP_ERR_INVALID;
  np_stats tmp;
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->device));
  return finish(c, (cudaStream_t)stream, stats ? stats : &tmp);
}

np_status np_bfs(np_ctx* c, const np_csr* g, int32_t src, int32_t* level, const np_config* cfg, void* stream,
                 np_stats* stats) {
  return solve(c, 0, g, src, level, nullptr, cfg, (cudaStream_t)stream, stats);
}

np_status np_sssp(np_ctx* c, const np_csr* g, int32_t src, uint32_t* dist, const np_config* cfg, void* stream,
                  np_stats* stats) {
  return solve(c, 1, g, src, nullptr, dist, cfg, (cudaStream_t)stream, stats);
}

np_status np_bezier(np_ctx* c, const float* ctrl, int32_t ncurves, int32_t* offsets, float* points, int64_t cap,
                    const np_config* cfg, void* stream, np_stats* stats) {
  if (!c || (ncurves > 0 && !ctrl) || !offsets || ncurves < 0 || cap < 0 || (cap > 0 && !points))
    return NP_ERR_INVALID;
  np_status st = check_config(cfg);
  if (st != NP_OK) return st;
  if (ncurves == 0) {
    std::lock_guard<std::mutex> lk(c->mu);
    NP_CK(cudaSetDevice(c->device));
    NP_CK(cudaMemsetAsync(offsets, 0, sizeof(int32_t), (cudaStream_t)stream));
    return stats ? finish(c, (cudaStream_t)stream, stats) : NP_OK;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->device));
  st = ensure_workspace(c, ncurves);
  if (st != NP_OK) return st;
  Args a;
  base_args(c, *cfg, a);
  a.count_fixed = ncurves;
  a.L_fixed = 0;
  a.b.ctrl = ctrl;
  a.b.points = reinterpret_cast<float2*>(points);
  a.offsets = offsets;
  a.cap = cap;
  st = fixed_pass(c, a, *cfg, bezier_kernels(), ncurves, (cudaStream_t)stream);
  if (st != NP_OK) return st;
  return finish(c, (cudaStream_t)stream, stats);
}

np_status np_run_nested(np_ctx* c, const np_parents* parents, int32_t count_kind, const np_csr* g,
                        const np_body* body, const np_config* cfg, void* stream, np_stats* stats) {
  if (!c || !parents || !body || parents->count < 0) return NP_ERR_INVALID;
  np_status st = check_config(cfg);
  if (st != NP_OK) return st;
  const BodyKernels* K = nullptr;
  if (count_kind == NP_COUNT_CSR_DEGREE) {
    if (body->kind == NP_BODY_BFS_VISIT) {
      st = check_csr(g, false);
      if (st != NP_OK) return st;
      if (!body->level || !body->next || !body->next_count || body->next_level < 1) return NP_ERR_INVALID;
      K = &bfs_kernels();
    } else if (body->kind == NP_BODY_SSSP_RELAX) {
      st = check_csr(g, true);
      if (st != NP_OK) return st;
      if (!body->dist || !body->stamp || !body->next || !body->next_count || body->iteration < 1)
        return NP_ERR_INVALID;
      K = &sssp_kernels();
    } else {
      return NP_ERR_UNSUPPORTED;
    }
  } else if (count_kind == NP_COUNT_BEZIER) {
    if (body->kind != NP_BODY_BEZIER_EVAL) return NP_ERR_UNSUPPORTED;
    if (!body->ctrl || !body->offsets || body->cap < 0 || (body->cap > 0 && !body->points)) return NP_ERR_INVALID;
    K = &bezier_kernels();
  } else {
    return NP_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (parents->count == 0) {
    if (count_kind == NP_COUNT_BEZIER) NP_CK(cudaMemsetAsync(body->offsets, 0, sizeof(int32_t), s));
    return stats ? finish(c, s, stats) : NP_OK;
  }
  st = ensure_workspace(c, parents->count);
  if (st != NP_OK) return st;
  Args a;
  base_args(c, *cfg, a);
  a.count_fixed = parents->count;
  a.ids = parents->ids;
  if (g) {
    a.row_ptr = g->row_ptr;
    a.b.col = g->col_idx;
    a.b.w = g->weights;
  }
  a.next_ovr = body->next;
  a.next_count_ovr = body->next_count;
  if (body->kind == NP_BODY_BFS_VISIT) {
    a.L_fixed = body->next_level - 1;
    a.b.level = body->level;
  } else if (body->kind == NP_BODY_SSSP_RELAX) {
    a.L_fixed = body->iteration - 1;
    a.b.dist = body->dist;
    a.b.stamp = body->stamp;
  } else {
    a.b.ctrl = body->ctrl;
    a.b.points = reinterpret_cast<float2*>(body->points);
    a.offsets = body->offsets;
    a.cap = body->cap;
  }
  st = fixed_pass(c, a, *cfg, *K, parents->count, s);
  if (st != NP_OK) return st;
  return finish(c, s, stats);
}

np_status np_bfs_host(np_ctx* c, int32_t n, int64_t m, const int32_t* row_ptr_host, const int32_t* col_idx_host,
                      int32_t src, int32_t* level_host, const np_config* cfg, void* stream, np_stats* stats) {
  if (!c || n < 1 || m < 0 || m >= INT_MAX || !row_ptr_host || (m > 0 && !col_idx_host) || !level_host)
    return NP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  size_t b_rp = align_up(sizeof(int32_t) * ((size_t)n + 1)), b_col = align_up(sizeof(int32_t) * (size_t)m);
  size_t b_out = align_up(sizeof(int32_t) * (size_t)n);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    NP_CK(cudaSetDevice(c->device));
    np_status st = stage_bytes(c, b_rp + b_col + b_out);
    if (st != NP_OK) return st;
  }
  int32_t* d_rp = reinterpret_cast<int32_t*>(c->stage);
  int32_t* d_col = reinterpret_cast<int32_t*>(c->stage + b_rp);
  int32_t* d_out = reinterpret_cast<int32_t*>(c->stage + b_rp + b_col);
  NP_CK(cudaMemcpyAsync(d_rp, row_ptr_host, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
  if (m) NP_CK(cudaMemcpyAsync(d_col, col_idx_host, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
  np_csr g{d_rp, d_col, nullptr, n, m};
  np_status st = np_bfs(c, &g, src, d_out, cfg, stream, nullptr);
  if (st != NP_OK) return st;
  NP_CK(cudaMemcpyAsync(level_host, d_out, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  np_stats tmp;
  return np_sync(c, stream, stats ? stats : &tmp);
}

np_status np_sssp_host(np_ctx* c, int32_t n, int64_t m, const int32_t* row_ptr_host, const int32_t* col_idx_host,
                       const uint32_t* weights_host, int32_t src, uint32_t* dist_host, const np_config* cfg,
                       void* stream, np_stats* stats) {
  if (!c || n < 1 || m < 0 || m >= INT_MAX || !row_ptr_host || (m > 0 && (!col_idx_host || !weights_host)) ||
      !dist_host)
    return NP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  size_t b_rp = align_up(sizeof(int32_t) * ((size_t)n + 1)), b_col = align_up(sizeof(int32_t) * (size_t)m);
  size_t b_out = align_up(sizeof(uint32_t) * (size_t)n);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    NP_CK(cudaSetDevice(c->device));
    np_status st = stage_bytes(c, b_rp + 2 * b_col + b_out);
    if (st != NP_OK) return st;
  }
  int32_t* d_rp = reinterpret_cast<int32_t*>(c->stage);
  int32_t* d_col = reinterpret_cast<int32_t*>(c->stage + b_rp);
  uint32_t* d_w = reinterpret_cast<uint32_t*>(c->stage + b_rp + b_col);
  uint32_t* d_out = reinterpret_cast<uint32_t*>(c->stage + b_rp + 2 * b_col);
  NP_CK(cudaMemcpyAsync(d_rp, row_ptr_host, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
  if (m) {
    NP_CK(cudaMemcpyAsync(d_col, col_idx_host, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    NP_CK(cudaMemcpyAsync(d_w, weights_host, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
  }
  np_csr g{d_rp, d_col, d_w, n, m};
  np_status st = np_sssp(c, &g, src, d_out, cfg, stream, nullptr);
  if (st != NP_OK) return st;
  NP_CK(cudaMemcpyAsync(dist_host, d_out, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  np_stats tmp;
  return np_sync(c, stream, stats ? stats : &tmp);
}

np_status np_profile_enable(np_ctx* c, int32_t on) {
  if (!c) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  c->profile = on != 0;
  return NP_OK;
}

np_status np_profile_read(np_ctx* c, np_profile* out, int32_t reset) {
  if (!c || !out) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->prof;
  if (reset) c->prof = np_profile{};
  return NP_OK;
}

np_status np_bezier_host(np_ctx* c, const float* ctrl_host, int32_t ncurves, int32_t* offsets_host,
                         float* points_host, int64_t cap, const np_config* cfg, void* stream, np_stats* stats) {
  if (!c || ncurves < 0 || (ncurves > 0 && !ctrl_host) || !offsets_host || cap < 0 || (cap > 0 && !points_host))
    return NP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b_ctrl = align_up(sizeof(float) * 6 * (size_t)ncurves), b_off = align_up(sizeof(int32_t) * ((size_t)ncurves + 1));
  const size_t b_pts = align_up(sizeof(float) * 2 * (size_t)cap);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    NP_CK(cudaSetDevice(c->device));
    np_status st = stage_bytes(c, b_ctrl + b_off + b_pts + 256);
    if (st != NP_OK) return st;
  }
  float* d_ctrl = reinterpret_cast<float*>(c->stage);
  int32_t* d_off = reinterpret_cast<int32_t*>(c->stage + b_ctrl);
  float* d_pts = reinterpret_cast<float*>(c->stage + b_ctrl + b_off);
  if (ncurves) NP_CK(cudaMemcpyAsync(d_ctrl, ctrl_host, sizeof(float) * 6 * (size_t)ncurves, cudaMemcpyHostToDevice, s));
  np_status st = np_bezier(c, d_ctrl, ncurves, d_off, d_pts, cap, cfg, stream, nullptr);
  if (st != NP_OK) return st;
  NP_CK(cudaMemcpyAsync(offsets_host, d_off, sizeof(int32_t) * ((size_t)ncurves + 1), cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  const int64_t total = offsets_host[ncurves] < cap ? offsets_host[ncurves] : cap;
  if (total > 0) NP_CK(cudaMemcpyAsync(points_host, d_pts, sizeof(float) * 2 * (size_t)total, cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  np_stats tmp;
  return np_sync(c, stream, stats ? stats : &tmp);
}

const char* np_status_string(np_status s) {
  switch (s) {
    case NP_OK: return "ok";
    case NP_ERR_INVALID: return "invalid argument";
    case NP_ERR_CUDA: return "CUDA error";
    case NP_ERR_NOMEM: return "out of device memory";
    case NP_ERR_CAPACITY: return "output capacity too small";
    case NP_ERR_LAUNCH: return "device-side launch refused (work serialised)";
    case NP_ERR_TIMEOUT: return "bounded device wait expired";
    case NP_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
  }
}

int32_t np_version(void) { return kVersion; }

}  // extern "C"
