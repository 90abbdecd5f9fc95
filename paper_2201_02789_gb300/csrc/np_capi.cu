// Host C ABI of the single-solve entry points (include/nestpar.h): whole
// BFS / SSSP solves, tessellation, one nesting pass over an explicit parent
// set, several traversals of one graph at once, host-buffer variants and the
// execution-time breakdown. The level-loop machinery is in np_engine.cu.
#include <cuda_runtime.h>

#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "nestpar.h"
#include "np_engine.h"

using namespace nestpar;

struct np_ctx {
  Engine e;
  Workspace w;
  int* ids = nullptr;                 // device copy of the sources of a multi-source solve
  int ids_cap = 0;
  unsigned long long* tri = nullptr;  // triangle-counting partial sums [kTcSlots]
  unsigned long long* dtag = nullptr; // packed SSSP state (dist << 32 | tag) of np_sssp / np_sssp_multi
  int64_t dtag_cap = 0;
  // device staging for the *_host entry points
  unsigned char* stage = nullptr;
  size_t stage_bytes = 0;
  std::mutex mu;
};

int nestpar_ctx_device(const np_ctx* c) { return c->e.device; }

namespace {

np_status ensure_dtag(np_ctx* c, int64_t total) {
  if (total <= c->dtag_cap) return NP_OK;
  if (c->dtag) {
    NP_CK(cudaDeviceSynchronize());
    cudaFree(c->dtag);
    c->dtag = nullptr;
    c->dtag_cap = 0;
  }
  NP_CK(cudaMalloc(&c->dtag, sizeof(unsigned long long) * (size_t)total));
  c->dtag_cap = total;
  return NP_OK;
}


constexpr int kVersion = 10200;  // 1.2.0

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
  NP_CK(cudaSetDevice(c->e.device));
  st = ws_ensure(c->w, g->n);
  if (st != NP_OK) return st;
  // SSSP runs in the packed form (distance and append tag in one word)
  const BodyKernels& K = kind == 0 ? bfs_kernels() : sssp64_kernels();
  Plan p = make_plan(K, *cfg);
  Args a;
  base_args(c->w, *cfg, a);
  a.row_ptr = g->row_ptr;
  a.b.col = g->col_idx;
  a.b.w = g->weights;
  a.b.level = level;
  a.b.dist = dist;
  a.b.stamp = wsp<int>(c->w, c->w.lay.off_stamp);
  if (p.sweep) a.n_vertices = g->n;
  if (kind == 1) {
    NP_TRY(ensure_dtag(c, g->n));
    a.b.dtag = c->dtag;
  }
  const int blocks = (int)((g->n + 255) / 256 < 4096 ? (g->n + 255) / 256 : 4096);
  if (c->e.profile) NP_CK(cudaEventRecord(c->e.ev[0], s));
  if (kind == 1)
    init_dtag_solve_kernel<<<blocks, 256, 0, s>>>(c->w.st, g->n, src, c->dtag, a.fr0, g->n + 2);
  else
    init_solve_kernel<<<blocks, 256, 0, s>>>(c->w.st, kind, g->n, src, level, dist, a.b.stamp, a.fr0, g->n + 2);
  NP_CK(cudaGetLastError());
  if (c->e.profile) {
    NP_CK(cudaEventRecord(c->e.ev[3], s));
    NP_CK(cudaEventSynchronize(c->e.ev[3]));
    float t = 0.f;
    NP_CK(cudaEventElapsedTime(&t, c->e.ev[0], c->e.ev[3]));
    c->e.prof.other_ms += t;
    c->e.prof.other_launches += 1;
  }
  c->e.prof_next_parents = 1;
  st = run_levels(c->e, c->w, p, a, *cfg, g->n, g->n + 2, s);
  if (st != NP_OK) return st;
  if (kind == 1) {
    dtag_to_dist_kernel<<<blocks, 256, 0, s>>>(g->n, c->dtag, dist);
    NP_CK(cudaGetLastError());
  }
  return finish(c->e, c->w, s, stats);
}

// Several traversals of one graph in one level loop: query q is vertex ids
// q * ld + v (ld a power of two >= n), so the frontiers of all queries form
// one parent set and their children aggregate into the same child grids.
np_status solve_multi(np_ctx* c, int kind, const np_csr* g, int nsrc, const int32_t* sources, int* level,
                      unsigned* dist, int64_t ld, const np_config* cfg, cudaStream_t s, np_stats* stats) {
  if (!c) return NP_ERR_INVALID;
  NP_TRY(check_config(cfg));
  NP_TRY(check_csr(g, kind == 1));
  if (nsrc < 1 || !sources || (kind == 0 && !level) || (kind == 1 && !dist)) return NP_ERR_INVALID;
  if (ld < g->n || (ld & (ld - 1)) != 0 || (int64_t)nsrc * ld > (int64_t)INT_MAX) return NP_ERR_INVALID;
  std::vector<int> ids((size_t)nsrc);
  for (int q = 0; q < nsrc; q++) {
    if (sources[q] < 0 || sources[q] >= g->n) return NP_ERR_INVALID;
    ids[(size_t)q] = (int)((int64_t)q * ld + sources[q]);
  }
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->e.device));
  const int64_t total = (int64_t)nsrc * ld;
  NP_TRY(ws_ensure(c->w, total));
  if (nsrc > c->ids_cap) {
    if (c->ids) {
      NP_CK(cudaDeviceSynchronize());
      cudaFree(c->ids);
      c->ids = nullptr;
      c->ids_cap = 0;
    }
    NP_CK(cudaMalloc(&c->ids, sizeof(int) * (size_t)nsrc));
    c->ids_cap = nsrc;
  }
  NP_CK(cudaMemcpyAsync(c->ids, ids.data(), sizeof(int) * (size_t)nsrc, cudaMemcpyHostToDevice, s));
  const BodyKernels& K = kind == 0 ? bfs_kernels() : sssp64_kernels();
  np_config mcfg = serial_for(*cfg, nsrc, g->m);
  Plan p = make_plan(K, mcfg);
  Args a;
  base_args(c->w, mcfg, a);
  a.row_ptr = g->row_ptr;
  a.b.col = g->col_idx;
  a.b.w = g->weights;
  a.b.level = level;
  a.b.dist = dist;
  a.b.stamp = wsp<int>(c->w, c->w.lay.off_stamp);
  a.b.vmask = (int)(ld - 1);
  // a swept frontier sweeps every query's state (padding entries stay unreached)
  if (p.sweep) a.n_vertices = (int)total;
  if (kind == 1) {
    NP_TRY(ensure_dtag(c, total));
    a.b.dtag = c->dtag;
    init_dtag_kernel<<<blocks_for(total), 256, 0, s>>>(total, c->dtag);
    NP_CK(cudaGetLastError());
    seed_dtag_kernel<<<blocks_for(nsrc), 256, 0, s>>>(c->w.st, c->ids, nsrc, c->dtag, a.fr0, g->n + 2);
  } else {
    fill_unreached_kernel<<<blocks_for(total), 256, 0, s>>>(kind, total, level, dist, a.b.stamp);
    NP_CK(cudaGetLastError());
    seed_sources_kernel<<<blocks_for(nsrc), 256, 0, s>>>(c->w.st, kind, c->ids, nsrc, level, dist, a.fr0, g->n + 2);
  }
  NP_CK(cudaGetLastError());
  c->e.prof_next_parents = nsrc;
  NP_TRY(run_levels(c->e, c->w, p, a, mcfg, total, g->n + 2, s));
  if (kind == 1) {
    dtag_to_dist_kernel<<<blocks_for(total), 256, 0, s>>>(total, c->dtag, dist);
    NP_CK(cudaGetLastError());
  }
  return finish(c->e, c->w, s, stats);
}

// One fixed pass over an explicit parent set.
np_status fixed_pass(np_ctx* c, const Args& a0, const np_config& cfg, const BodyKernels& K, int count,
                     cudaStream_t s) {
  Plan p = make_plan(K, cfg);
  Args a = a0;
  Grids g = grids_for(c->e, p, cfg, count);
  if (c->e.profile) {
    NP_CK(cudaEventRecord(c->e.ev[0], s));
    init_fixed_kernel<<<1, 1, 0, s>>>(c->w.st);
    NP_CK(cudaGetLastError());
    NP_CK(cudaEventRecord(c->e.ev[3], s));
    NP_CK(cudaEventSynchronize(c->e.ev[3]));
    float t = 0.f;
    NP_CK(cudaEventElapsedTime(&t, c->e.ev[0], c->e.ev[3]));
    c->e.prof.other_ms += t;
    c->e.prof.other_launches += 1;
    return profiled_pass(c->e, c->w, p, a, g, false, s);
  }
  if (p.mode == M_DEVICE_LAUNCH) {
    // device launches are joined by stream order only (a graph node does not
    // wait for the grids it launches): no graph for these forms
    init_fixed_kernel<<<1, 1, 0, s>>>(c->w.st);
    NP_CK(cudaGetLastError());
    return enqueue_pass(p, a, g, false, 0, s);
  }
  std::string key = graph_key("fixed", p, a, g, 1);
  auto it = c->w.graphs.find(key);
  cudaGraphExec_t exec = nullptr;
  if (it != c->w.graphs.end()) {
    exec = it->second.exec;
  } else {
    NP_CK(cudaStreamBeginCapture(c->e.cap_stream, cudaStreamCaptureModeThreadLocal));
    init_fixed_kernel<<<1, 1, 0, c->e.cap_stream>>>(c->w.st);
    cudaError_t le = cudaGetLastError();
    np_status st = le == cudaSuccess ? enqueue_pass(p, a, g, false, 0, c->e.cap_stream) : from_cuda(le);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->e.cap_stream, &graph);
    if (st != NP_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    NP_CK(e);
    st = cache_graph(c->w, key, graph, &exec);
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

// BFS (kind 0) or SSSP (kind 1) of a CSR graph in host memory: copies the graph
// into the context's staging buffer, solves, copies the result out, all on
// `stream`; with `wait`, then waits and reads the device status.
np_status host_solve(np_ctx* c, int kind, int32_t n, int64_t m, const int32_t* row_ptr_host,
                     const int32_t* col_idx_host, const uint32_t* weights_host, int32_t src, void* out_host,
                     const np_config* cfg, void* stream, np_stats* stats, bool wait) {
  if (!c || n < 1 || m < 0 || m >= INT_MAX || !row_ptr_host || (m > 0 && !col_idx_host) ||
      (kind == 1 && m > 0 && !weights_host) || !out_host)
    return NP_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b_rp = align_up(sizeof(int32_t) * ((size_t)n + 1)), b_col = align_up(sizeof(int32_t) * (size_t)m);
  const size_t b_w = kind == 1 ? b_col : 0, b_out = align_up(sizeof(int32_t) * (size_t)n);
  {
    std::lock_guard<std::mutex> lk(c->mu);
    NP_CK(cudaSetDevice(c->e.device));
    np_status st = stage_bytes(c, b_rp + b_col + b_w + b_out);
    if (st != NP_OK) return st;
  }
  int32_t* d_rp = reinterpret_cast<int32_t*>(c->stage);
  int32_t* d_col = reinterpret_cast<int32_t*>(c->stage + b_rp);
  uint32_t* d_w = kind == 1 ? reinterpret_cast<uint32_t*>(c->stage + b_rp + b_col) : nullptr;
  int32_t* d_out = reinterpret_cast<int32_t*>(c->stage + b_rp + b_col + b_w);
  NP_CK(cudaMemcpyAsync(d_rp, row_ptr_host, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
  if (m) {
    NP_CK(cudaMemcpyAsync(d_col, col_idx_host, sizeof(int32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
    if (kind == 1) NP_CK(cudaMemcpyAsync(d_w, weights_host, sizeof(uint32_t) * (size_t)m, cudaMemcpyHostToDevice, s));
  }
  np_csr g{d_rp, d_col, d_w, n, m};
  np_status st = kind == 1 ? np_sssp(c, &g, src, reinterpret_cast<uint32_t*>(d_out), cfg, stream, nullptr)
                           : np_bfs(c, &g, src, d_out, cfg, stream, nullptr);
  if (st != NP_OK) return st;
  NP_CK(cudaMemcpyAsync(out_host, d_out, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s));
  if (!wait) return NP_OK;
  NP_CK(cudaStreamSynchronize(s));
  np_stats tmp;
  return np_sync(c, stream, stats ? stats : &tmp);
}

}  // namespace

// ======================================================================= C ABI

extern "C" {

np_status np_config_default(np_config* cfg) {
  if (!cfg) return NP_ERR_INVALID;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->variant = NP_VARIANT_CDP;
  cfg->threshold = 32;
  cfg->cfactor = 4;
  cfg->granularity = NP_GRAN_GRID_HOST;
  cfg->group_blocks = 8;
  cfg->agg_threshold = 0;
  cfg->child_block = 64;
  cfg->parent_block = 256;
  cfg->scan = NP_SCAN_ATOMIC;
  cfg->driver = NP_DRIVER_AUTO;
  cfg->unroll = 4;
  cfg->parent_grid = 0;
  cfg->serial = NP_SERIAL_SPREAD;
  cfg->small_parents = NP_SMALL_PARENTS_MAX;
  cfg->sweep_parents = 4096;
  return NP_OK;
}

np_status np_create(np_ctx** out, int32_t device) {
  if (!out) return NP_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  NP_CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return NP_ERR_INVALID;
  NP_CK(cudaSetDevice(device));
  // plain CDP issues one device launch per parent: raise the pending-launch pool
  // (the driver caps the request; refused launches fall back to serial work)
  size_t cur = 0;
  if (cudaDeviceGetLimit(&cur, cudaLimitDevRuntimePendingLaunchCount) == cudaSuccess && cur < (1u << 20))
    cudaDeviceSetLimit(cudaLimitDevRuntimePendingLaunchCount, 1u << 20);
  cudaGetLastError();
  np_ctx* c = new np_ctx();
  np_status st = engine_init(c->e, device);
  if (st == NP_OK) st = ws_init(c->w);
  if (st != NP_OK) {
    np_destroy(c);
    return st;
  }
  *out = c;
  return NP_OK;
}

np_status np_destroy(np_ctx* c) {
  if (!c) return NP_ERR_INVALID;
  cudaSetDevice(c->e.device);
  cudaDeviceSynchronize();
  ws_release(c->w);
  if (c->stage) cudaFree(c->stage);
  if (c->ids) cudaFree(c->ids);
  if (c->tri) cudaFree(c->tri);
  if (c->dtag) cudaFree(c->dtag);
  engine_release(c->e);
  delete c;
  return NP_OK;
}

np_status np_workspace_size(int64_t max_parents, const np_config* cfg, size_t* bytes) {
  if (!bytes || max_parents < 0) return NP_ERR_INVALID;
  if (cfg && check_config(cfg) != NP_OK) return NP_ERR_INVALID;
  *bytes = layout_for(max_parents < 4096 ? 4096 : max_parents).total + sizeof(LevelState);
  return NP_OK;
}

np_status np_sync(np_ctx* c, void* stream, np_stats* stats) {
  if (!c) return NP_ERR_INVALID;
  np_stats tmp;
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->e.device));
  return finish(c->e, c->w, (cudaStream_t)stream, stats ? stats : &tmp);
}

np_status np_bfs(np_ctx* c, const np_csr* g, int32_t src, int32_t* level, const np_config* cfg, void* stream,
                 np_stats* stats) {
  return solve(c, 0, g, src, level, nullptr, cfg, (cudaStream_t)stream, stats);
}

np_status np_sssp(np_ctx* c, const np_csr* g, int32_t src, uint32_t* dist, const np_config* cfg, void* stream,
                  np_stats* stats) {
  return solve(c, 1, g, src, nullptr, dist, cfg, (cudaStream_t)stream, stats);
}

np_status np_triangles(np_ctx* c, const np_csr* dag, uint64_t* count, const np_config* cfg, void* stream,
                       np_stats* stats) {
  if (!c || !count) return NP_ERR_INVALID;
  NP_TRY(check_config(cfg));
  NP_TRY(check_csr(dag, false));
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->e.device));
  cudaStream_t s = (cudaStream_t)stream;
  if (!c->tri) NP_CK(cudaMalloc(&c->tri, sizeof(unsigned long long) * kTcSlots));
  NP_TRY(ws_ensure(c->w, dag->n));
  NP_CK(cudaMemsetAsync(c->tri, 0, sizeof(unsigned long long) * kTcSlots, s));
  Args a;
  base_args(c->w, *cfg, a);
  a.count_fixed = dag->n;
  a.L_fixed = 0;
  a.row_ptr = dag->row_ptr;
  a.b.col = dag->col_idx;
  a.b.row_ptr = dag->row_ptr;
  a.b.acc = c->tri;
  NP_TRY(fixed_pass(c, a, *cfg, tc_kernels(), dag->n, s));
  sum_u64_kernel<<<1, 256, 0, s>>>(c->tri, kTcSlots, reinterpret_cast<unsigned long long*>(count), 0);
  NP_CK(cudaGetLastError());
  return finish(c->e, c->w, s, stats);
}

np_status np_bfs_multi(np_ctx* c, const np_csr* g, int32_t nsrc, const int32_t* sources, int32_t* level, int64_t ld,
                       const np_config* cfg, void* stream, np_stats* stats) {
  return solve_multi(c, 0, g, nsrc, sources, level, nullptr, ld, cfg, (cudaStream_t)stream, stats);
}

np_status np_sssp_multi(np_ctx* c, const np_csr* g, int32_t nsrc, const int32_t* sources, uint32_t* dist, int64_t ld,
                        const np_config* cfg, void* stream, np_stats* stats) {
  return solve_multi(c, 1, g, nsrc, sources, nullptr, dist, ld, cfg, (cudaStream_t)stream, stats);
}

np_status np_bezier(np_ctx* c, const float* ctrl, int32_t ncurves, int32_t* offsets, float* points, int64_t cap,
                    const np_config* cfg, void* stream, np_stats* stats) {
  if (!c || (ncurves > 0 && !ctrl) || !offsets || ncurves < 0 || cap < 0 || (cap > 0 && !points))
    return NP_ERR_INVALID;
  np_status st = check_config(cfg);
  if (st != NP_OK) return st;
  if (ncurves == 0) {
    std::lock_guard<std::mutex> lk(c->mu);
    NP_CK(cudaSetDevice(c->e.device));
    NP_CK(cudaMemsetAsync(offsets, 0, sizeof(int32_t), (cudaStream_t)stream));
    return stats ? finish(c->e, c->w, (cudaStream_t)stream, stats) : NP_OK;
  }
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->e.device));
  st = ws_ensure(c->w, ncurves);
  if (st != NP_OK) return st;
  Args a;
  base_args(c->w, *cfg, a);
  a.count_fixed = ncurves;
  a.L_fixed = 0;
  a.b.ctrl = ctrl;
  a.b.points = reinterpret_cast<float2*>(points);
  a.offsets = offsets;
  a.cap = cap;
  st = fixed_pass(c, a, *cfg, bezier_kernels(), ncurves, (cudaStream_t)stream);
  if (st != NP_OK) return st;
  return finish(c->e, c->w, (cudaStream_t)stream, stats);
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
    } else if (body->kind == NP_BODY_TRIANGLES) {
      st = check_csr(g, false);
      if (st != NP_OK) return st;
      if (!body->tri_counts) return NP_ERR_INVALID;
      K = &tc_kernels();
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
  NP_CK(cudaSetDevice(c->e.device));
  cudaStream_t s = (cudaStream_t)stream;
  if (parents->count == 0) {
    if (count_kind == NP_COUNT_BEZIER) NP_CK(cudaMemsetAsync(body->offsets, 0, sizeof(int32_t), s));
    return stats ? finish(c->e, c->w, s, stats) : NP_OK;
  }
  st = ws_ensure(c->w, parents->count);
  if (st != NP_OK) return st;
  Args a;
  base_args(c->w, *cfg, a);
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
  } else if (body->kind == NP_BODY_TRIANGLES) {
    a.L_fixed = 0;
    a.b.row_ptr = g->row_ptr;
    a.b.acc = reinterpret_cast<unsigned long long*>(body->tri_counts);
  } else {
    a.b.ctrl = body->ctrl;
    a.b.points = reinterpret_cast<float2*>(body->points);
    a.offsets = body->offsets;
    a.cap = body->cap;
  }
  st = fixed_pass(c, a, *cfg, *K, parents->count, s);
  if (st != NP_OK) return st;
  return finish(c->e, c->w, s, stats);
}

np_status np_bfs_host(np_ctx* c, int32_t n, int64_t m, const int32_t* row_ptr_host, const int32_t* col_idx_host,
                      int32_t src, int32_t* level_host, const np_config* cfg, void* stream, np_stats* stats) {
  return host_solve(c, 0, n, m, row_ptr_host, col_idx_host, nullptr, src, level_host, cfg, stream, stats, true);
}

np_status np_sssp_host(np_ctx* c, int32_t n, int64_t m, const int32_t* row_ptr_host, const int32_t* col_idx_host,
                       const uint32_t* weights_host, int32_t src, uint32_t* dist_host, const np_config* cfg,
                       void* stream, np_stats* stats) {
  return host_solve(c, 1, n, m, row_ptr_host, col_idx_host, weights_host, src, dist_host, cfg, stream, stats, true);
}

np_status np_bfs_host_async(np_ctx* c, int32_t n, int64_t m, const int32_t* row_ptr_host,
                            const int32_t* col_idx_host, int32_t src, int32_t* level_host, const np_config* cfg,
                            void* stream) {
  return host_solve(c, 0, n, m, row_ptr_host, col_idx_host, nullptr, src, level_host, cfg, stream, nullptr, false);
}

np_status np_sssp_host_async(np_ctx* c, int32_t n, int64_t m, const int32_t* row_ptr_host,
                             const int32_t* col_idx_host, const uint32_t* weights_host, int32_t src,
                             uint32_t* dist_host, const np_config* cfg, void* stream) {
  return host_solve(c, 1, n, m, row_ptr_host, col_idx_host, weights_host, src, dist_host, cfg, stream, nullptr,
                    false);
}

np_status np_selftest_wait(np_ctx* c, int32_t which, int64_t limit_ns, void* stream) {
  if (!c || which < 0 || which > 1) return NP_ERR_INVALID;
  if (which == 1 && (limit_ns < 1000000 || limit_ns > 10000000000ll)) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  NP_CK(cudaSetDevice(c->e.device));
  cudaStream_t s = (cudaStream_t)stream;
  NP_TRY(ws_ensure(c->w, 4096));
  if (which == 0) {
    np_config cfg;
    np_config_default(&cfg);
    Args a;
    base_args(c->w, cfg, a);
    selftest_lookback_kernel<<<1, 32, 0, s>>>(a);
    NP_CK(cudaGetLastError());
  } else {
    LevelState* st = c->w.st;
    NP_CK(cudaMemsetAsync(&st->bar_count, 0, sizeof(unsigned), s));   // no stale arrivals
    unsigned long long lim = (unsigned long long)limit_ns;
    void* args[] = {&st, &lim};
    NP_CK(cudaLaunchCooperativeKernel((const void*)selftest_barrier_kernel, dim3(2), dim3(32), args, 0, s));
    // the next solve resets the barrier's arrival count (it is left at one)
  }
  np_stats tmp;
  return finish(c->e, c->w, s, &tmp);
}

np_status np_profile_enable(np_ctx* c, int32_t on) {
  if (!c) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  c->e.profile = on != 0;
  return NP_OK;
}

np_status np_profile_read(np_ctx* c, np_profile* out, int32_t reset) {
  if (!c || !out) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(c->mu);
  *out = c->e.prof;
  if (reset) c->e.prof = np_profile{};
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
    NP_CK(cudaSetDevice(c->e.device));
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
