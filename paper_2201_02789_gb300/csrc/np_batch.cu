// Batched solves (np_batch_*): many independent BFS / SSSP instances in one
// CUDA graph launch, with a per-size-class configuration and autotuner.
//
// Instances are grouped by size class (floor(log2 n), `width` powers of two
// per class) and each class is split into groups of bounded edge count. A
// group's instances are copied into one disjoint-union CSR (vertex ids and
// edge offsets shifted), so a multi-source traversal of the union from every
// instance's source gives each instance exactly its own result: no path
// crosses between components. Every group owns a Workspace (level state,
// frontiers, aggregation scratch); the batch graph has one branch per group:
// unreached fill -> source seeding -> conditional-while level loop. Branches
// share no state, so they run concurrently; none waits on another's blocks.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <mutex>
#include <vector>

#include "np_engine.h"

using namespace nestpar;

namespace {

__global__ void union_append_kernel(int* rp, int* col, unsigned* w, const int* srp, const int* scol,
                                    const unsigned* sw, int n, long long m, int voff, long long eoff) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long top = n > m ? (long long)n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < top; i += stride) {
    if (i < n) rp[voff + i] = (int)(srp[i] + eoff);
    if (i < m) {
      col[eoff + i] = scol[i] + voff;
      if (w) w[eoff + i] = sw[i];
    }
  }
}

struct Group {
  int cls = 0;
  int64_t vbase = 0;            // first element of the group in the result array
  int n = 0;
  int64_t m = 0;
  int* row_ptr = nullptr;       // union CSR (one allocation: row_ptr | col | w | ids)
  int* col = nullptr;
  unsigned* w = nullptr;
  int* ids = nullptr;           // union ids of the instances' sources
  unsigned long long* dtag = nullptr;   // SSSP: packed distance and append tag per vertex
  int nsrc = 0;
  unsigned char* mem = nullptr;
  Workspace ws;
  std::vector<int> members;
};

struct Class {
  int log2_lo = 0;
  std::vector<int> groups;
  np_config cfg{};
  double tuned_ms = 0.0;
  int candidates = 0;
  double dl_ms = 0.0;            // the fastest device-launch candidate (reported, not picked)
  int dl_gran = 0, dl_threshold = 0;
  int instances = 0;
  int64_t vertices = 0, edges = 0;
};

int floor_log2(int64_t n) {
  int k = 0;
  while ((int64_t(1) << (k + 1)) <= n) k++;
  return k;
}

bool batch_form_ok(const np_config& c) {
  return c.variant == NP_VARIANT_NODP || (c.variant == NP_VARIANT_CDP && c.granularity == NP_GRAN_GRID_HOST);
}

}  // namespace

struct np_batch {
  Engine e;
  int kind = 0;
  int width = 2;
  std::vector<Group> groups;
  std::vector<Class> classes;
  std::vector<int64_t> offsets;   // per instance, into the result array
  int64_t total = 0;
  int count = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* graph_out = nullptr;
  std::mutex mu;
};

namespace {

void drop_batch_graph(np_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->graph_out = nullptr;
}

// SSSP groups run in the packed form (distance and append tag in one word)
const BodyKernels& kernels_of(int kind) { return kind == 0 ? bfs_kernels() : sssp64_kernels(); }

void group_args(np_batch* b, Group& g, const np_config& cfg, void* out, Args& a) {
  base_args(g.ws, cfg, a);
  a.row_ptr = g.row_ptr;
  a.b.col = g.col;
  a.b.w = g.w;
  a.b.level = b->kind == 0 ? reinterpret_cast<int*>(out) + g.vbase : nullptr;
  a.b.dist = b->kind == 1 ? reinterpret_cast<unsigned*>(out) + g.vbase : nullptr;
  a.b.stamp = wsp<int>(g.ws, g.ws.lay.off_stamp);
  a.b.dtag = g.dtag;
  a.n_vertices = g.n;   // (a swept frontier sweeps the group's union)
}

// fill + seed for one group on stream s (used by the tuner)
np_status enqueue_group_init(np_batch* b, Group& g, const Args& a, cudaStream_t s) {
  if (b->kind == 1) {
    init_dtag_kernel<<<blocks_for(g.n), 256, 0, s>>>(g.n, g.dtag);
    NP_CK(cudaGetLastError());
    seed_dtag_kernel<<<blocks_for(g.nsrc), 256, 0, s>>>(g.ws.st, g.ids, g.nsrc, g.dtag, a.fr0, g.n + 2);
  } else {
    fill_unreached_kernel<<<blocks_for(g.n), 256, 0, s>>>(b->kind, g.n, a.b.level, a.b.dist, a.b.stamp);
    NP_CK(cudaGetLastError());
    seed_sources_kernel<<<blocks_for(g.nsrc), 256, 0, s>>>(g.ws.st, b->kind, g.ids, g.nsrc, a.b.level, a.b.dist,
                                                           a.fr0, g.n + 2);
  }
  NP_CK(cudaGetLastError());
  return NP_OK;
}

// SSSP: the group's distances out of the packed state
np_status enqueue_group_result(np_batch* b, Group& g, const Args& a, cudaStream_t s) {
  if (b->kind != 1) return NP_OK;
  dtag_to_dist_kernel<<<blocks_for(g.n), 256, 0, s>>>(g.n, g.dtag, a.b.dist);
  NP_CK(cudaGetLastError());
  return NP_OK;
}

np_status add_kernel_node(cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps, const void* fn, int grid,
                          int block, void** args, cudaGraphNode_t* node) {
  cudaKernelNodeParams kp = {};
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  kp.extra = nullptr;
  NP_CK(cudaGraphAddKernelNode(node, graph, deps, ndeps, &kp));
  return NP_OK;
}

np_status build_batch_graph(np_batch* b, void* out) {
  drop_batch_graph(b);
  cudaGraph_t graph = nullptr;
  NP_CK(cudaGraphCreate(&graph, 0));
  for (Group& g : b->groups) {
    const np_config& cfg = b->classes[(size_t)g.cls].cfg;
    Plan p = make_plan(kernels_of(b->kind), cfg);
    Args a;
    group_args(b, g, cfg, out, a);
    Grids gr = grids_for(b->e, p, cfg, g.n);
    int kind = b->kind;
    long long total = g.n;
    int* level = a.b.level;
    unsigned* dist = a.b.dist;
    int* stamp = a.b.stamp;
    void* fill_args[] = {&kind, &total, &level, &dist, &stamp};
    unsigned long long* dtag = g.dtag;
    void* fill64_args[] = {&total, &dtag};
    cudaGraphNode_t n1, n2, n3, n4;
    np_status st = kind == 1 ? add_kernel_node(graph, nullptr, 0, (const void*)init_dtag_kernel, blocks_for(g.n), 256,
                                               fill64_args, &n1)
                             : add_kernel_node(graph, nullptr, 0, (const void*)fill_unreached_kernel, blocks_for(g.n),
                                               256, fill_args, &n1);
    LevelState* lst = g.ws.st;
    const int* ids = g.ids;
    int nsrc = g.nsrc;
    int* fr0 = a.fr0;
    int maxl = g.n + 2;
    void* seed_args[] = {&lst, &kind, &ids, &nsrc, &level, &dist, &fr0, &maxl};
    void* seed64_args[] = {&lst, &ids, &nsrc, &dtag, &fr0, &maxl};
    if (st == NP_OK)
      st = kind == 1 ? add_kernel_node(graph, &n1, 1, (const void*)seed_dtag_kernel, blocks_for(g.nsrc), 256,
                                       seed64_args, &n2)
                     : add_kernel_node(graph, &n1, 1, (const void*)seed_sources_kernel, blocks_for(g.nsrc), 256,
                                       seed_args, &n2);
    if (st == NP_OK) st = add_while_node(b->e, g.ws.st, graph, &n2, 1, p, a, gr, cfg.unroll, &n3);
    void* out64_args[] = {&total, &dtag, &dist};
    if (st == NP_OK && kind == 1)
      st = add_kernel_node(graph, &n3, 1, (const void*)dtag_to_dist_kernel, blocks_for(g.n), 256, out64_args, &n4);
    if (st != NP_OK) {
      cudaGraphDestroy(graph);
      return st;
    }
  }
  cudaGraphExec_t exec = nullptr;
  np_status st = instantiate(graph, &exec);
  if (st != NP_OK) {
    cudaGraphDestroy(graph);
    return st;
  }
  b->graph = graph;
  b->exec = exec;
  b->graph_out = out;
  return NP_OK;
}

void add_stats(np_stats& acc, const np_stats& s) {
  acc.levels += s.levels;
  acc.parents += s.parents;
  acc.serial_parents += s.serial_parents;
  acc.launch_parents += s.launch_parents;
  acc.device_launches += s.device_launches;
  acc.aggregated_grids += s.aggregated_grids;
  acc.child_blocks += s.child_blocks;
  acc.items += s.items;
  acc.pushes += s.pushes;
  acc.launch_failures += s.launch_failures;
  acc.timeouts += s.timeouts;
  acc.child_items += s.child_items;
  acc.graph_iterations += s.graph_iterations;
  acc.error |= s.error;
}

np_status batch_stats(np_batch* b, cudaStream_t s, np_stats* stats) {
  np_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  np_status worst = NP_OK;
  for (Group& g : b->groups) {
    np_stats one;
    np_status st = finish(b->e, g.ws, s, &one);
    if (st != NP_OK && worst == NP_OK) worst = st;
    add_stats(acc, one);
  }
  if (stats) *stats = acc;
  return worst;
}

// Runs the groups of class `ci` alone under cfg, reps times; min time in ms.
// Device-launch forms run as stream-ordered launches (host-replayed level
// chunks); a launch the device refused ran serially and still gave the exact
// result, so with tolerate_launch it does not fail the timing.
np_status time_class(np_batch* b, int ci, const np_config& cfg, void* out, int reps, cudaStream_t s, double* ms,
                     bool tolerate_launch = false) {
  Class& c = b->classes[(size_t)ci];
  Plan p = make_plan(kernels_of(b->kind), cfg);
  double best = 1e30;
  for (int r = 0; r < reps; r++) {
    NP_CK(cudaEventRecord(b->e.ev[0], s));
    for (int gi : c.groups) {
      Group& g = b->groups[(size_t)gi];
      Args a;
      group_args(b, g, cfg, out, a);
      NP_TRY(enqueue_group_init(b, g, a, s));
      NP_TRY(run_levels(b->e, g.ws, p, a, cfg, g.n, g.n + 2, s));
      NP_TRY(enqueue_group_result(b, g, a, s));
    }
    NP_CK(cudaEventRecord(b->e.ev[1], s));
    NP_CK(cudaEventSynchronize(b->e.ev[1]));
    float t = 0.f;
    NP_CK(cudaEventElapsedTime(&t, b->e.ev[0], b->e.ev[1]));
    if (t < best) best = t;
  }
  for (int gi : c.groups) {
    np_stats one;
    const np_status fs = finish(b->e, b->groups[(size_t)gi].ws, s, &one);
    if (fs != NP_OK && !(tolerate_launch && fs == NP_ERR_LAUNCH)) return fs;
  }
  *ms = best;
  return NP_OK;
}

}  // namespace

int nestpar_ctx_device(const np_ctx* c);

extern "C" {

np_status np_batch_create(np_ctx* ctx, int32_t count, const np_csr* graphs, const int32_t* sources,
                          const np_batch_options* opt, np_batch** out) {
  if (!ctx || count < 1 || !graphs || !sources || !opt || !out) return NP_ERR_INVALID;
  *out = nullptr;
  if (opt->kind != NP_BATCH_BFS && opt->kind != NP_BATCH_SSSP) return NP_ERR_INVALID;
  const int width = opt->class_log2_width == 0 ? 2 : opt->class_log2_width;
  if (width < 1 || width > 31) return NP_ERR_INVALID;
  const int64_t max_edges = opt->max_group_edges == 0 ? (int64_t(1) << 30) : opt->max_group_edges;
  if (max_edges < 1 || max_edges >= INT_MAX) return NP_ERR_INVALID;
  NP_TRY(check_config(&opt->config));
  if (!batch_form_ok(opt->config)) return NP_ERR_UNSUPPORTED;
  for (int i = 0; i < count; i++) {
    NP_TRY(check_csr(&graphs[i], opt->kind == NP_BATCH_SSSP));
    if (sources[i] < 0 || sources[i] >= graphs[i].n) return NP_ERR_INVALID;
  }
  const int device = nestpar_ctx_device(ctx);
  NP_CK(cudaSetDevice(device));
  np_batch* b = new np_batch();
  b->kind = opt->kind;
  b->width = width;
  b->count = count;
  np_status st = engine_init(b->e, device);
  if (st != NP_OK) {
    np_batch_destroy(b);
    return st;
  }
  // classes in ascending size; instances keep their order within a class
  std::vector<int> cls_of((size_t)count);
  std::vector<int> keys;
  for (int i = 0; i < count; i++) {
    const int k = floor_log2(graphs[i].n) / width * width;
    cls_of[(size_t)i] = k;
    keys.push_back(k);
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  b->offsets.assign((size_t)count, 0);
  int64_t vbase = 0;
  for (int k : keys) {
    Class c;
    c.log2_lo = k;
    c.cfg = opt->config;
    const int ci = (int)b->classes.size();
    Group* cur = nullptr;
    for (int i = 0; i < count; i++) {
      if (cls_of[(size_t)i] != k) continue;
      const np_csr& gi = graphs[i];
      if (!cur || cur->m + gi.m > max_edges || (int64_t)cur->n + gi.n > (int64_t(1) << 30)) {
        b->groups.emplace_back();
        cur = &b->groups.back();
        cur->cls = ci;
        cur->vbase = vbase;
        c.groups.push_back((int)b->groups.size() - 1);
      }
      b->offsets[(size_t)i] = vbase;
      cur->members.push_back(i);
      cur->n += gi.n;
      cur->m += gi.m;
      vbase += gi.n;
      c.instances += 1;
      c.vertices += gi.n;
      c.edges += gi.m;
    }
    b->classes.push_back(c);
  }
  b->total = vbase;
  // The inputs may have been written by any stream: wait for the device, then
  // check every graph before anything indexes it.
  cudaStream_t s = b->e.cap_stream;
  {
    int* scratch = nullptr;
    st = from_cuda(cudaDeviceSynchronize());
    if (st == NP_OK) st = from_cuda(cudaMalloc(&scratch, sizeof(int)));
    if (st == NP_OK) st = check_csr_device(graphs, count, scratch, s);
    if (scratch) cudaFree(scratch);
    if (st != NP_OK) {
      np_batch_destroy(b);
      return st;
    }
  }
  // union copies
  for (Group& g : b->groups) {
    g.nsrc = (int)g.members.size();
    const size_t brp = align_up(sizeof(int) * ((size_t)g.n + 1)), bcol = align_up(sizeof(int) * (size_t)g.m);
    const size_t bw = opt->kind == NP_BATCH_SSSP ? align_up(sizeof(unsigned) * (size_t)g.m) : 0;
    const size_t bids = align_up(sizeof(int) * (size_t)g.nsrc);
    const size_t bd64 = opt->kind == NP_BATCH_SSSP ? align_up(sizeof(unsigned long long) * (size_t)g.n) : 0;
    st = from_cuda(cudaMalloc(&g.mem, brp + bcol + bw + bids + bd64 + kAlign));
    if (st == NP_OK) st = ws_init(g.ws);
    if (st == NP_OK) st = ws_ensure(g.ws, g.n);
    if (st != NP_OK) {
      np_batch_destroy(b);
      return st;
    }
    g.row_ptr = reinterpret_cast<int*>(g.mem);
    g.col = reinterpret_cast<int*>(g.mem + brp);
    g.w = bw ? reinterpret_cast<unsigned*>(g.mem + brp + bcol) : nullptr;
    g.ids = reinterpret_cast<int*>(g.mem + brp + bcol + bw);
    g.dtag = bd64 ? reinterpret_cast<unsigned long long*>(g.mem + brp + bcol + bw + bids) : nullptr;
    std::vector<int> ids;
    int voff = 0;
    long long eoff = 0;
    for (int i : g.members) {
      const np_csr& gi = graphs[i];
      union_append_kernel<<<blocks_for(std::max<int64_t>(gi.n, gi.m)), 256, 0, s>>>(
          g.row_ptr, g.col, g.w, gi.row_ptr, gi.col_idx, gi.weights, gi.n, gi.m, voff, eoff);
      ids.push_back(voff + sources[i]);
      voff += gi.n;
      eoff += gi.m;
    }
    const int mtot = (int)g.m;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(g.row_ptr + g.n, &mtot, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(g.ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      np_batch_destroy(b);
      return from_cuda(e);
    }
  }
  *out = b;
  return NP_OK;
}

np_status np_batch_destroy(np_batch* b) {
  if (!b) return NP_ERR_INVALID;
  cudaSetDevice(b->e.device);
  cudaDeviceSynchronize();
  drop_batch_graph(b);
  for (Group& g : b->groups) {
    ws_release(g.ws);
    if (g.mem) cudaFree(g.mem);
  }
  engine_release(b->e);
  delete b;
  return NP_OK;
}

np_status np_batch_layout(const np_batch* b, int64_t* offsets, int64_t* total) {
  if (!b) return NP_ERR_INVALID;
  if (offsets) std::memcpy(offsets, b->offsets.data(), sizeof(int64_t) * b->offsets.size());
  if (total) *total = b->total;
  return NP_OK;
}

np_status np_batch_classes(const np_batch* b, np_batch_class* out, int32_t max, int32_t* nclasses) {
  if (!b || max < 0 || (max > 0 && !out)) return NP_ERR_INVALID;
  if (nclasses) *nclasses = (int32_t)b->classes.size();
  for (int i = 0; i < max && i < (int)b->classes.size(); i++) {
    const Class& c = b->classes[(size_t)i];
    np_batch_class r;
    std::memset(&r, 0, sizeof(r));
    r.log2_lo = c.log2_lo;
    r.instances = c.instances;
    r.groups = (int32_t)c.groups.size();
    r.vertices = c.vertices;
    r.edges = c.edges;
    r.config = c.cfg;
    r.tuned_ms = c.tuned_ms;
    r.candidates = c.candidates;
    r.device_launch_ms = c.dl_ms;
    r.device_launch_granularity = c.dl_gran;
    r.device_launch_threshold = c.dl_threshold;
    out[i] = r;
  }
  return NP_OK;
}

np_status np_batch_set_config(np_batch* b, int32_t cls, const np_config* cfg) {
  if (!b || cls < 0 || cls >= (int)b->classes.size()) return NP_ERR_INVALID;
  NP_TRY(check_config(cfg));
  if (!batch_form_ok(*cfg)) return NP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(b->mu);
  b->classes[(size_t)cls].cfg = *cfg;
  b->classes[(size_t)cls].tuned_ms = 0.0;
  drop_batch_graph(b);
  return NP_OK;
}

np_status np_batch_tune(np_batch* b, void* out, int32_t reps, void* stream) {
  if (!b || !out || reps < 0) return NP_ERR_INVALID;
  if (reps == 0) reps = 3;
  std::lock_guard<std::mutex> lk(b->mu);
  NP_CK(cudaSetDevice(b->e.device));
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<np_config> cands;
  {
    np_config c = b->classes.empty() ? np_config{} : b->classes[0].cfg;
    np_config nodp = c;
    nodp.variant = NP_VARIANT_NODP;
    nodp.granularity = NP_GRAN_GRID_HOST;
    cands.push_back(nodp);
    for (int T : {8, 32, 128, 512})
      for (int cf : {2, 8})
        for (int cb : {32, 128}) {
          np_config x = c;
          x.variant = NP_VARIANT_CDP;
          x.granularity = NP_GRAN_GRID_HOST;
          x.threshold = T;
          x.cfactor = cf;
          x.child_block = cb;
          cands.push_back(x);
        }
  }
  for (size_t ci = 0; ci < b->classes.size(); ci++) {
    double best = 1e30;
    np_config pick = b->classes[ci].cfg;
    for (const np_config& c : cands) {
      double ms = 0.0;
      // one untimed run builds the class's graphs
      NP_TRY(time_class(b, (int)ci, c, out, 1, s, &ms));
      NP_TRY(time_class(b, (int)ci, c, out, reps, s, &ms));
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    // the pick with a swept frontier (every grid level's children only reduce,
    // a sweep over the group's vertex state forms the next frontier)
    int timed = (int)cands.size();
    np_config x = pick;
    x.sweep_parents = 1;
    if (pick.sweep_parents != 1 && sweeps(x)) {
      double ms = 0.0;
      NP_TRY(time_class(b, (int)ci, x, out, 1, s, &ms));
      NP_TRY(time_class(b, (int)ci, x, out, reps, s, &ms));
      timed++;
      if (ms < best) {
        best = ms;
        pick = x;
      }
    }
    b->classes[ci].cfg = pick;
    b->classes[ci].tuned_ms = best;
    b->classes[ci].candidates = timed;
    // the device-launch granularities, for the record (Section VII-C's third axis)
    double dl_best = 1e30;
    for (int gran : {NP_GRAN_BLOCK, NP_GRAN_MULTIBLOCK, NP_GRAN_GRID_DEVICE})
      for (int T : {32, 512}) {
        np_config x = b->classes[ci].cfg;
        x.variant = NP_VARIANT_CDP;
        x.granularity = gran;
        x.group_blocks = 8;
        x.threshold = T;
        x.cfactor = 4;
        x.child_block = 64;
        x.driver = NP_DRIVER_AUTO;
        double ms = 0.0;
        NP_TRY(time_class(b, (int)ci, x, out, 1, s, &ms, true));
        NP_TRY(time_class(b, (int)ci, x, out, reps, s, &ms, true));
        if (ms < dl_best) {
          dl_best = ms;
          b->classes[ci].dl_gran = gran;
          b->classes[ci].dl_threshold = T;
        }
      }
    b->classes[ci].dl_ms = dl_best;
  }
  drop_batch_graph(b);
  for (Group& g : b->groups) ws_drop_graphs(g.ws);
  return NP_OK;
}

np_status np_batch_run(np_batch* b, void* out, void* stream, np_stats* stats) {
  if (!b || !out) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(b->mu);
  NP_CK(cudaSetDevice(b->e.device));
  if (!b->exec || b->graph_out != out) NP_TRY(build_batch_graph(b, out));
  NP_CK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  if (!stats) return NP_OK;
  return batch_stats(b, (cudaStream_t)stream, stats);
}

}  // extern "C"
