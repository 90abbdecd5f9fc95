// Serving (np_server_*): continuous batching of BFS / SSSP queries over
// resident graphs.
//
// One pool per (graph, kind). A pool has S query slots; slot q owns the ids
// q * npad + v (npad = next power of two >= n) of its level or distance array,
// and the pool runs one level loop whose frontier holds the vertices of every
// resident query, so the children of all queries go through the same
// threshold / coarsening / aggregation path (Section V's aggregation across
// queries). Between levels the pool admits queued queries into free slots:
// the slot's arrays are reset and its source joins the current frontier at
// the current level L0 (BFS levels are stored absolute and reported minus
// L0). After `levels_per_step` levels a histogram of the frontier counts each
// slot's remaining vertices; a resident query with none left is finished and
// its result is copied to the caller's array. All of one pool's step is a
// single CUDA graph (admission table upload, slot reset, source push, the
// levels, histogram, result copy, count read-back) on the pool's own stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstring>
#include <deque>
#include <mutex>
#include <vector>

#include "np_engine.h"

using namespace nestpar;

namespace {

constexpr int kMaxSlots = 1024;

// Admission table, uploaded from pinned host memory at the start of a step.
struct __align__(16) Ctl {
  int nadm;
  int pad[3];
  // followed by int4 adm[S] {slot, src, out low, out high} and int busy[S]
};

size_t ctl_bytes(int S) { return sizeof(Ctl) + sizeof(int4) * (size_t)S + sizeof(int) * (size_t)S; }
int4* ctl_adm(Ctl* c) { return reinterpret_cast<int4*>(c + 1); }

__device__ __forceinline__ const int4* dctl_adm(const Ctl* c) { return reinterpret_cast<const int4*>(c + 1); }
__device__ __forceinline__ const int* dctl_busy(const Ctl* c, int S) {
  return reinterpret_cast<const int*>(dctl_adm(c) + S);
}

// Resets the arrays of the slots admitted this step (blockIdx.y = admission).
// SSSP pools keep the packed state (distance << 32 | append tag).
__global__ void slot_reset_kernel(const Ctl* ctl, int kind, int lg, int* level, unsigned long long* dtag) {
  if ((int)blockIdx.y >= ctl->nadm) return;
  const int slot = dctl_adm(ctl)[blockIdx.y].x;
  const long long base = (long long)slot << lg;
  const int npad = 1 << lg;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < npad; v += gridDim.x * blockDim.x) {
    if (kind == 0)
      level[base + v] = -1;
    else
      dtag[base + v] = 0xffffffff00000000ull;
  }
}

// Puts the admitted sources into the frontier of the current level.
__global__ void slot_admit_kernel(LevelState* st, const Ctl* ctl, int kind, int lg, int* level,
                                  unsigned long long* dtag, int* fr0, int* fr1, unsigned long long* slot_out,
                                  int* slot_L0) {
  __shared__ int c0, L;
  const int nadm = ctl->nadm;
  if (nadm <= 0) return;
  if (threadIdx.x == 0) {
    L = st->base;
    c0 = st->count[L % 3];
  }
  __syncthreads();
  int* fr = (L & 1) ? fr1 : fr0;
  for (int i = threadIdx.x; i < nadm; i += blockDim.x) {
    const int4 a = dctl_adm(ctl)[i];
    const int id = (a.x << lg) | a.y;
    if (kind == 0)
      level[id] = L;
    else
      dtag[id] = 0ull;
    fr[c0 + i] = id;
    slot_out[a.x] = ((unsigned long long)(unsigned)a.w << 32) | (unsigned)a.z;
    slot_L0[a.x] = L;
  }
  __syncthreads();
  if (threadIdx.x == 0) st->count[L % 3] = c0 + nadm;
}

// active[q] = frontier entries of slot q at the current level; active[S] = level.
__global__ void slot_histogram_kernel(const LevelState* st, const int* fr0, const int* fr1, int lg, int S,
                                      int* active) {
  __shared__ int h[kMaxSlots];
  for (int q = threadIdx.x; q < S; q += blockDim.x) h[q] = 0;
  __syncthreads();
  const int L = __ldcg(&st->base);
  const int cnt = __ldcg(&st->count[L % 3]);
  const int* ids = (L & 1) ? fr1 : fr0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    atomicAdd(&h[__ldcg(&ids[i]) >> lg], 1);
  __syncthreads();
  for (int q = threadIdx.x; q < S; q += blockDim.x)
    if (h[q]) atomicAdd(&active[q], h[q]);
  if (blockIdx.x == 0 && threadIdx.x == 0) active[S] = L;
}

// Copies every resident slot with no frontier entries left to its caller's array.
__global__ void slot_retire_kernel(const Ctl* ctl, int S, const int* active, int kind, int lg, int n,
                                   const int* level, const unsigned long long* dtag,
                                   const unsigned long long* slot_out, const int* slot_L0) {
  const int slot = blockIdx.y;
  if (!dctl_busy(ctl, S)[slot] || __ldcg(&active[slot]) != 0) return;
  const long long base = (long long)slot << lg;
  const int L0 = slot_L0[slot];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    if (kind == 0) {
      const int l = level[base + v];
      reinterpret_cast<int*>(slot_out[slot])[v] = l >= 0 ? l - L0 : -1;
    } else {
      reinterpret_cast<unsigned*>(slot_out[slot])[v] = (unsigned)(dtag[base + v] >> 32);
    }
  }
}

struct Query {
  int graph, kind, src;
  void* out;
  int slot = -1;
  int done = 0;
  int64_t submit_step = 0, admit_step = -1, finish_step = -1;
};

struct Pool {
  int graph = 0, kind = 0;
  int n = 0, lg = 0, S = 0;
  np_csr g{};
  np_config cfg{};
  uint64_t bytes_per_slot = 0;
  Workspace ws;
  unsigned char* mem = nullptr;   // state | ctl | slot_out | slot_L0 | active
  int* level = nullptr;
  unsigned long long* dtag = nullptr;
  Ctl* d_ctl = nullptr;
  unsigned long long* slot_out = nullptr;
  int* slot_L0 = nullptr;
  int* active = nullptr;
  Ctl* h_ctl = nullptr;           // pinned
  int* h_active = nullptr;        // pinned [S + 2]: per-slot counts, level, error word
  cudaStream_t stream = nullptr;
  cudaGraph_t graph_def = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int64_t> slot_query;
  std::deque<int64_t> queue;
  bool launched = false;
};

int ceil_log2(int n) {
  int k = 0;
  while ((1 << k) < n) k++;
  return k;
}

size_t pool_state_bytes(int kind, int lg, int S) {
  const size_t elems = (size_t)S << lg;
  return align_up((kind == 0 ? sizeof(int) : sizeof(unsigned long long)) * elems) + align_up(ctl_bytes(S)) + align_up(sizeof(unsigned long long) * S) +
         align_up(sizeof(int) * S) + align_up(sizeof(int) * (S + 1));
}

uint64_t pool_bytes(int kind, int lg, int S) {
  const int64_t elems = (int64_t)S << lg;
  return (uint64_t)pool_state_bytes(kind, lg, S) + layout_for(elems < 4096 ? 4096 : elems).total;
}

}  // namespace

struct np_server {
  Engine e;
  std::vector<Pool> pools;
  std::vector<Query> queries;
  int levels_per_step = 2;
  int64_t step = 0;
  std::vector<int64_t> finished;    // tickets finished since the last np_server_finished
  std::mutex mu;
};

namespace {

np_status build_pool_graph(np_server* sv, Pool& p) {
  Engine& e = sv->e;
  const BodyKernels& K = p.kind == 0 ? bfs_kernels() : sssp64_kernels();
  Plan plan = make_plan(K, p.cfg);
  Args a;
  base_args(p.ws, p.cfg, a);
  a.row_ptr = p.g.row_ptr;
  a.b.col = p.g.col_idx;
  a.b.w = p.g.weights;
  a.b.level = p.level;
  a.b.dtag = p.dtag;
  a.b.stamp = wsp<int>(p.ws, p.ws.lay.off_stamp);
  a.b.vmask = (1 << p.lg) - 1;
  const int64_t elems = (int64_t)p.S << p.lg;
  if (plan.sweep) {
    // the sweep covers every slot's state; with slots of at least one sweep
    // chunk it skips the slots this step's admission table marks idle
    a.n_vertices = (int)elems;
    if ((1 << p.lg) >= kSweepVertices) {
      a.sweep_lg = p.lg;
      a.sweep_busy = reinterpret_cast<const int*>(ctl_adm(p.d_ctl) + p.S);
    }
  }
  Grids gr = grids_for(e, plan, p.cfg, elems);
  cudaStream_t cs = e.cap_stream;
  NP_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  np_status st = NP_OK;
  cudaError_t ce = cudaMemcpyAsync(p.d_ctl, p.h_ctl, ctl_bytes(p.S), cudaMemcpyHostToDevice, cs);
  if (ce == cudaSuccess) {
    const int bx = blocks_for(1ll << p.lg, 256, 64);
    slot_reset_kernel<<<dim3(bx, p.S), 256, 0, cs>>>(p.d_ctl, p.kind, p.lg, p.level, p.dtag);
    slot_admit_kernel<<<1, 256, 0, cs>>>(p.ws.st, p.d_ctl, p.kind, p.lg, p.level, p.dtag, a.fr0, a.fr1, p.slot_out,
                                         p.slot_L0);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) {
    for (int k = 0; k < sv->levels_per_step && st == NP_OK; k++) st = enqueue_pass(plan, a, gr, true, k, cs);
    if (st == NP_OK) st = enqueue_advance(p.ws.st, sv->levels_per_step, cs, true);
  }
  if (ce == cudaSuccess && st == NP_OK) ce = cudaMemsetAsync(p.active, 0, sizeof(int) * (size_t)(p.S + 1), cs);
  if (ce == cudaSuccess && st == NP_OK) {
    slot_histogram_kernel<<<std::max(1, std::min(e.sms * 2, blocks_for(elems))), 256, 0, cs>>>(
        p.ws.st, a.fr0, a.fr1, p.lg, p.S, p.active);
    const int bx = blocks_for(p.n, 256, 64);
    slot_retire_kernel<<<dim3(bx, p.S), 256, 0, cs>>>(p.d_ctl, p.S, p.active, p.kind, p.lg, p.n, p.level, p.dtag,
                                                       p.slot_out, p.slot_L0);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess && st == NP_OK)
    ce = cudaMemcpyAsync(p.h_active, p.active, sizeof(int) * (size_t)(p.S + 1), cudaMemcpyDeviceToHost, cs);
  if (ce == cudaSuccess && st == NP_OK)   // the pool's device error word
    ce = cudaMemcpyAsync(p.h_active + p.S + 1, &p.ws.st->error, sizeof(unsigned), cudaMemcpyDeviceToHost, cs);
  cudaGraph_t graph = nullptr;
  cudaError_t ee = cudaStreamEndCapture(cs, &graph);
  if (st != NP_OK || ce != cudaSuccess || ee != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (st != NP_OK) return st;
    return from_cuda(ce != cudaSuccess ? ce : ee);
  }
  cudaGraphExec_t exec = nullptr;
  st = instantiate(graph, &exec);
  if (st != NP_OK) {
    cudaGraphDestroy(graph);
    return st;
  }
  p.graph_def = graph;
  p.exec = exec;
  return NP_OK;
}

void release_pool(Pool& p) {
  if (p.exec) cudaGraphExecDestroy(p.exec);
  if (p.graph_def) cudaGraphDestroy(p.graph_def);
  ws_release(p.ws);
  if (p.mem) cudaFree(p.mem);
  if (p.h_ctl) cudaFreeHost(p.h_ctl);
  if (p.h_active) cudaFreeHost(p.h_active);
  if (p.stream) cudaStreamDestroy(p.stream);
  p = Pool{};
}

np_status init_pool(np_server* sv, Pool& p) {
  NP_TRY(ws_init(p.ws));
  const int64_t elems = (int64_t)p.S << p.lg;
  NP_TRY(ws_ensure(p.ws, elems));
  const size_t b_state = align_up((p.kind == 0 ? sizeof(int) : sizeof(unsigned long long)) * (size_t)elems);
  const size_t b_ctl = align_up(ctl_bytes(p.S));
  const size_t b_out = align_up(sizeof(unsigned long long) * p.S);
  const size_t b_l0 = align_up(sizeof(int) * p.S);
  const size_t b_act = align_up(sizeof(int) * (p.S + 1));
  NP_CK(cudaMalloc(&p.mem, b_state + b_ctl + b_out + b_l0 + b_act));
  NP_CK(cudaMemset(p.mem, 0, b_state + b_ctl + b_out + b_l0 + b_act));
  p.level = p.kind == 0 ? reinterpret_cast<int*>(p.mem) : nullptr;
  p.dtag = p.kind == 1 ? reinterpret_cast<unsigned long long*>(p.mem) : nullptr;
  p.d_ctl = reinterpret_cast<Ctl*>(p.mem + b_state);
  p.slot_out = reinterpret_cast<unsigned long long*>(p.mem + b_state + b_ctl);
  p.slot_L0 = reinterpret_cast<int*>(p.mem + b_state + b_ctl + b_out);
  p.active = reinterpret_cast<int*>(p.mem + b_state + b_ctl + b_out + b_l0);
  NP_CK(cudaMallocHost(&p.h_ctl, ctl_bytes(p.S)));
  std::memset(p.h_ctl, 0, ctl_bytes(p.S));
  NP_CK(cudaMallocHost(&p.h_active, sizeof(int) * (size_t)(p.S + 2)));
  std::memset(p.h_active, 0, sizeof(int) * (size_t)(p.S + 2));
  NP_CK(cudaStreamCreateWithFlags(&p.stream, cudaStreamNonBlocking));
  p.slot_query.assign((size_t)p.S, -1);
  // empty pool: level 0, no parents, max_levels unbounded
  seed_sources_kernel<<<1, 32, 0, p.stream>>>(p.ws.st, p.kind, nullptr, 0, p.level, nullptr,
                                              wsp<int>(p.ws, p.ws.lay.off_fr0), INT_MAX - 64);
  NP_CK(cudaGetLastError());
  NP_CK(cudaStreamSynchronize(p.stream));
  return build_pool_graph(sv, p);
}

}  // namespace

int nestpar_ctx_device(const np_ctx* c);

extern "C" {

np_status np_server_create(np_ctx* ctx, const np_csr* graphs, int32_t ngraphs, const np_server_options* opt,
                           np_server** out) {
  if (!ctx || !graphs || ngraphs < 1 || !opt || !out) return NP_ERR_INVALID;
  *out = nullptr;
  const int max_slots = opt->max_slots == 0 ? 64 : opt->max_slots;
  const int lps = opt->levels_per_step == 0 ? 2 : opt->levels_per_step;
  if (max_slots < 1 || max_slots > kMaxSlots || lps < 1 || lps > 16) return NP_ERR_INVALID;
  const np_config* cfgs[2] = {&opt->bfs_config, &opt->sssp_config};
  for (int k = 0; k < 2; k++) {
    NP_TRY(check_config(cfgs[k]));
    const np_config& c = *cfgs[k];
    if (!(c.variant == NP_VARIANT_NODP || c.granularity == NP_GRAN_GRID_HOST)) return NP_ERR_UNSUPPORTED;
  }
  for (int i = 0; i < ngraphs; i++) {
    NP_TRY(check_csr(&graphs[i], false));
    if (graphs[i].n > (1 << 30)) return NP_ERR_INVALID;
  }
  const int device = nestpar_ctx_device(ctx);
  NP_CK(cudaSetDevice(device));
  uint64_t budget = opt->memory_budget;
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    NP_CK(cudaMemGetInfo(&fr, &tot));
    budget = fr / 4;
  }
  np_server* sv = new np_server();
  sv->levels_per_step = lps;
  np_status st = engine_init(sv->e, device);
  // the graphs may have been written by any stream: wait, then check each once
  if (st == NP_OK) {
    int* scratch = nullptr;
    st = from_cuda(cudaDeviceSynchronize());
    if (st == NP_OK) st = from_cuda(cudaMalloc(&scratch, sizeof(int)));
    if (st == NP_OK) st = check_csr_device(graphs, ngraphs, scratch, sv->e.cap_stream);
    if (scratch) cudaFree(scratch);
  }
  const int npools = 2 * ngraphs;
  const uint64_t share = budget / (uint64_t)npools;
  for (int gi = 0; gi < ngraphs && st == NP_OK; gi++) {
    for (int kind = 0; kind < 2 && st == NP_OK; kind++) {
      Pool p;
      p.graph = gi;
      p.kind = kind;
      p.g = graphs[gi];
      p.n = graphs[gi].n;
      p.lg = ceil_log2(p.n);
      p.cfg = *cfgs[kind];
      if (kind == 1 && !p.g.weights && p.g.m > 0) {
        p.S = 0;   // no weights: this graph serves BFS only
        p.bytes_per_slot = pool_bytes(kind, p.lg, 1);
        sv->pools.push_back(p);
        continue;
      }
      int S = 0;
      const int cap = std::min<int64_t>(max_slots, (int64_t(1) << 31) / (int64_t(1) << p.lg) - 1);
      for (int s = 1; s <= cap; s++) {
        if (pool_bytes(kind, p.lg, s) > share) break;
        S = s;
      }
      p.bytes_per_slot = pool_bytes(kind, p.lg, 1);
      if (S < 1) {
        st = NP_ERR_NOMEM;
        break;
      }
      p.S = S;
      p.cfg = serial_for(p.cfg, S, p.g.m);
      // (a pool's swept frontier sweeps its busy slots only: see build_pool_graph)
      if (((int64_t)S << p.lg) > (int64_t)INT_MAX) p.cfg.sweep_parents = 0;
      sv->pools.push_back(p);
      st = init_pool(sv, sv->pools.back());
    }
  }
  if (st != NP_OK) {
    np_server_destroy(sv);
    return st;
  }
  *out = sv;
  return NP_OK;
}

np_status np_server_destroy(np_server* sv) {
  if (!sv) return NP_ERR_INVALID;
  cudaSetDevice(sv->e.device);
  cudaDeviceSynchronize();
  for (Pool& p : sv->pools) release_pool(p);
  engine_release(sv->e);
  delete sv;
  return NP_OK;
}

np_status np_server_pool_info(const np_server* sv, int32_t graph, int32_t kind, int32_t* slots,
                              uint64_t* bytes_per_slot) {
  if (!sv || kind < 0 || kind > 1 || graph < 0 || 2 * graph + kind >= (int)sv->pools.size()) return NP_ERR_INVALID;
  const Pool& p = sv->pools[(size_t)(2 * graph + kind)];
  if (slots) *slots = p.S;
  if (bytes_per_slot) *bytes_per_slot = p.bytes_per_slot;
  return NP_OK;
}

np_status np_server_submit(np_server* sv, int32_t graph, int32_t kind, int32_t src, void* out, int64_t* ticket) {
  if (!sv || !out || kind < 0 || kind > 1 || graph < 0 || 2 * graph + kind >= (int)sv->pools.size())
    return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  Pool& p = sv->pools[(size_t)(2 * graph + kind)];
  if (p.S < 1) return NP_ERR_UNSUPPORTED;
  if (src < 0 || src >= p.n) return NP_ERR_INVALID;
  Query q;
  q.graph = graph;
  q.kind = kind;
  q.src = src;
  q.out = out;
  q.submit_step = sv->step;
  const int64_t t = (int64_t)sv->queries.size();
  sv->queries.push_back(q);
  p.queue.push_back(t);
  if (ticket) *ticket = t;
  return NP_OK;
}

np_status np_server_step(np_server* sv, int32_t* in_flight) {
  if (!sv) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  NP_CK(cudaSetDevice(sv->e.device));
  for (Pool& p : sv->pools) {
    p.launched = false;
    if (p.S < 1) continue;
    int nadm = 0;
    int4* adm = ctl_adm(p.h_ctl);
    int* busy = reinterpret_cast<int*>(adm + p.S);
    for (int s = 0; s < p.S && !p.queue.empty(); s++) {
      if (p.slot_query[(size_t)s] >= 0) continue;
      const int64_t t = p.queue.front();
      p.queue.pop_front();
      Query& q = sv->queries[(size_t)t];
      const unsigned long long ptr = (unsigned long long)(uintptr_t)q.out;
      adm[nadm++] = make_int4(s, q.src, (int)(unsigned)(ptr & 0xffffffffull), (int)(unsigned)(ptr >> 32));
      busy[s] = 1;
      p.slot_query[(size_t)s] = t;
      q.slot = s;
      q.admit_step = sv->step;
    }
    p.h_ctl->nadm = nadm;
    bool any = false;
    for (int s = 0; s < p.S; s++) any = any || busy[s];
    if (!any) continue;
    NP_CK(cudaGraphLaunch(p.exec, p.stream));
    p.launched = true;
  }
  np_status worst = NP_OK;
  for (Pool& p : sv->pools) {
    if (!p.launched) continue;
    NP_CK(cudaStreamSynchronize(p.stream));
    int* busy = reinterpret_cast<int*>(ctl_adm(p.h_ctl) + p.S);
    for (int s = 0; s < p.S; s++) {
      if (!busy[s] || p.h_active[s] != 0) continue;
      Query& q = sv->queries[(size_t)p.slot_query[(size_t)s]];
      q.done = 1;
      q.finish_step = sv->step;
      sv->finished.push_back(p.slot_query[(size_t)s]);
      busy[s] = 0;
      p.slot_query[(size_t)s] = -1;
    }
    const unsigned err = (unsigned)p.h_active[p.S + 1];
    if (err) {
      if (worst == NP_OK) worst = status_from_bits(err);
      NP_CK(cudaMemsetAsync(&p.ws.st->error, 0, sizeof(unsigned), p.stream));
      NP_CK(cudaStreamSynchronize(p.stream));
    }
  }
  sv->step += 1;
  if (in_flight) {
    int64_t k = 0;
    for (const Pool& p : sv->pools) {
      k += (int64_t)p.queue.size();
      for (int s = 0; s < p.S; s++) k += p.slot_query[(size_t)s] >= 0;
    }
    *in_flight = (int32_t)k;
  }
  return worst;
}

np_status np_server_finished(np_server* sv, int64_t* tickets, int32_t max, int32_t* count) {
  if (!sv || !count || max < 0 || (max > 0 && !tickets)) return NP_ERR_INVALID;
  std::lock_guard<std::mutex> lk(sv->mu);
  const int k = (int)std::min<size_t>((size_t)max, sv->finished.size());
  if (k) std::memcpy(tickets, sv->finished.data(), sizeof(int64_t) * (size_t)k);
  sv->finished.erase(sv->finished.begin(), sv->finished.begin() + k);
  *count = k;
  return NP_OK;
}

np_status np_server_poll(const np_server* sv, int64_t ticket, np_query_info* info) {
  if (!sv || !info || ticket < 0 || ticket >= (int64_t)sv->queries.size()) return NP_ERR_INVALID;
  const Query& q = sv->queries[(size_t)ticket];
  std::memset(info, 0, sizeof(*info));
  info->done = q.done;
  info->graph = q.graph;
  info->kind = q.kind;
  info->slot = q.done ? -1 : q.slot;
  info->submit_step = q.submit_step;
  info->admit_step = q.admit_step;
  info->finish_step = q.finish_step;
  return NP_OK;
}

}  // extern "C"
