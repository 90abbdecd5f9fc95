// Host engine: workspaces, plans, grids and the level-loop drivers.
//
// Level loop. A level is one parent grid (persistent CTAs over the frontier,
// which lives in device memory) plus, for grid-host aggregation, one
// stream-ordered persistent child grid whose size is read from device memory.
// Forms without a device launch site (NODP, grid-host aggregation) run the
// whole loop inside a conditional-while CUDA graph: `unroll` levels per body
// iteration, a one-thread kernel setting the condition, no host round trip.
// The device-launch forms are never captured into a graph: measured on GB300
// (CUDA 13.0, driver 580), a kernel node of a CUDA graph counts as complete
// before the grids it launched from the device (fire-and-forget or tail
// launch) have finished, so the next node could read a level or a result that
// its children are still writing. A kernel launched on a stream does wait for
// its children. So those forms enqueue `unroll` levels directly on the stream
// and read the frontier size back after each chunk. NP_DRIVER_HOST is the
// paper's own form: one host launch per level and a read-back after each.
#include "np_engine.h"

#include <climits>
#include <cstring>

namespace nestpar {

np_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return NP_OK;
  if (e == cudaErrorMemoryAllocation) return NP_ERR_NOMEM;
  return NP_ERR_CUDA;
}

np_status status_from_bits(unsigned bits) {
  if (bits & kErrTimeout) return NP_ERR_TIMEOUT;
  if (bits & kErrCapacity) return NP_ERR_CAPACITY;
  if (bits & kErrLaunch) return NP_ERR_LAUNCH;
  return NP_OK;
}

// ------------------------------------------------------------- device side

__device__ __forceinline__ void reset_slots(LevelState* st) {
  for (int k = 0; k < 4; k++) {
    st->ticket[k] = 0;
    st->agg_records[k] = 0;
    st->agg_blocks[k] = 0;
    st->agg_acc[k] = 0ull;
    st->child_ticket[k] = 0;
    st->pack_acc[k] = 0ull;
    st->pack_records[k] = 0;
    st->pack_items[k] = 0;
    st->pack_ticket[k] = 0;
  }
  for (int k = 0; k < S_N; k++) st->s[k] = 0ull;
  st->body_iters = 0;
  st->bar_count = 0u;
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

__global__ void fill_unreached_kernel(int kind, long long total, int* level, unsigned* dist, int* stamp) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += stride) {
    if (kind == 0) {
      level[v] = -1;
    } else {
      dist[v] = 0xffffffffu;
      stamp[v] = -1;
    }
  }
}

__global__ void seed_sources_kernel(LevelState* st, int kind, const int* ids, int nsrc, int* level, unsigned* dist,
                                    int* fr0, int max_levels) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x) {
    const int id = ids[i];
    if (kind == 0)
      level[id] = 0;
    else
      dist[id] = 0u;
    fr0[i] = id;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->base = 0;
    st->count[0] = nsrc;
    st->count[1] = 0;
    st->count[2] = 0;
    st->max_levels = max_levels;
    reset_slots(st);
  }
}

__global__ void csr_check_kernel(const int* row_ptr, const int* col, int n, long long m, int* bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long top = n > m ? (long long)n : m;
  bool ok = true;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < top; i += stride) {
    if (i < n) ok = ok && row_ptr[i] <= row_ptr[i + 1];
    if (i < m) {
      const int v = col[i];
      ok = ok && v >= 0 && v < n;
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ok = ok && row_ptr[0] == 0 && (long long)row_ptr[n] == m;
  if (!ok) atomicOr(bad, 1);
}

__global__ void sum_u64_kernel(const unsigned long long* part, int n, unsigned long long* out, int accumulate) {
  __shared__ unsigned long long s[32];
  unsigned long long v = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += part[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; w++) t += s[w];
    *out = accumulate ? *out + t : t;
  }
}

__global__ void init_dtag_kernel(long long total, unsigned long long* dtag) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += stride)
    dtag[v] = 0xffffffff00000000ull;
}

__global__ void seed_dtag_kernel(LevelState* st, const int* ids, int nsrc, unsigned long long* dtag, int* fr0,
                                 int max_levels) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsrc; i += gridDim.x * blockDim.x) {
    dtag[ids[i]] = 0ull;
    fr0[i] = ids[i];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->base = 0;
    st->count[0] = nsrc;
    st->count[1] = 0;
    st->count[2] = 0;
    st->max_levels = max_levels;
    reset_slots(st);
  }
}

__global__ void init_dtag_solve_kernel(LevelState* st, int n, int src, unsigned long long* dtag, int* fr0,
                                       int max_levels) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    dtag[v] = v == src ? 0ull : 0xffffffff00000000ull;
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

__global__ void dtag_to_dist_kernel(long long total, const unsigned long long* dtag, unsigned* dist) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < total; v += stride)
    dist[v] = (unsigned)(dtag[v] >> 32);
}

// Checks of the bounded waits (np_selftest_wait): each waits on a flag that
// nothing sets and must give up with the timeout bit set.
// A decoupled look-back for tile 1 of a scan whose tile 0 never publishes
// (an epoch no solve reaches).
__global__ void selftest_lookback_kernel(Args a) {
  const unsigned long long epoch = ((__ldcg(&a.st->solve_id) + (1ull << 28)) << 31) | 7ull;
  lookback(a.lb_flag, a.lb_agg, a.lb_incl, 1, 0, epoch, V4{1u, 0u, 0u, 0u}, a.st);
}

// A grid barrier that one CTA (blockIdx.x == 1) never reaches.
__global__ void selftest_barrier_kernel(LevelState* st, unsigned long long limit_ns) {
  __shared__ int s_ok;
  if (blockIdx.x == 1) return;
  grid_barrier(st, &s_ok, limit_ns);
}

// Between graph bodies or chunks: the next body position 0 is level base + K.
__global__ void advance_base_kernel(LevelState* st, int K) {
  NP_PDL_ENTRY();
  st->base += K;
}

// End of a conditional-while body of K levels: move base on and continue while
// the next level has parents. The iteration cap turns a level loop that failed
// to terminate into an error instead of an endless loop.
__global__ void set_cond_kernel(LevelState* st, cudaGraphConditionalHandle h, int K) {
  NP_PDL_ENTRY();
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

// --------------------------------------------------------------- host side

Layout layout_for(int64_t parents) {
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
  L.off_prec = take(sizeof(int4) * L.P2);
  L.off_pfirst = take(sizeof(int) * (L.P2 + 2));
  L.total = o;
  return L;
}

np_status engine_init(Engine& e, int device) {
  e.device = device;
  cudaDeviceProp prop;
  NP_CK(cudaGetDeviceProperties(&prop, device));
  e.sms = prop.multiProcessorCount;
  NP_CK(cudaMallocHost(&e.pin, 64));
  NP_CK(cudaMallocHost(&e.pin_state, sizeof(LevelState)));
  NP_CK(cudaStreamCreateWithFlags(&e.cap_stream, cudaStreamNonBlocking));
  for (int k = 0; k < 4; k++) NP_CK(cudaEventCreate(&e.ev[k]));
  return NP_OK;
}

void engine_release(Engine& e) {
  if (e.pin) cudaFreeHost(e.pin);
  if (e.pin_state) cudaFreeHost(e.pin_state);
  if (e.cap_stream) cudaStreamDestroy(e.cap_stream);
  for (int k = 0; k < 4; k++)
    if (e.ev[k]) cudaEventDestroy(e.ev[k]);
  e = Engine{};
}

np_status ws_init(Workspace& w) {
  NP_CK(cudaMalloc(&w.st, sizeof(LevelState)));
  NP_CK(cudaMemset(w.st, 0, sizeof(LevelState)));
  return NP_OK;
}

void ws_drop_graphs(Workspace& w) {
  for (auto& kv : w.graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  w.graphs.clear();
}

void ws_release(Workspace& w) {
  ws_drop_graphs(w);
  if (w.ws) cudaFree(w.ws);
  if (w.st) cudaFree(w.st);
  w.ws = nullptr;
  w.st = nullptr;
  w.cap_parents = 0;
}

np_status ws_ensure(Workspace& w, int64_t parents) {
  if (parents <= w.cap_parents && w.ws) return NP_OK;
  int64_t want = parents < 4096 ? 4096 : parents;
  Layout L = layout_for(want);
  ws_drop_graphs(w);
  if (w.ws) {
    NP_CK(cudaDeviceSynchronize());
    cudaFree(w.ws);
    w.ws = nullptr;
    w.cap_parents = 0;
  }
  unsigned char* p = nullptr;
  NP_CK(cudaMalloc(&p, L.total));
  NP_CK(cudaMemset(p, 0, L.total));
  w.ws = p;
  w.lay = L;
  w.cap_parents = want;
  return NP_OK;
}

int occupancy(Engine& e, const void* fn, int block) {
  auto key = std::make_pair(fn, block);
  auto it = e.occ.find(key);
  if (it != e.occ.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, 0) != cudaSuccess || n < 1) n = 1;
  e.occ[key] = n;
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
  if (cfg->driver < NP_DRIVER_AUTO || cfg->driver > NP_DRIVER_PERSISTENT) return NP_ERR_INVALID;
  if (cfg->unroll < 1 || cfg->unroll > 16) return NP_ERR_INVALID;
  if (cfg->parent_grid < 0) return NP_ERR_INVALID;
  if (cfg->serial != NP_SERIAL_SPREAD && cfg->serial != NP_SERIAL_PACKED && cfg->serial != NP_SERIAL_BLOCK)
    return NP_ERR_INVALID;
  if (cfg->small_parents < 0 || cfg->small_parents > NP_SMALL_PARENTS_MAX) return NP_ERR_INVALID;
  if (cfg->sweep_parents < 0) return NP_ERR_INVALID;
  for (int k = 0; k < 1; k++)
    if (cfg->reserved[k] != 0) return NP_ERR_INVALID;
  return NP_OK;
}

np_config serial_for(const np_config& cfg, int64_t copies, int64_t m) {
  np_config c = cfg;
  if (copies * m >= (int64_t)INT_MAX) c.serial = NP_SERIAL_SPREAD;
  return c;
}

bool sweeps(const np_config& cfg) {
  return cfg.sweep_parents > 0 && cfg.variant == NP_VARIANT_CDP && cfg.granularity == NP_GRAN_GRID_HOST &&
         cfg.serial == NP_SERIAL_SPREAD && cfg.driver != NP_DRIVER_PERSISTENT;
}

int serial_form(const np_config& cfg) {
  if (cfg.variant != NP_VARIANT_CDP || cfg.granularity != NP_GRAN_GRID_HOST) return NP_SERIAL_SPREAD;
  // packed children number their items per chunk: a parent meets at most one chunk start
  if (cfg.serial == NP_SERIAL_PACKED && cfg.threshold > kPackMaxT) return NP_SERIAL_BLOCK;
  return cfg.serial;
}

Plan make_plan(const BodyKernels& K, const np_config& cfg) {
  Plan p;
  const int cfi = cf_index(cfg.cfactor);
  if (cfg.variant == NP_VARIANT_NODP) {
    // warp tiles; with granularity NONE the CTA-tiled kernel of the
    // device-launch forms without its launch code (dead-launch-code baseline)
    p.parent = cfg.granularity == NP_GRAN_NONE ? K.parent_nodp_cta : K.parent_nodp;
    p.loop = cfg.granularity == NP_GRAN_NONE ? nullptr : K.level_loop_nodp;
    p.mode = M_NODP;
    p.gran = G_NODP;
  } else if (cfg.granularity == NP_GRAN_GRID_HOST) {
    // (the persistent level loop keeps the warp-tiled parent phase)
    const int form = serial_form(cfg);
    p.parent = form == NP_SERIAL_SPREAD ? K.parent_grid_host : K.parent_cta;
    p.child = form == NP_SERIAL_PACKED ? K.child_agg_pack[cfi] : K.child_agg[cfi];
    p.loop = K.level_loop_agg[cfi];
    p.small = cfg.small_parents > 0 ? K.level_small : nullptr;
    p.child_idle = cfg.threshold == INT32_MAX && form != NP_SERIAL_PACKED;
    if (sweeps(cfg) && K.parent_sweep) {
      p.parent = K.parent_sweep;
      p.child = K.child_sweep[cfi];
      p.sweep = K.frontier_sweep;
    }
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

void base_args(const Workspace& w, const np_config& cfg, Args& a) {
  std::memset(&a, 0, sizeof(a));
  a.st = w.st;
  a.fr0 = wsp<int>(w, w.lay.off_fr0);
  a.fr1 = wsp<int>(w, w.lay.off_fr1);
  a.rec = wsp<int4>(w, w.lay.off_rec);
  a.boff = wsp<int>(w, w.lay.off_boff);
  a.lb_flag = wsp<unsigned long long>(w, w.lay.off_lb_flag);
  a.lb_agg = wsp<uint4>(w, w.lay.off_lb_agg);
  a.lb_incl = wsp<uint4>(w, w.lay.off_lb_incl);
  a.ob_flag = wsp<unsigned long long>(w, w.lay.off_ob_flag);
  a.ob_agg = wsp<uint4>(w, w.lay.off_ob_agg);
  a.ob_incl = wsp<uint4>(w, w.lay.off_ob_incl);
  a.grp_ctr = wsp<int>(w, w.lay.off_grp_ctr);
  a.grp_acc = wsp<unsigned long long>(w, w.lay.off_grp_acc);
  a.grp_total = wsp<uint2>(w, w.lay.off_grp_total);
  a.threshold = cfg.threshold;
  a.cfactor = cfg.cfactor;
  a.child_block = cfg.child_block;
  a.group_blocks = cfg.granularity == NP_GRAN_MULTIBLOCK ? cfg.group_blocks : 0;
  a.agg_threshold = (cfg.granularity == NP_GRAN_WARP || cfg.granularity == NP_GRAN_BLOCK) ? cfg.agg_threshold : 0;
  a.scan = cfg.scan;
  a.pack = serial_form(cfg) == NP_SERIAL_PACKED ? 1 : 0;
  a.small_parents = cfg.small_parents;
  a.sweep_parents = sweeps(cfg) ? cfg.sweep_parents : 0;
  a.prec = wsp<int4>(w, w.lay.off_prec);
  a.pfirst = wsp<int>(w, w.lay.off_pfirst);
  a.b.st = w.st;
  a.b.vmask = 0x7fffffff;
  a.count_fixed = -1;
}

Grids grids_for(Engine& e, const Plan& p, const np_config& cfg, int64_t max_parents) {
  Grids g{};
  g.pblock = cfg.parent_block;
  g.cblock = cfg.child_block;
  int64_t tiles = (max_parents + g.pblock - 1) / g.pblock;
  if (tiles < 1) tiles = 1;
  int64_t pg = cfg.parent_grid > 0 ? cfg.parent_grid : (int64_t)occupancy(e, p.parent, g.pblock) * e.sms;
  if (pg > tiles) pg = tiles;
  g.pgrid = (int)pg;
  // the persistent child grid hosts cb-thread child blocks in CTAs of at least 256 threads
  g.cthreads = g.cblock < 256 ? 256 : g.cblock;
  g.cgrid = p.child ? occupancy(e, p.child, g.cthreads) * e.sms : 0;
  return g;
}

int resolve_driver(const Plan& p, const np_config& cfg) {
  if (cfg.driver != NP_DRIVER_AUTO) return cfg.driver;
  return p.mode == M_DEVICE_LAUNCH ? NP_DRIVER_CHUNK : NP_DRIVER_WHILE;
}

namespace {

// A launch that may be scheduled while its predecessor on the stream is still
// running (programmatic dependent launch); the kernel waits for it itself.
cudaError_t launch_pdl(const void* fn, dim3 grid, dim3 block, void** args, cudaStream_t s, bool pdl) {
  if (!pdl) return cudaLaunchKernel(fn, grid, block, args, 0, s);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

constexpr bool kPdl = NP_PDL != 0;

AggSeg make_seg(const Args& a, const Grids& g, bool level_mode) {
  AggSeg seg{};
  seg.rec = a.rec;
  seg.boff = a.boff;
  seg.mode = a.scan == 0 ? 1 : 2;
  seg.k = a.k;
  seg.level_mode = level_mode ? 1 : 0;
  seg.fr0 = a.fr0;
  seg.fr1 = a.fr1;
  seg.cb = g.cblock;
  seg.pack = a.pack;
  seg.sweep_parents = a.sweep_parents;
  seg.prec = a.prec;
  seg.pfirst = a.pfirst;
  return seg;
}

BodyArgs child_body(const Args& a, bool level_mode) {
  BodyArgs b = a.b;
  if (!level_mode) {
    b.L = a.L_fixed;
    b.next = a.next_ovr;
    b.next_count = a.next_count_ovr;
  }
  return b;
}

}  // namespace

// CTAs of the frontier sweep: kSweepVertices state elements each, at most as
// many as the resident child grid (the sweep loops over the rest).
int sweep_grid(const Args& a, const Grids& g) {
  const int64_t need = ((int64_t)a.n_vertices + kSweepVertices - 1) / kSweepVertices;
  const int cap = g.cgrid > 0 ? g.cgrid : 1;
  return need < 1 ? 1 : (need > cap ? cap : (int)need);
}

// Enqueues the grids of one level (level mode, at body position k) or of one
// fixed pass.
np_status enqueue_pass(const Plan& p, Args a, const Grids& g, bool level_mode, int k, cudaStream_t s) {
  a.k = level_mode ? k : 0;
  // device-launch forms must complete with their children: no early launch
  const bool pdl = kPdl && p.mode != M_DEVICE_LAUNCH;
  void* pargs[] = {&a};
  NP_CK(launch_pdl(p.parent, dim3(g.pgrid), dim3(g.pblock), pargs, s, pdl));
  if (p.mode == M_GRID_HOST && !p.child_idle) {
    AggSeg seg = make_seg(a, g, level_mode);
    BodyArgs b = child_body(a, level_mode);
    void* cargs[] = {&b, &seg};
    NP_CK(launch_pdl(p.child, dim3(g.cgrid), dim3(g.cthreads), cargs, s, pdl));
  }
  if (p.sweep && level_mode) NP_CK(launch_pdl(p.sweep, dim3(sweep_grid(a, g)), dim3(256), pargs, s, pdl));
  return NP_OK;
}

np_status enqueue_advance(LevelState* st, int K, cudaStream_t s, bool after_launch_free) {
  // after a device-launch form it must wait for the level's children: no early launch
  void* args[] = {&st, &K};
  NP_CK(launch_pdl((const void*)advance_base_kernel, dim3(1), dim3(1), args, s, kPdl && after_launch_free));
  return NP_OK;
}

// Profile mode: the grids of one level (or pass) launched one by one between
// CUDA events, then waited for; times go to the engine's breakdown.
np_status profiled_pass(Engine& e, const Workspace& w, const Plan& p, Args a, const Grids& g, bool level_mode,
                        cudaStream_t s) {
  a.k = 0;
  void* pargs[] = {&a};
  NP_CK(cudaEventRecord(e.ev[0], s));
  NP_CK(cudaLaunchKernel(p.parent, dim3(g.pgrid), dim3(g.pblock), pargs, 0, s));
  NP_CK(cudaEventRecord(e.ev[1], s));
  bool child = false, other = false;
  if (p.mode == M_GRID_HOST && !p.child_idle) {
    AggSeg seg = make_seg(a, g, level_mode);
    BodyArgs b = child_body(a, level_mode);
    void* cargs[] = {&b, &seg};
    NP_CK(cudaLaunchKernel(p.child, dim3(g.cgrid), dim3(g.cthreads), cargs, 0, s));
    child = true;
  }
  NP_CK(cudaEventRecord(e.ev[2], s));
  if (level_mode) {
    // the frontier sweep counts with the level bookkeeping ("other")
    if (p.sweep) NP_CK(cudaLaunchKernel(p.sweep, dim3(sweep_grid(a, g)), dim3(256), pargs, 0, s));
    advance_base_kernel<<<1, 1, 0, s>>>(w.st, 1);
    NP_CK(cudaGetLastError());
    other = true;
  }
  NP_CK(cudaEventRecord(e.ev[3], s));
  NP_CK(cudaEventSynchronize(e.ev[3]));
  float t01 = 0.f, t12 = 0.f, t23 = 0.f;
  NP_CK(cudaEventElapsedTime(&t01, e.ev[0], e.ev[1]));
  NP_CK(cudaEventElapsedTime(&t12, e.ev[1], e.ev[2]));
  NP_CK(cudaEventElapsedTime(&t23, e.ev[2], e.ev[3]));
  e.prof.parent_ms += t01;
  e.prof.parent_launches += 1;
  if (child) {
    e.prof.child_ms += t12;
    e.prof.child_launches += 1;
  }
  if (other) {
    e.prof.other_ms += t23;
    e.prof.other_launches += 1;
  }
  if (level_mode) {
    const int k = e.prof.levels;
    const double lvl = (double)t01 + (child ? (double)t12 : 0.0);
    if (lvl > e.prof.longest_level_ms) e.prof.longest_level_ms = lvl;
    if (k < NP_PROFILE_LEVELS) {
      e.prof.level_parents[k] = e.prof_next_parents;
      e.prof.level_parent_ms[k] = t01;
      e.prof.level_child_ms[k] = child ? t12 : 0.0;
      e.prof.levels = k + 1;
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

np_status cache_graph(Workspace& w, const std::string& key, cudaGraph_t graph, cudaGraphExec_t* out) {
  cudaGraphExec_t exec = nullptr;
  np_status st = instantiate(graph, &exec);
  if (st != NP_OK) {
    cudaGraphDestroy(graph);
    return st;
  }
  if (w.graphs.size() >= 64) ws_drop_graphs(w);
  w.graphs[key] = GraphEntry{graph, exec};
  *out = exec;
  return NP_OK;
}

np_status instantiate(cudaGraph_t graph, cudaGraphExec_t* exec) {
  cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *exec = nullptr;
    return e == cudaErrorInvalidValue ? NP_ERR_UNSUPPORTED : from_cuda(e);
  }
  return NP_OK;
}

np_status chunk_graph(Engine& e, Workspace& w, const Plan& p, const Args& a, const Grids& g, int K,
                      cudaGraphExec_t* out) {
  std::string key = graph_key("chunk", p, a, g, K);
  auto it = w.graphs.find(key);
  if (it != w.graphs.end()) {
    *out = it->second.exec;
    return NP_OK;
  }
  NP_CK(cudaStreamBeginCapture(e.cap_stream, cudaStreamCaptureModeThreadLocal));
  np_status st = NP_OK;
  for (int k = 0; k < K && st == NP_OK; k++) st = enqueue_pass(p, a, g, true, k, e.cap_stream);
  if (st == NP_OK) st = enqueue_advance(w.st, K, e.cap_stream, p.mode != M_DEVICE_LAUNCH);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(e.cap_stream, &graph);
  if (st != NP_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  NP_CK(ce);
  return cache_graph(w, key, graph, out);
}

np_status add_while_node(Engine& e, LevelState* st, cudaGraph_t graph, const cudaGraphNode_t* deps, size_t ndeps,
                         const Plan& p, const Args& a, const Grids& g, int K, cudaGraphNode_t* node) {
  cudaGraphConditionalHandle h;
  NP_CK(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
  // With the small-level loop: one run of it before the loop, which sets the
  // loop's condition itself (a traversal that stays small never enters it).
  cudaGraphNode_t pre;
  if (p.small) {
    Args sa = a;
    int k0 = 0, in_body = 0;
    void* sargs[] = {&sa, &h, &k0, &in_body};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(p.small);
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(1024);
    kp.kernelParams = sargs;
    NP_CK(cudaGraphAddKernelNode(&pre, graph, deps, ndeps, &kp));
    deps = &pre;
    ndeps = 1;
  }
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  NP_CK(cudaGraphAddNode(node, graph, deps, nullptr, ndeps, &cp));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  NP_CK(cudaStreamBeginCaptureToGraph(e.cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  np_status s = NP_OK;
  for (int k = 0; k < K && s == NP_OK; k++) s = enqueue_pass(p, a, g, true, k, e.cap_stream);
  // end of the body: the small-level loop, or a one-thread kernel, moves the
  // base on and sets the condition
  cudaError_t le;
  if (p.small) {
    Args sa = a;
    int in_body = 1;
    void* sargs[] = {&sa, &h, &K, &in_body};
    le = launch_pdl(p.small, dim3(1), dim3(1024), sargs, e.cap_stream, kPdl);
  } else {
    void* cargs[] = {&st, &h, &K};
    le = launch_pdl((const void*)set_cond_kernel, dim3(1), dim3(1), cargs, e.cap_stream, kPdl);
  }
  cudaError_t ce = cudaStreamEndCapture(e.cap_stream, &body);
  if (s != NP_OK) return s;
  NP_CK(le);
  NP_CK(ce);
  return NP_OK;
}

np_status while_graph(Engine& e, Workspace& w, const Plan& p, const Args& a, const Grids& g, int K,
                      cudaGraphExec_t* out) {
  std::string key = graph_key("while", p, a, g, K);
  auto it = w.graphs.find(key);
  if (it != w.graphs.end()) {
    *out = it->second.exec;
    return NP_OK;
  }
  cudaGraph_t graph = nullptr;
  NP_CK(cudaGraphCreate(&graph, 0));
  cudaGraphNode_t node;
  np_status st = add_while_node(e, w.st, graph, nullptr, 0, p, a, g, K, &node);
  if (st != NP_OK) {
    cudaGraphDestroy(graph);
    return st;
  }
  return cache_graph(w, key, graph, out);
}

np_status read_header(Engine& e, const Workspace& w, cudaStream_t s, int* level, int* count) {
  NP_CK(cudaMemcpyAsync(e.pin, w.st, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));   // base, count[3]
  NP_CK(cudaStreamSynchronize(s));
  *level = e.pin[0];
  *count = e.pin[1 + e.pin[0] % 3];
  return NP_OK;
}

np_status finish(Engine& e, const Workspace& w, cudaStream_t s, np_stats* stats) {
  if (!stats) return NP_OK;
  NP_CK(cudaMemcpyAsync(e.pin_state, w.st, sizeof(LevelState), cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  const LevelState& h = *e.pin_state;
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
    NP_CK(cudaMemsetAsync(&w.st->error, 0, sizeof(unsigned), s));
    NP_CK(cudaStreamSynchronize(s));
  }
  return status_from_bits(h.error);
}

np_status launch_level_loop(Engine& e, const Plan& p, const Args& a, const np_config& cfg, int max_levels,
                            cudaStream_t s) {
  // one block size for both phases: a multiple of 32 (parent warps) and of the
  // child block (child sub-blocks), at least the parent block and 256
  const int cb = cfg.child_block;
  int blk = cfg.parent_block > 256 ? cfg.parent_block : 256;
  if (blk < cb) blk = cb;
  blk = (blk + cb - 1) / cb * cb;
  if (blk > 1024) return NP_ERR_UNSUPPORTED;
  // the whole resident grid, or parent_grid CTAs (a small grid keeps the
  // per-level barriers cheap on small problems)
  const int full = occupancy(e, p.loop, blk) * e.sms;
  const int grid = cfg.parent_grid > 0 && cfg.parent_grid < full ? cfg.parent_grid : full;
  Args aa = a;
  aa.k = 0;
  int ml = max_levels;
  void* args[] = {&aa, &ml};
  NP_CK(cudaLaunchCooperativeKernel(p.loop, dim3(grid), dim3(blk), args, 0, s));
  return NP_OK;
}

np_status run_levels(Engine& e, Workspace& w, const Plan& p, const Args& a, const np_config& cfg, int64_t parents,
                     int max_levels, cudaStream_t s) {
  Grids g = grids_for(e, p, cfg, parents);
  const int driver = resolve_driver(p, cfg);
  if ((driver == NP_DRIVER_WHILE || driver == NP_DRIVER_PERSISTENT) && p.mode == M_DEVICE_LAUNCH)
    return NP_ERR_UNSUPPORTED;
  if (driver == NP_DRIVER_PERSISTENT && !p.loop) return NP_ERR_UNSUPPORTED;
  if (e.profile) {
    // per-level records describe this call only
    e.prof.levels = 0;
    e.prof.longest_level_ms = 0.0;
    for (int iter = 0;; iter++) {
      if (iter > max_levels + 16) return NP_ERR_TIMEOUT;
      NP_TRY(profiled_pass(e, w, p, a, g, true, s));
      int level = 0, count = 0;
      NP_TRY(read_header(e, w, s, &level, &count));
      e.prof_next_parents = count;
      if (count <= 0 || level >= max_levels) break;
    }
    return NP_OK;
  }
  if (driver == NP_DRIVER_WHILE) {
    cudaGraphExec_t exec;
    NP_TRY(while_graph(e, w, p, a, g, cfg.unroll, &exec));
    NP_CK(cudaGraphLaunch(exec, s));
    return NP_OK;
  }
  if (driver == NP_DRIVER_PERSISTENT) return launch_level_loop(e, p, a, cfg, max_levels, s);
  cudaGraphExec_t exec = nullptr;
  if (driver == NP_DRIVER_CHUNK && p.mode != M_DEVICE_LAUNCH) NP_TRY(chunk_graph(e, w, p, a, g, cfg.unroll, &exec));
  const int K = driver == NP_DRIVER_CHUNK ? cfg.unroll : 1;
  for (int iter = 0;; iter++) {
    if (iter > max_levels + 16) return NP_ERR_TIMEOUT;   // a level failed to advance
    if (exec) {
      NP_CK(cudaGraphLaunch(exec, s));
    } else {
      for (int k = 0; k < K; k++) NP_TRY(enqueue_pass(p, a, g, true, k, s));
      NP_TRY(enqueue_advance(w.st, K, s, p.mode != M_DEVICE_LAUNCH));
    }
    int level = 0, count = 0;
    NP_TRY(read_header(e, w, s, &level, &count));
    if (count <= 0 || level >= max_levels) break;
  }
  return NP_OK;
}

np_status check_csr_device(const np_csr* graphs, int count, int* scratch, cudaStream_t s) {
  NP_CK(cudaMemsetAsync(scratch, 0, sizeof(int), s));
  for (int i = 0; i < count; i++) {
    const np_csr& g = graphs[i];
    const long long top = g.n > g.m ? (long long)g.n : g.m;
    csr_check_kernel<<<blocks_for(top), 256, 0, s>>>(g.row_ptr, g.col_idx, g.n, g.m, scratch);
    NP_CK(cudaGetLastError());
  }
  int bad = 0;
  NP_CK(cudaMemcpyAsync(&bad, scratch, sizeof(int), cudaMemcpyDeviceToHost, s));
  NP_CK(cudaStreamSynchronize(s));
  return bad ? NP_ERR_INVALID : NP_OK;
}

np_status check_csr(const np_csr* g, bool need_w) {
  if (!g || !g->row_ptr || (!g->col_idx && g->m > 0) || g->n < 1 || g->m < 0 || g->m >= INT_MAX) return NP_ERR_INVALID;
  if (need_w && !g->weights && g->m > 0) return NP_ERR_INVALID;
  return NP_OK;
}

}  // namespace nestpar
