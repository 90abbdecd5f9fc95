// Allocation-free tessellation entry point (np_bezier_noalloc).
//
// Its scratch (level state, aggregation records and block offsets, look-back
// tile states) lives in one file-scope __device__ array sized for
// NP_NOALLOC_MAX_CURVES curves, so a call allocates nothing: no cudaMalloc,
// no pinned host memory, no graph, no event, no stream. Host code cannot use
// the array's name as a device address (on the host it names a stand-in
// object), so the device address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels as a pointer.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "nestpar.h"
#include "np_engine.h"

using namespace nestpar;

namespace {

constexpr size_t al256(size_t x) { return (x + 255) / 256 * 256; }
constexpr int kMaxCurves = NP_NOALLOC_MAX_CURVES;
constexpr int kSlots = ((kMaxCurves + 1023) / 1024) * 1024 + 1024;   // records, block offsets
constexpr int kTiles = kSlots / 32 + 64;                              // parent tiles (>= 64 parents each)
constexpr size_t kOffRec = al256(sizeof(LevelState));
constexpr size_t kOffBoff = kOffRec + al256(sizeof(int4) * kSlots);
constexpr size_t kOffLbFlag = kOffBoff + al256(sizeof(int) * kSlots);
constexpr size_t kOffLbAgg = kOffLbFlag + al256(sizeof(unsigned long long) * kTiles);
constexpr size_t kOffLbIncl = kOffLbAgg + al256(sizeof(uint4) * kTiles);
constexpr size_t kOffObFlag = kOffLbIncl + al256(sizeof(uint4) * kTiles);
constexpr size_t kOffObAgg = kOffObFlag + al256(sizeof(unsigned long long) * kTiles);
constexpr size_t kOffObIncl = kOffObAgg + al256(sizeof(uint4) * kTiles);
constexpr size_t kOffGrpCtr = kOffObIncl + al256(sizeof(uint4) * kTiles);
constexpr size_t kOffGrpAcc = kOffGrpCtr + al256(sizeof(int) * kTiles);
constexpr size_t kOffGrpTot = kOffGrpAcc + al256(sizeof(unsigned long long) * kTiles);
constexpr size_t kScratchBytes = kOffGrpTot + al256(sizeof(uint2) * kTiles);   // about 1.5 MB

// The scratch. Every GPU that loads the library holds it until the process exits.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
struct DeviceScratch {
  unsigned char* base = nullptr;   // device address of g_scratch on this device
  int sms = 0;
};
std::mutex g_mu;
DeviceScratch g_devices[kMaxDevices];

// Per-call reset of what must start at zero (the epoch only grows, so the
// look-back flags of earlier calls never match a later call).
__global__ void noalloc_reset_kernel(LevelState* st) {
  st->solve_id += 1;
  st->body_iters = 0;
  st->bar_count = 0u;
  for (int k = 0; k < 4; k++) {
    st->ticket[k] = 0;
    st->agg_records[k] = 0;
    st->agg_blocks[k] = 0;
    st->agg_acc[k] = 0ull;
    st->child_ticket[k] = 0;
  }
  st->error = 0u;
  for (int k = 0; k < S_N; k++) st->s[k] = 0ull;
}

// Set-up on the current device, first call only: find the array's device
// address and clear it. Done on the caller's stream; no allocation.
np_status device_scratch(cudaStream_t s, DeviceScratch* out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NP_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  DeviceScratch& d = g_devices[dev];
  if (!d.base) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return NP_ERR_CUDA;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
      return NP_ERR_CUDA;
    if (cudaMemsetAsync(p, 0, kScratchBytes, s) != cudaSuccess) return NP_ERR_CUDA;
    d.base = static_cast<unsigned char*>(p);
    d.sms = sms;
  }
  *out = d;
  return NP_OK;
}

// After the call's kernels: a bounded wait that gave up (look-back timeout)
// leaves offsets it could not finish, so the total becomes -1 for the caller
// to see (a call that completed never writes a negative total).
__global__ void noalloc_status_kernel(const LevelState* st, int* offsets, int ncurves) {
  if (st->error & kErrTimeout) offsets[ncurves] = -1;
}

}  // namespace

extern "C" np_status np_bezier_noalloc(const float* ctrl, int32_t ncurves, int32_t* offsets, float* points,
                                       int64_t cap, const np_config* cfg, void* stream) {
  if ((ncurves > 0 && !ctrl) || !offsets || ncurves < 0 || cap < 0 || (cap > 0 && !points))
    return NP_ERR_INVALID;
  np_status cs = check_config(cfg);   // the argument checks of np_bezier
  if (cs != NP_OK) return cs;
  if (ncurves > kMaxCurves) return NP_ERR_INVALID;   // beyond the static scratch
  const bool nodp = cfg->variant == NP_VARIANT_NODP;
  // device launches, and packed serial children (records beyond the static scratch), are not run here
  if (!nodp && (cfg->granularity != NP_GRAN_GRID_HOST || serial_form(*cfg) == NP_SERIAL_PACKED))
    return NP_ERR_UNSUPPORTED;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ncurves == 0) return cudaMemsetAsync(offsets, 0, sizeof(int32_t), s) == cudaSuccess ? NP_OK : NP_ERR_CUDA;

  DeviceScratch d;
  np_status st = device_scratch(s, &d);
  if (st != NP_OK) return st;
  LevelState* state = reinterpret_cast<LevelState*>(d.base);

  Args a;
  std::memset(&a, 0, sizeof(a));
  a.st = state;
  a.count_fixed = ncurves;
  a.L_fixed = 0;
  a.rec = reinterpret_cast<int4*>(d.base + kOffRec);
  a.boff = reinterpret_cast<int*>(d.base + kOffBoff);
  a.lb_flag = reinterpret_cast<unsigned long long*>(d.base + kOffLbFlag);
  a.lb_agg = reinterpret_cast<uint4*>(d.base + kOffLbAgg);
  a.lb_incl = reinterpret_cast<uint4*>(d.base + kOffLbIncl);
  a.ob_flag = reinterpret_cast<unsigned long long*>(d.base + kOffObFlag);
  a.ob_agg = reinterpret_cast<uint4*>(d.base + kOffObAgg);
  a.ob_incl = reinterpret_cast<uint4*>(d.base + kOffObIncl);
  a.grp_ctr = reinterpret_cast<int*>(d.base + kOffGrpCtr);
  a.grp_acc = reinterpret_cast<unsigned long long*>(d.base + kOffGrpAcc);
  a.grp_total = reinterpret_cast<uint2*>(d.base + kOffGrpTot);
  a.threshold = cfg->threshold;
  a.cfactor = cfg->cfactor;
  a.child_block = cfg->child_block;
  a.scan = cfg->scan;
  a.offsets = offsets;
  a.cap = cap;
  a.b.st = state;
  a.b.vmask = 0x7fffffff;
  a.b.ctrl = ctrl;
  a.b.points = reinterpret_cast<float2*>(points);

  // the kernels np_bezier runs for this configuration
  const BodyKernels& K = bezier_kernels();
  const Plan plan = make_plan(K, *cfg);
  const void* parent = plan.parent;
  const int pb = cfg->parent_block, cb = cfg->child_block;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, parent, pb, 0) != cudaSuccess || occ < 1) occ = 1;
  int pgrid = cfg->parent_grid > 0 ? cfg->parent_grid : occ * d.sms;
  const int tiles = (ncurves + pb - 1) / pb;
  if (pgrid > tiles) pgrid = tiles;

  noalloc_reset_kernel<<<1, 1, 0, s>>>(state);
  if (cudaGetLastError() != cudaSuccess) return NP_ERR_CUDA;
  void* pargs[] = {&a};
  if (cudaLaunchKernel(parent, dim3(pgrid), dim3(pb), pargs, 0, s) != cudaSuccess) return NP_ERR_CUDA;
  if (!nodp) {
    AggSeg seg;
    std::memset(&seg, 0, sizeof(seg));
    seg.rec = a.rec;
    seg.boff = a.boff;
    seg.mode = a.scan == NP_SCAN_LOOKBACK ? 1 : 2;
    seg.cb = cb;
    const int cthreads = cb < 256 ? 256 : cb;
    BodyArgs b = a.b;
    int cocc = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cocc, plan.child, cthreads, 0) != cudaSuccess ||
        cocc < 1)
      cocc = 1;
    void* cargs[] = {&b, &seg};
    if (cudaLaunchKernel(plan.child, dim3(cocc * d.sms), dim3(cthreads), cargs, 0, s) != cudaSuccess)
      return NP_ERR_CUDA;
  }
  noalloc_status_kernel<<<1, 1, 0, s>>>(state, offsets, ncurves);
  if (cudaGetLastError() != cudaSuccess) return NP_ERR_CUDA;
  return NP_OK;
}
