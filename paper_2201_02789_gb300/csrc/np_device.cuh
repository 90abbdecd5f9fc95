// Device side of the nested-parallelism engine (sm_103a).
//
// One "level" runs the children of a set of parents. Parents are processed in
// tiles taken from an atomic ticket, so tile order = parent order and a tile
// only ever waits (in a look-back) on tiles that running threads already own:
// warp-sized tiles for the forms without device launches (parent_warp), tiles
// of `parent_block` parents per CTA for the device-launch forms, whose block
// granularity needs CTA tiles (parent_kernel). For every parent the child
// count N is computed (Section III-D: the number of child threads, not
// gDim * bDim), then:
//
//   NODP        the parent loops over its N children (no launch code at all);
//   N < T       the parent loops over its children (thresholding, Section III-A);
//   N >= T      the children go to a child grid of ceil(ceil(N/bDim)/CF)
//               coarsened blocks (coarsening, Section IV-B), launched
//               per parent (GRAN_NONE) or aggregated (Sections II-B, V-A).
//
// Aggregation scans the coarsened block counts of the launching parents of a
// scope (warp shuffles, a block scan, a decoupled look-back across the tiles
// of a group of blocks or of the whole grid, or the paper's packed 64-bit
// atomic), stores one record {parent, row start, N} per launching parent and
// the scanned block offset, and one thread launches Sum(cg) blocks. Each
// aggregated child block finds its parent by a 32-ary warp search over the
// offsets, then runs CF original blocks of that parent (disaggregation outside
// the coarsening loop, Section VI).
//
// Level bookkeeping is slot based so that no kernel has to finish a level:
// level L = base + k, where base only changes between graph bodies and k is
// the kernel's position in the body; per-level counters live in slot L % 4,
// and the parent grid of level L clears the slot and frontier count that
// level L + 2 will use.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Tuning knobs (compile time): items a child thread keeps in flight, items a
// serialising parent thread keeps in flight, optional register caps.
// 1: aggregated child blocks stage their edge lists in shared memory with the
// bulk-copy engine, one block ahead (bodies with contiguous lists, CF <= 8)
#ifndef NP_TMA_STAGE
#define NP_TMA_STAGE 0
#endif
#ifndef NP_CHILD_BATCH
#define NP_CHILD_BATCH 8
#endif
#ifndef NP_SERIAL_BATCH
#define NP_SERIAL_BATCH 8
#endif
// Programmatic dependent launch between the kernels of the launch-free level
// loop: each such kernel lets the next one be scheduled at once, then waits
// for its own predecessor to complete before it reads anything. A kernel
// without this entry is never launched with the attribute.
#ifndef NP_PDL
#define NP_PDL 1
#endif

#if NP_PDL
#define NP_PDL_ENTRY()                          \
  do {                                          \
    cudaTriggerProgrammaticLaunchCompletion();  \
    cudaGridDependencySynchronize();            \
  } while (0)
#else
#define NP_PDL_ENTRY() \
  do {                 \
  } while (0)
#endif

// items per lane per round of the aggregated form's spread serial loop
#ifndef NP_SPREAD_BATCH
#define NP_SPREAD_BATCH 8
#endif
// aggregated child blocks of 4 original blocks read edge lists with 16-byte
// loads (an option: the scalar loads are already coalesced, 128 bytes per warp
// instruction, and measured faster)
#ifndef NP_VEC4
#define NP_VEC4 0
#endif
// triangle counting: intersect lists of comparable length by a blocked merge
// (else by binary searches of the longer list)
#ifndef NP_TC_MERGE
#define NP_TC_MERGE 1
#endif
// The load that filters a child item before its atomic (level[v] for BFS,
// dist(v) for SSSP). Only the atomic decides, and a stale value can only be
// an older one (levels are claimed once, distances only fall), so a filter
// read through L1 (1) can cost an unneeded atomic but never a wrong result.
#ifndef NP_FILTER_L1
#define NP_FILTER_L1 1
#endif
#if NP_FILTER_L1
#define NP_FILTER_LOAD(p) __ldca(p)
#else
#define NP_FILTER_LOAD(p) __ldcg(p)
#endif
// 1: a relaxation reads dist(v) first and issues the atomic only when it would
// lower it; 0: every relaxation issues the atomic (one dependent round trip
// fewer, more atomics)
#ifndef NP_SSSP_PRECHECK
#define NP_SSSP_PRECHECK 1
#endif
#ifdef NP_CHILD_MAXREG
#define NP_CHILD_BOUNDS __maxnreg__(NP_CHILD_MAXREG)
#define NP_CHILD_AGG_BOUNDS(CF) __maxnreg__(NP_CHILD_MAXREG)
#else
#define NP_CHILD_BOUNDS __launch_bounds__(1024)
// the aggregated child grid with up to 4 blocks per coarsened block fits in 48
// registers without spilling: five 256-thread CTAs per SM instead of four
#define NP_CHILD_AGG_BOUNDS(CF) __maxnreg__((CF) <= 4 ? 48 : 64)
#endif
#ifdef NP_PARENT_MAXREG
#define NP_PARENT_BOUNDS __maxnreg__(NP_PARENT_MAXREG)
#else
#define NP_PARENT_BOUNDS __launch_bounds__(kMaxParentBlock)
#endif

namespace nestpar {

constexpr int kMaxParentBlock = 512;
constexpr unsigned kErrLaunch = 1u, kErrTimeout = 2u, kErrCapacity = 4u;
constexpr int kSpinLimit = 1 << 21;   // polls before a look-back wait gives up
constexpr unsigned kFull = 0xffffffffu;

enum Gran : int { G_NONE = 0, G_WARP = 1, G_BLOCK = 2, G_MULTIBLOCK = 3, G_GRID_DEVICE = 4,
                  G_GRID_HOST = 5, G_NODP = 6 };
enum Stat : int { S_LEVELS, S_PARENTS, S_SERIAL, S_LAUNCHP, S_DEVLAUNCH, S_AGGGRID, S_CBLOCKS,
                  S_ITEMS, S_PUSHES, S_LFAIL, S_TIMEOUT, S_CITEMS, S_N };

// Device-resident state of one solve. Level L reads frontier buffer L&1 with
// count[L%3] and appends to buffer (L+1)&1 / count[(L+1)%3]; the parent
// kernel of level L zeroes count[(L+2)%3], which level L+1 appends to.
// base and count[] share one 16-byte word: one load gives L and its size.
struct __align__(16) LevelState {
  int base;                      // level of body position 0; changes only between bodies
  int count[3];
  unsigned long long solve_id;   // look-back epoch of level L: solve_id << 31 | L (never reused)
  int max_levels;
  unsigned error;
  int ticket[4];                 // slot L % 4: next parent tile of level L
  int agg_records[4];            // slot L % 4: grid-host totals, look-back scan
  int agg_blocks[4];
  unsigned long long agg_acc[4]; // slot L % 4: grid-host totals, atomic scan (parents << 40 | blocks)
  unsigned long long s[S_N];     // counters (np_stats)
  int body_iters;                // conditional-while iterations of this solve (bounded)
  int pad;
  int child_ticket[4];           // slot L % 4: next chunk of aggregated blocks (balanced bodies)
  unsigned bar_count;            // grid barrier of the persistent level loop: arrivals
  unsigned bar_gen;              // and generation
};

__device__ __forceinline__ unsigned long long level_epoch(const LevelState* st, int L) {
  return (__ldcg(&st->solve_id) << 31) | (unsigned long long)(unsigned)L;
}

// Level L of a level-mode kernel at body position k, and that level's frontier size.
__device__ __forceinline__ void level_of(const LevelState* st, int k, int& L, int& count) {
  const int4 h = __ldcg(reinterpret_cast<const int4*>(st));
  L = h.x + k;
  const int m = L % 3;
  count = m == 0 ? h.y : (m == 1 ? h.z : h.w);
}

// Run by one thread of the parent grid of level L: clear what level L + 2
// will use, and count the level.
__device__ __forceinline__ void level_open(LevelState* st, int L, int count) {
  const int s2 = (L + 2) & 3;
  st->ticket[s2] = 0;
  st->agg_records[s2] = 0;
  st->agg_blocks[s2] = 0;
  st->agg_acc[s2] = 0ull;
  st->child_ticket[s2] = 0;
  st->count[(L + 2) % 3] = 0;
  if (count > 0) {
    atomicAdd(&st->s[S_LEVELS], 1ull);
    if (L > 0) atomicAdd(&st->s[S_PUSHES], (unsigned long long)count);
  }
}

// What a child item needs; passed by value to every child grid.
struct BodyArgs {
  const int* col;
  const unsigned* w;
  int* level;
  unsigned* dist;
  int* stamp;
  const float* ctrl;
  float2* points;
  int* next;
  int* next_count;
  LevelState* st;
  int L;                         // BFS writes L+1; SSSP stamps L+1
  // Several traversals of one graph at once: a vertex id is q * 2^k + v, the
  // graph vertex is id & vmask and per-query state is indexed by the id; a
  // single traversal has vmask = all ones.
  int vmask;
  const int* row_ptr;            // triangle counting: row bounds of a child's vertex
  unsigned long long* acc;       // triangle counting: kTcSlots partial counts
  unsigned long long* dtag;      // SSSP, packed form: dist << 32 | tag per vertex
};

struct Args {
  LevelState* st;
  const int* ids;                // fixed-count mode: parent ids (NULL = 0..count-1)
  int* fr0;
  int* fr1;
  int* next_ovr;                 // fixed-count mode: append target
  int* next_count_ovr;
  int count_fixed;               // >= 0: fixed-count mode (one pass, no level bookkeeping)
  int L_fixed;
  const int* row_ptr;
  BodyArgs b;
  int* offsets;
  long long cap;
  int4* rec;
  int* boff;
  unsigned long long* lb_flag;   // look-back tile states of the aggregation scan
  uint4* lb_agg;
  uint4* lb_incl;
  unsigned long long* ob_flag;   // look-back tile states of the output-offset scan
  uint4* ob_agg;
  uint4* ob_incl;
  int* grp_ctr;                  // multi-block group arrival counters
  unsigned long long* grp_acc;   // multi-block packed atomic accumulators
  uint2* grp_total;              // multi-block look-back totals
  int threshold;
  int cfactor;
  int child_block;
  int group_blocks;              // 0 = whole grid (grid granularity)
  int agg_threshold;
  int scan;                      // 0 look-back, 1 atomic
  int k;                         // level mode: position in the graph body (level = base + k)
  int pad;
};

struct AggSeg {
  const int4* rec;
  const int* boff;
  int* fr0;                      // level mode: frontier buffers, to find this level's append target
  int* fr1;
  int nrec;
  int total;
  int mode;                      // 0: fixed segment; 1: grid-host, look-back totals; 2: grid-host, atomic totals
  int k;                         // level mode: position in the graph body
  int level_mode;                // 1: take L, next and next_count from the level state
  int cb;                        // child block size; a CTA hosts blockDim.x / cb child blocks
  int pad;
};

// ---------------------------------------------------------------- primitives

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}
__host__ __device__ __forceinline__ int ceil_div(int a, int b) { return (a + b - 1) / b; }

struct V3 {
  unsigned a, b, c;
};
__device__ __forceinline__ V3 v3add(V3 x, V3 y) { return V3{x.a + y.a, x.b + y.b, x.c + y.c}; }
__device__ __forceinline__ V3 warp_sum3(V3 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.a += __shfl_xor_sync(kFull, v.a, o);
    v.b += __shfl_xor_sync(kFull, v.b, o);
    v.c += __shfl_xor_sync(kFull, v.c, o);
  }
  return v;
}

// Decoupled look-back (single-pass prefix scan over tiles): run by one full
// warp; returns the exclusive prefix of tile `tile` within [first, tile].
// Flags hold (epoch << 2) | status, status 1 = aggregate published,
// 2 = inclusive prefix published. Waits are bounded: on expiry the error word
// gets kErrTimeout and the wait is abandoned (result then wrong, never a hang).
__device__ inline V3 lookback(unsigned long long* flag, uint4* agg, uint4* incl, int tile, int first,
                       unsigned long long epoch, V3 mine, LevelState* st) {
  const int lane = threadIdx.x & 31;
  const unsigned long long fA = (epoch << 2) | 1ull, fP = (epoch << 2) | 2ull;
  if (tile == first) {
    if (lane == 0) {
      incl[tile] = make_uint4(mine.a, mine.b, mine.c, 0u);
      st_release_u64(&flag[tile], fP);
    }
    return V3{0, 0, 0};
  }
  if (lane == 0) {
    agg[tile] = make_uint4(mine.a, mine.b, mine.c, 0u);
    st_release_u64(&flag[tile], fA);
  }
  V3 excl{0, 0, 0};
  int j = tile - 1;
  for (;;) {
    const int idx = j - lane;
    const bool in = idx >= first;
    unsigned long long f = fP;
    bool timed_out = false;
    if (in) {
      f = ld_acquire_u64(&flag[idx]);
      int spins = 0;
      while ((f >> 2) != epoch || (f & 3ull) == 0ull) {
        if (++spins > kSpinLimit) {
          timed_out = true;
          break;
        }
        __nanosleep(32);
        f = ld_acquire_u64(&flag[idx]);
      }
      if (timed_out) {
        atomicOr(&st->error, kErrTimeout);
        atomicAdd(&st->s[S_TIMEOUT], 1ull);
        f = fP;
      }
    }
    const bool isP = (f & 3ull) == 2ull;
    V3 v{0, 0, 0};
    if (in && !timed_out) {
      uint4 x = __ldcg(isP ? &incl[idx] : &agg[idx]);
      v = V3{x.x, x.y, x.z};
    }
    const unsigned pm = __ballot_sync(kFull, isP);
    const int stop = pm ? __ffs(pm) - 1 : 31;
    if (lane > stop) v = V3{0, 0, 0};
    excl = v3add(excl, warp_sum3(v));
    if (pm) break;
    j -= 32;
  }
  if (lane == 0) {
    V3 inc = v3add(excl, mine);
    incl[tile] = make_uint4(inc.a, inc.b, inc.c, 0u);
    st_release_u64(&flag[tile], fP);
  }
  return excl;
}

// Exclusive scan of two counters over the CTA. Returns this thread's exclusive
// values and the CTA totals (in all threads). Uses s[0..32].
__device__ __forceinline__ void block_scan2(unsigned a, unsigned b, unsigned& ea, unsigned& eb,
                                            unsigned& ta, unsigned& tb, uint2* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned xa = __shfl_up_sync(kFull, ia, o), xb = __shfl_up_sync(kFull, ib, o);
    if (lane >= o) {
      ia += xa;
      ib += xb;
    }
  }
  if (lane == 31) s[warp] = make_uint2(ia, ib);
  __syncthreads();
  if (warp == 0) {
    uint2 t = lane < nw ? s[lane] : make_uint2(0u, 0u);
    unsigned xa = t.x, xb = t.y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned ya = __shfl_up_sync(kFull, xa, o), yb = __shfl_up_sync(kFull, xb, o);
      if (lane >= o) {
        xa += ya;
        xb += yb;
      }
    }
    if (lane < nw) s[lane] = make_uint2(xa - t.x, xb - t.y);   // exclusive warp prefix
    if (lane == 31) s[32] = make_uint2(xa, xb);               // CTA total
  }
  __syncthreads();
  uint2 wp = s[warp];
  ea = wp.x + ia - a;
  eb = wp.y + ib - b;
  ta = s[32].x;
  tb = s[32].y;
  __syncthreads();
}

// Largest j in [lo, hi) with boff[j] <= B, for strictly increasing boff and
// boff[lo] <= B: a 32-ary search run by one warp (one probe per lane and one
// ballot per round, no block barrier), every lane returns j. Each warp of a
// child block runs it on its own, so the block never waits on itself.
__device__ __forceinline__ int warp_search(const int* boff, int lo, int hi, int B) {
  const int lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const int stride = ceil_div(hi - lo, 32);
    const int idx = lo + lane * stride;
    const bool p = idx < hi && __ldcg(&boff[idx]) <= B;
    const int c = max(__popc(__ballot_sync(kFull, p)), 1);   // >= 1 by the precondition; clamped to stay in range
    lo += (c - 1) * stride;
    hi = min(hi, lo + stride);
  }
  const int idx = lo + lane;
  const bool p = idx < hi && __ldcg(&boff[idx]) <= B;
  return lo + max(__popc(__ballot_sync(kFull, p)), 1) - 1;
}

// The same search when the answer is usually close to lo (the next parent of
// a contiguous run of blocks): one 32-entry window first, the full search only
// when B lies beyond it.
__device__ __forceinline__ int warp_search_near(const int* boff, int lo, int hi, int B) {
  const int lane = threadIdx.x & 31;
  const int idx = lo + lane;
  const bool p = idx < hi && __ldcg(&boff[idx]) <= B;
  const int c = __popc(__ballot_sync(kFull, p));
  if (c < 32 || lo + 32 >= hi) return lo + max(c, 1) - 1;
  return warp_search(boff, lo + 31, hi, B);
}

// ------------------------------------------------------------ frontier sinks
//
// Appends to the next frontier go through a sink. All appends of a level hit
// one counter, so the sinks keep atomics on it rare and frontiers exact (no
// holes):
//   StageSink  the 32 lanes of a warp append a batch together into a
//              shared-memory buffer of the CTA (one shared atomic per warp
//              batch); the CTA flushes the buffer with one global atomic when it
//              finishes; what does not fit goes to global memory at once;
//   CtaSink    the same buffer filled by diverged lanes (the serial loops of the
//              CTA-tiled parent kernel), flushed once per tile;
//   WarpSink   one exact reservation per warp batch (device-launched child
//              grids of one parent, which are too small to stage).
struct WarpSink {
  int* next;
  int* count;
  template <int K>
  __device__ __forceinline__ void push(const bool (&pf)[K], const int (&v)[K]) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < K; k++) c += pf[k] ? 1 : 0;
    if (!__any_sync(kFull, c != 0)) return;   // most batches append nothing: skip the scan
    const int lane = threadIdx.x & 31;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    const int total = __shfl_sync(kFull, inc, 31);
    if (total == 0) return;
    int r = inc - c;
    int b0 = 0;
    if (lane == 31) b0 = atomicAdd(count, total);
    b0 = __shfl_sync(kFull, b0, 31);
#pragma unroll
    for (int k = 0; k < K; k++)
      if (pf[k]) next[b0 + r++] = v[k];
  }
};

constexpr int kCtaStage = 2048;   // shared staging slots of a child / warp-tiled parent CTA

struct StageSink {
  int* next;
  int* count;
  int* q;    // shared staging buffer [kCtaStage]
  int* qn;   // shared fill counter (counts appends beyond the buffer too)
  template <int K>
  __device__ __forceinline__ void push(const bool (&pf)[K], const int (&v)[K]) {
    int c = 0;
#pragma unroll
    for (int k = 0; k < K; k++) c += pf[k] ? 1 : 0;
    if (!__any_sync(kFull, c != 0)) return;   // most batches append nothing: skip the scan
    const int lane = threadIdx.x & 31;
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int x = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += x;
    }
    const int total = __shfl_sync(kFull, inc, 31);
    if (total == 0) return;
    int pos = 0;
    if (lane == 0) pos = atomicAdd(qn, total);
    pos = __shfl_sync(kFull, pos, 0);
    const int fit = max(0, min(total, kCtaStage - pos));   // appends that land in the buffer
    int gb = 0;
    if (fit < total) {
      if (lane == 0) gb = atomicAdd(count, total - fit);
      gb = __shfl_sync(kFull, gb, 0);
    }
    int r = inc - c;
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (pf[k]) {
        if (r < fit) q[pos + r] = v[k];
        else next[gb + (r - fit)] = v[k];
        r++;
      }
    }
  }
};

// Run by every thread of the CTA once it is done appending: one atomic on the
// level counter reserves the staged appends, then the CTA copies them out.
__device__ __forceinline__ void stage_flush(const int* q, int* qn, int* next, int* count, int* s_base) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const int n = min(*qn, kCtaStage);
    *s_base = n > 0 ? atomicAdd(count, n) : 0;
    *qn = n;
  }
  __syncthreads();
  const int n = *qn, base = *s_base;
  for (int i = threadIdx.x; i < n; i += blockDim.x) next[base + i] = q[i];
}

constexpr int kStageSlots = 1024;   // shared-memory staging slots per parent CTA

struct CtaSink {
  int* next;
  int* count;
  int* q;    // shared staging buffer [kStageSlots]
  int* qn;   // shared fill counter (may exceed kStageSlots: the excess went to global memory)
  template <int K>
  __device__ __forceinline__ void push(const bool (&pf)[K], const int (&v)[K]) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      if (!pf[k]) continue;
      const int pos = atomicAdd(qn, 1);
      if (pos < kStageSlots) {
        q[pos] = v[k];
      } else {
        next[atomicAdd(count, 1)] = v[k];
      }
    }
  }
};

// ------------------------------------------------------------------- bodies
//
// A body gives the child count of a parent (count), what every child of a
// parent shares (parent), the loads of one child item (fetch) and the effect
// of a batch of K items of one thread (apply_batch), which reports the
// vertices to append to the next frontier. A batch issues all its loads, then
// all its atomics, before it uses any of their results, so a thread keeps K
// memory operations in flight.

// BFS (Section VII): child item = out-edge u->v; claims v for level L+1.
struct BfsBody {
  static constexpr bool kOffsets = false;
  static constexpr bool kPushes = true;
  static constexpr bool kBalance = false;   // child blocks cost the same: static ranges
  static constexpr int kStage = 1;          // edge lists the child can stage: col
  struct P {
    int base;
    int qbase;   // query part of the ids of this parent's children
  };
  struct F {
    int v;
  };
  __device__ static void count(const Args& a, int pid, int& base, int& N) {
    const int u = pid & a.b.vmask;
    base = __ldg(&a.row_ptr[u]);
    N = __ldg(&a.row_ptr[u + 1]) - base;
  }
  __device__ static P parent(const BodyArgs& b, int pid, int base, int) { return P{base, pid & ~b.vmask}; }
  __device__ static P shfl(const P& p, int src) {
    return P{__shfl_sync(kFull, p.base, src), __shfl_sync(kFull, p.qbase, src)};
  }
  __device__ static F fetch(const BodyArgs& b, const P& p, int i) { return F{p.qbase | __ldg(&b.col[p.base + i])}; }
  __device__ static F fetch_from(const P& p, int col, unsigned) { return F{p.qbase | col}; }
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&)[K], const int (&)[K], const F (&f)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
    int cur[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      v[k] = f[k].v;
      cur[k] = valid[k] ? NP_FILTER_LOAD(&b.level[v[k]]) : 0;
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      push[k] = valid[k] && cur[k] == -1;
      if (push[k]) cur[k] = atomicCAS(&b.level[v[k]], -1, b.L + 1);
    }
#pragma unroll
    for (int k = 0; k < K; k++) push[k] = push[k] && cur[k] == -1;
  }
};

// SSSP (Section VII): child item = relaxation of out-edge u->v with weight w.
struct SsspBody {
  static constexpr bool kOffsets = false;
  static constexpr bool kPushes = true;
  static constexpr bool kBalance = false;
  static constexpr int kStage = 2;          // col and w
  struct P {
    int base;
    unsigned du;
    int qbase;   // query part of the ids of this parent's children
  };
  struct F {
    int v;
    unsigned w;
  };
  __device__ static void count(const Args& a, int pid, int& base, int& N) {
    const int u = pid & a.b.vmask;
    base = __ldg(&a.row_ptr[u]);
    N = __ldg(&a.row_ptr[u + 1]) - base;
  }
  __device__ static P parent(const BodyArgs& b, int pid, int base, int) {
    return P{base, __ldcg(&b.dist[pid]), pid & ~b.vmask};
  }
  __device__ static F fetch(const BodyArgs& b, const P& p, int i) {
    return F{p.qbase | __ldg(&b.col[p.base + i]), __ldg(&b.w[p.base + i])};
  }
  __device__ static F fetch_from(const P& p, int col, unsigned w) { return F{p.qbase | col, w}; }
  __device__ static P shfl(const P& p, int src) {
    return P{__shfl_sync(kFull, p.base, src), (unsigned)__shfl_sync(kFull, (int)p.du, src),
             __shfl_sync(kFull, p.qbase, src)};
  }
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&p)[K], const int (&)[K], const F (&f)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
    unsigned nd[K], cur[K];
    bool live[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      v[k] = f[k].v;
      live[k] = p[k].du != 0xffffffffu;
      const unsigned long long s = (unsigned long long)p[k].du + f[k].w;
      nd[k] = s >= 0xffffffffull ? 0xfffffffeu : (unsigned)s;
      cur[k] = (valid[k] && live[k]) ? NP_FILTER_LOAD(&b.dist[v[k]]) : 0u;
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      push[k] = valid[k] && live[k] && nd[k] < cur[k];
      if (push[k]) cur[k] = atomicMin(&b.dist[v[k]], nd[k]);
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      push[k] = push[k] && nd[k] < cur[k];
      if (push[k]) push[k] = atomicExch(&b.stamp[v[k]], b.L + 1) != b.L + 1;
    }
  }
};

// Triangle counting (the second CSR workload): parent = vertex u of an
// acyclic orientation of an undirected graph (sorted out-lists N+), child
// item i = out-edge u -> v, which counts the w in both N+(u) and N+(v); every
// triangle is counted once, at its edge from the lowest to the middle vertex
// of the orientation. The shorter list is walked and each of its entries is
// searched for in the longer one. Counts go to kTcSlots spread partial sums.
constexpr int kTcSlots = 256;

__device__ __forceinline__ bool sorted_contains(const int* a, int n, int key) {
  int lo = 0, hi = n;   // first index with a[i] >= key
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(&a[mid]) < key) lo = mid + 1;
    else hi = mid;
  }
  return lo < n && __ldg(&a[lo]) == key;
}

// |A ∩ B| of two strictly increasing lists by a blocked merge: per step four
// entries of each list, all 16 pairs compared, then the block with the smaller
// maximum moves on (both when the maxima are equal). No pair of blocks is
// compared twice, and a block is left only when nothing after the other list's
// current block can equal one of its entries, so each common entry is counted
// once. Entries past a list's end read as INT_MAX in A and INT_MAX - 1 in B,
// which match neither each other nor a vertex id. The loop's dependent chain
// is (na + nb) / 4 loads of consecutive entries (mostly L1 hits), against
// min(na, nb) binary searches of log2(max) probes each.
__device__ __forceinline__ unsigned intersect_merge4(const int* A, int na, const int* B, int nb) {
  unsigned c = 0;
  int i = 0, j = 0;
  while (i < na && j < nb) {
    int a[4], bb[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      a[q] = i + q < na ? __ldg(&A[i + q]) : INT_MAX;
      bb[q] = j + q < nb ? __ldg(&B[j + q]) : INT_MAX - 1;
    }
#pragma unroll
    for (int p = 0; p < 4; p++)
#pragma unroll
      for (int q = 0; q < 4; q++) c += a[p] == bb[q] ? 1u : 0u;
    const int amax = a[3], bmax = bb[3];
    if (amax <= bmax) i += 4;
    if (bmax <= amax) j += 4;
  }
  return c;
}

struct TcBody {
  static constexpr bool kOffsets = false;
  static constexpr bool kPushes = false;
  static constexpr bool kBalance = true;    // block cost varies with the lists' lengths
  static constexpr int kStage = 0;
  struct P {
    int base;
    int n;
  };
  struct F {
    int v;
  };
  __device__ static void count(const Args& a, int pid, int& base, int& N) {
    base = __ldg(&a.row_ptr[pid]);
    N = __ldg(&a.row_ptr[pid + 1]) - base;
  }
  __device__ static P parent(const BodyArgs&, int, int base, int N) { return P{base, N}; }
  __device__ static P shfl(const P& p, int src) {
    return P{__shfl_sync(kFull, p.base, src), __shfl_sync(kFull, p.n, src)};
  }
  __device__ static F fetch(const BodyArgs& b, const P& p, int i) { return F{__ldg(&b.col[p.base + i])}; }
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&p)[K], const int (&)[K], const F (&f)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
    int vb[K], vn[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      push[k] = false;
      v[k] = 0;
      vb[k] = valid[k] ? __ldg(&b.row_ptr[f[k].v]) : 0;
      vn[k] = valid[k] ? __ldg(&b.row_ptr[f[k].v + 1]) - vb[k] : 0;
    }
    unsigned c = 0;
#pragma unroll
    for (int k = 0; k < K; k++) {
      const int* nu = b.col + p[k].base;
      const int* nv = b.col + vb[k];
      const bool walk_u = p[k].n <= vn[k];
      const int* walk = walk_u ? nu : nv;
      const int* look = walk_u ? nv : nu;
      const int nw = walk_u ? p[k].n : vn[k], nl = walk_u ? vn[k] : p[k].n;
      if (NP_TC_MERGE && nl <= 16 * nw) {
        c += intersect_merge4(walk, nw, look, nl);   // lists of comparable length
      } else {
        for (int t = 0; t < nw; t++) c += sorted_contains(look, nl, __ldg(&walk[t])) ? 1u : 0u;
      }
    }
    if (c) atomicAdd(&b.acc[blockIdx.x & (kTcSlots - 1)], (unsigned long long)c);
  }
};

// SSSP with the distance and the append tag in one 64-bit word per vertex:
// dtag[v] = dist(v) << 32 | t(v), where t(v) = L + 1 of the last iteration
// that lowered dist(v) (0 before any). One 64-bit atomicMin of
// (nd << 32 | L + 1) both relaxes and decides the append: v joins the next
// frontier iff nd was strictly below the old distance and the old tag was not
// L + 1 (the first strict improvement of v in this iteration). An equal
// distance keeps the older, smaller tag, so a later strict improvement in the
// same iteration still sees whether v was appended. This saves the stamp
// exchange, one dependent L2 round trip per improving batch.
struct Sssp64Body {
  static constexpr bool kOffsets = false;
  static constexpr bool kPushes = true;
  static constexpr bool kBalance = false;
  static constexpr int kStage = 2;          // col and w
  struct P {
    int base;
    unsigned du;
    int qbase;
  };
  struct F {
    int v;
    unsigned w;
  };
  __device__ static void count(const Args& a, int pid, int& base, int& N) {
    const int u = pid & a.b.vmask;
    base = __ldg(&a.row_ptr[u]);
    N = __ldg(&a.row_ptr[u + 1]) - base;
  }
  __device__ static P parent(const BodyArgs& b, int pid, int base, int) {
    return P{base, (unsigned)(__ldcg(&b.dtag[pid]) >> 32), pid & ~b.vmask};
  }
  __device__ static F fetch(const BodyArgs& b, const P& p, int i) {
    return F{p.qbase | __ldg(&b.col[p.base + i]), __ldg(&b.w[p.base + i])};
  }
  __device__ static F fetch_from(const P& p, int col, unsigned w) { return F{p.qbase | col, w}; }
  __device__ static P shfl(const P& p, int src) {
    return P{__shfl_sync(kFull, p.base, src), (unsigned)__shfl_sync(kFull, (int)p.du, src),
             __shfl_sync(kFull, p.qbase, src)};
  }
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&p)[K], const int (&)[K], const F (&f)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
    const unsigned tag = (unsigned)(b.L + 1);
    unsigned long long nd[K], cur[K];
    bool live[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      v[k] = f[k].v;
      live[k] = p[k].du != 0xffffffffu;
      const unsigned long long s = (unsigned long long)p[k].du + f[k].w;
      nd[k] = ((s >= 0xffffffffull ? 0xfffffffeull : s) << 32) | tag;
#if NP_SSSP_PRECHECK
      cur[k] = (valid[k] && live[k]) ? NP_FILTER_LOAD(&b.dtag[v[k]]) : 0ull;
#else
      cur[k] = 0xffffffffffffffffull;
#endif
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      push[k] = valid[k] && live[k] && (nd[k] >> 32) < (cur[k] >> 32);
      if (push[k]) cur[k] = atomicMin(&b.dtag[v[k]], nd[k]);
    }
#pragma unroll
    for (int k = 0; k < K; k++)
      push[k] = push[k] && (nd[k] >> 32) < (cur[k] >> 32) && (unsigned)cur[k] != tag;
  }
};

// BT (Section VII): parent = quadratic curve; child item j = point j.
struct BezierBody {
  static constexpr bool kOffsets = true;
  static constexpr bool kPushes = false;
  static constexpr bool kBalance = false;
  static constexpr int kStage = 0;
  struct P {
    float x0, y0, x1, y1, x2, y2;
    int base;
    float denom;
  };
  struct F {};
  // Point count in FP64 with correctly rounded operations only, so that it is
  // bit-identical to a serial FP64 evaluation (no contraction into FMA).
  __device__ static int point_count_fp64(const float* p) {
    const double x0 = p[0], y0 = p[1], x1 = p[2], y1 = p[3], x2 = p[4], y2 = p[5];
    const double sx = __dadd_rn(__dsub_rn(x0, __dmul_rn(2.0, x1)), x2);
    const double sy = __dadd_rn(__dsub_rn(y0, __dmul_rn(2.0, y1)), y2);
    const double cx = __dsub_rn(x2, x0), cy = __dsub_rn(y2, y0);
    const double s2 = __dadd_rn(__dmul_rn(sx, sx), __dmul_rn(sy, sy));
    const double c2 = __dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy));
    if (c2 == 0.0) return s2 > 0.0 ? 4096 : 4;
    const double kappa = __ddiv_rn(__dsqrt_rn(s2), __dsqrt_rn(c2));
    const double t = ceil(__dmul_rn(__dsqrt_rn(kappa), 64.0));
    if (t < 4.0) return 4;
    if (t > 4096.0) return 4096;
    return (int)t;
  }
  // The same count without FP64 arithmetic where that is provably the same
  // number (FP64 throughput is low on this GPU). When every coordinate is
  // k * 2^-24 with 0 <= k < 2^24, the FP64 second difference, chord and their
  // squared norms above are exact: s2 = S * 2^-48 and c2 = C * 2^-48 with
  // integers S < 2^53, C < 2^49. The exact t = 64 (S / C)^(1/4) then has
  // ceil(t) = the least m with m^4 C >= 2^24 S, found with 128-bit integers;
  // the FP64 evaluation carries a relative error below 3e-16 (four correctly
  // rounded operations), so it has the same ceiling unless t^4 lies within a
  // relative 2^-40 of m^4 or (m-1)^4, where the FP64 sequence itself decides.
  // Other inputs also take the FP64 sequence.
  __device__ static int point_count(const float* p) {
    unsigned k[6];
#pragma unroll
    for (int i = 0; i < 6; i++) {
      const float f = p[i] * 16777216.0f;   // exact: a power-of-two scale
      if (!(f >= 0.0f && f < 16777216.0f && f == truncf(f))) return point_count_fp64(p);
      k[i] = (unsigned)f;
    }
    const long long sx = (long long)k[0] - 2ll * k[2] + k[4], sy = (long long)k[1] - 2ll * k[3] + k[5];
    const long long cx = (long long)k[4] - k[0], cy = (long long)k[5] - k[1];
    const unsigned long long S = (unsigned long long)(sx * sx) + (unsigned long long)(sy * sy);
    const unsigned long long C = (unsigned long long)(cx * cx) + (unsigned long long)(cy * cy);
    if (C == 0) return S > 0 ? 4096 : 4;
    if (S == 0) return 4;                                   // t = 0 exactly, in FP64 too
    using u128 = unsigned __int128;
    const u128 A = (u128)S << 24;                          // t^4 * C
    auto q4 = [&](unsigned long long m) -> u128 { const u128 m2 = (u128)(m * m); return m2 * m2 * C; };
    if (A > q4(4097)) return 4096;                          // t > 4097: clamped, far from any tie
    // estimate, then the exact ceiling by at most a few integer steps
    unsigned long long m = (unsigned long long)ceilf(64.0f * sqrtf(sqrtf((float)S / (float)C)));
    if (m < 1) m = 1;
    if (m > 4097) m = 4097;
    for (int it = 0; it < 8 && m > 1 && A <= q4(m - 1); it++) m--;
    for (int it = 0; it < 8 && A > q4(m); it++) m++;
    const u128 hi = q4(m), lo = q4(m - 1);
    const bool exact_m = A <= hi && A > lo;
    const bool near = (hi - A) <= (hi >> 40) || (m > 1 && (A - lo) <= (lo >> 40));
    if (!exact_m || near) return point_count_fp64(p);
    return m < 4 ? 4 : (m > 4096 ? 4096 : (int)m);
  }
  __device__ static void count(const Args& a, int pid, int& base, int& N) {
    base = 0;
    N = point_count(a.b.ctrl + 6 * (size_t)pid);
  }
  __device__ static P parent(const BodyArgs& b, int pid, int base, int N) {
    const float* c = b.ctrl + 6 * (size_t)pid;
    return P{__ldg(c), __ldg(c + 1), __ldg(c + 2), __ldg(c + 3), __ldg(c + 4), __ldg(c + 5), base,
             (float)(N - 1)};
  }
  __device__ static P shfl(const P& p, int src) {
    return P{__shfl_sync(kFull, p.x0, src), __shfl_sync(kFull, p.y0, src), __shfl_sync(kFull, p.x1, src),
             __shfl_sync(kFull, p.y1, src), __shfl_sync(kFull, p.x2, src), __shfl_sync(kFull, p.y2, src),
             __shfl_sync(kFull, p.base, src), __shfl_sync(kFull, p.denom, src)};
  }
  __device__ static F fetch(const BodyArgs&, const P&, int) { return F{}; }
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&p)[K], const int (&idx)[K], const F (&)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
#pragma unroll
    for (int k = 0; k < K; k++) {
      push[k] = false;
      v[k] = 0;
      if (!valid[k]) continue;
      const P& q = p[k];
      const float t = (float)idx[k] / q.denom;
      const float u = 1.0f - t;
      const float b0 = u * u, b1 = 2.0f * u * t, b2 = t * t;
      b.points[q.base + idx[k]] =
          make_float2(b0 * q.x0 + b1 * q.x1 + b2 * q.x2, b0 * q.y0 + b1 * q.y1 + b2 * q.y2);
    }
  }
};

// --------------------------------------------------------------- child side

// One coarsened child block: CF consecutive original blocks of one parent
// (Section IV-B; contiguous original blocks), in batches of up to 8 original
// blocks whose items are all loaded before any is applied.
template <class Body, int CF, class Sink>
__device__ __forceinline__ void run_coarsened(const BodyArgs& b, const typename Body::P& p, int N, int cb, int B,
                                              int tid, Sink& sink) {
  constexpr int KB = CF < NP_CHILD_BATCH ? CF : NP_CHILD_BATCH;
#pragma unroll
  for (int k0 = 0; k0 < CF; k0 += KB) {
    if ((cb * CF + k0) * B >= N) break;   // uniform across the block
    typename Body::F f[KB];
    bool v[KB];
    int idx[KB];
#pragma unroll
    for (int k = 0; k < KB; k++) {
      idx[k] = (cb * CF + k0 + k) * B + tid;
      v[k] = idx[k] < N;
      f[k] = v[k] ? Body::fetch(b, p, idx[k]) : typename Body::F{};
    }
    bool pf[KB];
    int pv[KB];
    typename Body::P pk[KB];
#pragma unroll
    for (int k = 0; k < KB; k++) pk[k] = p;
    Body::template apply_batch<KB>(b, pk, idx, f, v, pf, pv);
    if constexpr (Body::kPushes) sink.template push<KB>(pf, pv);
  }
}

// Serial version of a parent's children (thresholding's fallback, the NODP
// form): the parent thread walks its children in order, four at a time.
template <class Body>
__device__ __forceinline__ void run_serial(const BodyArgs& b, int pid, int base, int N, CtaSink& sink) {
  constexpr int KS = NP_SERIAL_BATCH;
  const typename Body::P p = Body::parent(b, pid, base, N);
  for (int i0 = 0; i0 < N; i0 += KS) {
    typename Body::F f[KS];
    bool v[KS];
    int idx[KS];
#pragma unroll
    for (int k = 0; k < KS; k++) {
      idx[k] = i0 + k;
      v[k] = idx[k] < N;
      f[k] = v[k] ? Body::fetch(b, p, idx[k]) : typename Body::F{};
    }
    bool pf[KS];
    int pv[KS];
    typename Body::P pk[KS];
#pragma unroll
    for (int k = 0; k < KS; k++) pk[k] = p;
    Body::template apply_batch<KS>(b, pk, idx, f, v, pf, pv);
    if constexpr (Body::kPushes) sink.template push<KS>(pf, pv);
  }
}

__device__ __forceinline__ void add_stat(LevelState* st, int k, unsigned long long v) {
  if (v) atomicAdd(&st->s[k], v);
}

// Child grid of one parent (plain CDP, thresholded or coarsened launch).
template <class Body, int CF>
__global__ void NP_CHILD_BOUNDS child_direct(BodyArgs b, int pid, int base, int N) {
  const typename Body::P p = Body::parent(b, pid, base, N);
  WarpSink sink{b.next, b.next_count};
  run_coarsened<Body, CF>(b, p, N, blockIdx.x, blockDim.x, threadIdx.x, sink);
}

// Persistent aggregated child grid for bodies whose blocks differ widely in
// cost: each CTA takes the next blockDim.x / cb aggregated blocks from the
// level's ticket (one child block per sub-block) until none are left. A
// sub-block's blocks only move forward, so the parent search continues from
// the last record. Bodies without appends only (no staging).
template <class Body, int CF>
__device__ __forceinline__ void child_agg_balanced(const BodyArgs& b, const int4* rec, const int* boff, int nrec,
                                                   int total, int cb, int* ticket, int* s_next) {
  const int per_cta = (int)blockDim.x / cb;
  const int local = (int)threadIdx.x / cb, stid = (int)threadIdx.x % cb;
  int j = -1, next_off = 0, off = 0, N = 0, done = 0;
  typename Body::P p{};
  WarpSink sink{b.next, b.next_count};
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) *s_next = atomicAdd(ticket, per_cta);
    __syncthreads();
    const int first = *s_next;
    if (first >= total) break;
    const int B0 = first + local;
    if (B0 < total) {
      if (j < 0 || B0 >= next_off) {
        j = j < 0 ? warp_search(boff, 0, nrec, B0) : warp_search_near(boff, j + 1, nrec, B0);
        const int4 r = __ldcg(&rec[j]);
        off = __ldcg(&boff[j]);
        next_off = j + 1 < nrec ? __ldcg(&boff[j + 1]) : 0x7fffffff;
        N = r.z;
        p = Body::parent(b, r.x, r.y, r.z);
      }
      run_coarsened<Body, CF>(b, p, N, B0 - off, cb, stid, sink);
      done++;
    }
  }
  if (stid == 0 && done) add_stat(b.st, S_CBLOCKS, (unsigned long long)done);
}

// ------------------------------------------- TMA-staged aggregated child blocks
//
// The edge lists of an aggregated child block (cb * CF consecutive items of
// one parent) are contiguous, so one elected thread per child block copies
// them into shared memory with the bulk-copy engine (cp.async.bulk into an
// mbarrier), one block ahead: the copy of block B + 1 runs while block B does
// its distance loads and atomics, taking the edge-list round trip off each
// block's dependent chain. Only the 16-byte aligned interior of a block's
// range is copied (the copy engine needs 16-byte aligned addresses and sizes);
// the up to three items at either end are read directly. Every mbarrier wait
// is bounded in time.
constexpr int kTmaItems = 256;   // items of one staged child block at most (cb * CF)
constexpr int kTmaSubs = 8;      // staged child blocks per CTA at most
constexpr unsigned long long kTmaWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the phase with the given parity; gives up (timeout bit) after kTmaWaitNs.
__device__ __forceinline__ void mbar_wait(unsigned long long* bar, unsigned parity, LevelState* st) {
  if (mbar_try_wait(bar, parity)) return;
  const unsigned long long t0 = timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (timer_ns() - t0 > kTmaWaitNs) {
      atomicOr(&st->error, kErrTimeout);
      return;
    }
  }
}

template <class Body, int CF>
__device__ __forceinline__ void child_agg_staged(const BodyArgs& b, const int4* rec, const int* boff, int nrec,
                                                 int total, int cb, bool count_blocks, int* s_stage, int* s_stage_n,
                                                 int* s_stage_base) {
  __shared__ __align__(16) int s_col[kTmaSubs][kTmaItems];
  __shared__ __align__(16) unsigned s_w[kTmaSubs][kTmaItems];
  __shared__ __align__(8) unsigned long long s_bar[kTmaSubs];
  constexpr bool kW = Body::kStage == 2;
  if (threadIdx.x == 0) *s_stage_n = 0;
  const int per_cta = (int)blockDim.x / cb;
  const int local = (int)threadIdx.x / cb, stid = (int)threadIdx.x % cb;
  const int sub = (int)blockIdx.x * per_cta + local;
  const int chunk = ceil_div(total, (int)gridDim.x * per_cta);
  const int first = sub * chunk;
  const int last = min(total, first + chunk);
  const int span = cb * CF;
  unsigned long long* bar = &s_bar[local];
  if (stid == 0) mbar_init(bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  StageSink sink{b.next, b.next_count, s_stage, s_stage_n};
  auto sub_sync = [&]() {
    if (cb == 32)
      __syncwarp();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(1 + local), "r"(cb) : "memory");
  };
  // stage items [bl * span, min(N, (bl + 1) * span)) of a parent whose list starts at `base`
  auto stage = [&](int base, int N, int bl, int& a0, int& a1) -> bool {
    const int e0 = base + bl * span, e1 = base + min(N, (bl + 1) * span);
    a0 = (e0 + 3) & ~3;
    a1 = e1 & ~3;
    if (a1 <= a0) return false;
    if (stid == 0) {
      const unsigned bytes = (unsigned)(a1 - a0) * 4u;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, kW ? 2u * bytes : bytes);
      bulk_to_smem(&s_col[local][0], b.col + a0, bytes, bar);
      if constexpr (kW) bulk_to_smem(&s_w[local][0], b.w + a0, bytes, bar);
    }
    return true;
  };
  int j = -1, off = 0, next_off = 0, next2 = 0x7fffffff, N = 0, base = 0;
  int4 rn = make_int4(0, 0, 0, 0);
  typename Body::P p{};
  int ca0 = 0, ca1 = 0;
  bool cur = false;
  unsigned phase = 0;
  if (first < last) {
    j = warp_search(boff, 0, nrec, first);
    const int4 r = __ldcg(&rec[j]);
    off = __ldcg(&boff[j]);
    next_off = j + 1 < nrec ? __ldcg(&boff[j + 1]) : 0x7fffffff;
    N = r.z;
    base = r.y;
    p = Body::parent(b, r.x, r.y, r.z);
    if (j + 1 < nrec) rn = __ldcg(&rec[j + 1]);
    next2 = j + 2 < nrec ? __ldcg(&boff[j + 2]) : 0x7fffffff;
    cur = stage(base, N, first - off, ca0, ca1);
  }
  for (int B0 = first; B0 < last; B0++) {
    const int bl = B0 - off;
    if (cur) {
      mbar_wait(bar, phase, b.st);
      phase ^= 1u;
    }
    typename Body::F f[CF];
    bool v[CF];
    int idx[CF];
#pragma unroll
    for (int k = 0; k < CF; k++) {
      idx[k] = (bl * CF + k) * cb + stid;
      v[k] = idx[k] < N;
      const int e = base + idx[k];
      if (!v[k])
        f[k] = typename Body::F{};
      else if (cur && e >= ca0 && e < ca1)
        f[k] = Body::fetch_from(p, s_col[local][e - ca0], kW ? s_w[local][e - ca0] : 0u);
      else
        f[k] = Body::fetch(b, p, idx[k]);
    }
    sub_sync();   // the buffer is free again
    // the next block: same parent, or (blocks are contiguous and a launching
    // parent has at least one) parent j + 1; stage its lists now
    bool nxt = false;
    int na0 = 0, na1 = 0;
    if (B0 + 1 < last) {
      if (B0 + 1 < next_off)
        nxt = stage(base, N, bl + 1, na0, na1);
      else if (B0 + 1 < next2)
        nxt = stage(rn.y, rn.z, 0, na0, na1);
    }
    bool pf[CF];
    int pv[CF];
    typename Body::P pk[CF];
#pragma unroll
    for (int k = 0; k < CF; k++) pk[k] = p;
    Body::template apply_batch<CF>(b, pk, idx, f, v, pf, pv);
    if constexpr (Body::kPushes) sink.template push<CF>(pf, pv);
    if (B0 + 1 < last && B0 + 1 >= next_off) {
      int4 r;
      if (B0 + 1 < next2) {
        j++;
        r = rn;
        off = next_off;
        next_off = next2;
      } else {
        j = warp_search_near(boff, j + 1, nrec, B0 + 1);
        r = __ldcg(&rec[j]);
        off = __ldcg(&boff[j]);
        next_off = j + 1 < nrec ? __ldcg(&boff[j + 1]) : 0x7fffffff;
      }
      N = r.z;
      base = r.y;
      p = Body::parent(b, r.x, r.y, r.z);
      if (j + 1 < nrec) rn = __ldcg(&rec[j + 1]);
      next2 = j + 2 < nrec ? __ldcg(&boff[j + 2]) : 0x7fffffff;
    }
    cur = nxt;
    ca0 = na0;
    ca1 = na1;
  }
  if constexpr (Body::kPushes) stage_flush(s_stage, s_stage_n, b.next, b.next_count, s_stage_base);
  if (count_blocks && stid == 0 && last > first) add_stat(b.st, S_CBLOCKS, (unsigned long long)(last - first));
  __syncthreads();
  if (stid == 0) mbar_inval(bar);
}

// One coarsened block of 4 original blocks (cb threads, 4·cb edges of one
// parent) with 16-byte edge-list loads: thread t reads edges [a0 + 4t, a0 + 4t + 4)
// of the block's window, a0 = the block's first edge rounded down to a multiple
// of 4, with one int4 load per array when all four lie before the block's end
// (edges before the block's start are read and ignored; they belong to the
// list before it). A vector that straddles the end, and the up to three edges
// past a0 + 4·cb, are read one by one, so no load leaves [a0, end of block).
// Requires col (and w) 16-byte aligned.
template <class Body, class Sink>
__device__ __forceinline__ void run_coarsened_vec4(const BodyArgs& b, const typename Body::P& p, int base, int N,
                                                   int bl, int cb, int tid, Sink& sink) {
  constexpr bool kW = Body::kStage == 2;
  const int span = 4 * cb;
  const int e0 = base + bl * span;
  const int e1 = min(base + N, e0 + span);
  const int a0 = e0 & ~3;
  const int ea = a0 + 4 * tid;
  typename Body::F f[5];
  bool v[5];
  int idx[5];
  int c[4] = {0, 0, 0, 0};
  unsigned w[4] = {0u, 0u, 0u, 0u};
  if (ea + 4 <= e1) {
    const int4 c4 = __ldg(reinterpret_cast<const int4*>(b.col + ea));
    c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
    if constexpr (kW) {
      const uint4 w4 = __ldg(reinterpret_cast<const uint4*>(b.w + ea));
      w[0] = w4.x; w[1] = w4.y; w[2] = w4.z; w[3] = w4.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < 4; q++) {
      if (ea + q >= e0 && ea + q < e1) {
        c[q] = __ldg(&b.col[ea + q]);
        if constexpr (kW) w[q] = __ldg(&b.w[ea + q]);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const int e = ea + q;
    v[q] = e >= e0 && e < e1;
    idx[q] = e - base;
    f[q] = v[q] ? Body::fetch_from(p, c[q], w[q]) : typename Body::F{};
  }
  // the block's last edges past the aligned window
  const int et = a0 + span + tid;
  v[4] = tid < 3 && et < e1;
  idx[4] = et - base;
  f[4] = v[4] ? Body::fetch_from(p, __ldg(&b.col[et]), kW ? __ldg(&b.w[et]) : 0u) : typename Body::F{};
  bool pf[5];
  int pv[5];
  typename Body::P pk[5];
#pragma unroll
  for (int k = 0; k < 5; k++) pk[k] = p;
  Body::template apply_batch<5>(b, pk, idx, f, v, pf, pv);
  if constexpr (Body::kPushes) sink.template push<5>(pf, pv);
}

// Aggregated child blocks [0, total) of the records rec[0, nrec) with block
// offsets boff: disaggregation + coarsened body. A CTA hosts blockDim.x / cb
// child blocks of cb threads that run independently (no CTA barrier on this
// path). With fewer child blocks than aggregated blocks (the persistent
// grid-host forms, whose size is fixed before the total is known) each child
// block takes a contiguous range of aggregated blocks, so after the first
// search the parent index only moves forward.
template <class Body, int CF>
__device__ __forceinline__ void child_agg_run(const BodyArgs& b, const int4* rec, const int* boff, int nrec,
                                              int total, int cb, bool count_blocks, int* s_stage, int* s_stage_n,
                                              int* s_stage_base, int* ticket = nullptr) {
  if constexpr (Body::kBalance) {
    if (ticket) {
      child_agg_balanced<Body, CF>(b, rec, boff, nrec, total, cb, ticket, s_stage_n);
      return;
    }
  }
  if constexpr (NP_TMA_STAGE && Body::kStage > 0 && CF <= 8) {
    const bool aligned = (((unsigned long long)b.col | (Body::kStage == 2 ? (unsigned long long)b.w : 0ull)) & 15ull) == 0;
    if (aligned && cb * CF <= kTmaItems && (int)blockDim.x / cb <= kTmaSubs) {
      child_agg_staged<Body, CF>(b, rec, boff, nrec, total, cb, count_blocks, s_stage, s_stage_n, s_stage_base);
      return;
    }
  }
  if (threadIdx.x == 0) *s_stage_n = 0;
  const int per_cta = (int)blockDim.x / cb;
  const int sub = (int)blockIdx.x * per_cta + (int)threadIdx.x / cb, stid = (int)threadIdx.x % cb;
  const int chunk = ceil_div(total, (int)gridDim.x * per_cta);
  const int first = sub * chunk;
  const int last = min(total, first + chunk);
  int j = -1, next_off = 0, off = 0, N = 0, base = 0;
  // record j + 1 and the offset of record j + 2, loaded one record ahead
  int4 rn = make_int4(0, 0, 0, 0);
  int next2 = 0x7fffffff;
  typename Body::P p{};
  __syncthreads();
  StageSink sink{b.next, b.next_count, s_stage, s_stage_n};
  bool vec4 = false;
  if constexpr (NP_VEC4 && CF == 4 && Body::kStage > 0)
    vec4 = ((reinterpret_cast<unsigned long long>(b.col) |
             (Body::kStage == 2 ? reinterpret_cast<unsigned long long>(b.w) : 0ull)) & 15ull) == 0ull;
  for (int B0 = first; B0 < last; B0++) {
    if (j < 0 || B0 >= next_off) {
      int4 r;
      if (j >= 0 && B0 < next2) {
        // blocks are contiguous and a launching parent has at least one block,
        // so the next record is j + 1, already loaded
        j++;
        r = rn;
        off = next_off;
        next_off = next2;
      } else {
        j = j < 0 ? warp_search(boff, 0, nrec, B0) : warp_search_near(boff, j + 1, nrec, B0);
        r = __ldcg(&rec[j]);
        off = __ldcg(&boff[j]);
        next_off = j + 1 < nrec ? __ldcg(&boff[j + 1]) : 0x7fffffff;
      }
      N = r.z;
      base = r.y;
      p = Body::parent(b, r.x, r.y, r.z);
      if (j + 1 < nrec) rn = __ldcg(&rec[j + 1]);
      next2 = j + 2 < nrec ? __ldcg(&boff[j + 2]) : 0x7fffffff;
    }
    if constexpr (NP_VEC4 && CF == 4 && Body::kStage > 0) {
      if (vec4) {
        run_coarsened_vec4<Body>(b, p, base, N, B0 - off, cb, stid, sink);
        continue;
      }
    }
    run_coarsened<Body, CF>(b, p, N, B0 - off, cb, stid, sink);
  }
  if constexpr (Body::kPushes) stage_flush(s_stage, s_stage_n, b.next, b.next_count, s_stage_base);
  // persistent (grid-host) forms count their blocks here; device-launched
  // grids are counted by the launching parent
  if (count_blocks && stid == 0 && last > first) add_stat(b.st, S_CBLOCKS, (unsigned long long)(last - first));
}

// Totals of the grid-host aggregation of level L (look-back or atomic scan).
__device__ __forceinline__ void agg_totals(const LevelState* st, int L, int mode, int& nrec, int& total) {
  const int slot = L & 3;
  if (mode == 1) {
    nrec = __ldcg(&st->agg_records[slot]);
    total = __ldcg(&st->agg_blocks[slot]);
  } else {
    const unsigned long long acc = __ldcg(&st->agg_acc[slot]);
    nrec = (int)(acc >> 40);
    total = (int)(acc & ((1ull << 40) - 1));
  }
}

// Aggregated child grid: a device-launched grid over one segment (mode 0), or
// the stream-ordered persistent grid of the grid-host form, whose level and
// totals are read from the level state.
template <class Body, int CF>
__global__ void NP_CHILD_AGG_BOUNDS(CF) child_agg(BodyArgs b, AggSeg s) {
  NP_PDL_ENTRY();
  __shared__ int s_stage[kCtaStage];
  __shared__ int s_stage_n, s_stage_base;
  int nrec = s.nrec, total = s.total;
  if (s.mode != 0) {
    int L = b.L;
    if (s.level_mode) {
      L = __ldcg(&b.st->base) + s.k;
      b.L = L;
      b.next = (L & 1) ? s.fr0 : s.fr1;
      b.next_count = &b.st->count[(L + 1) % 3];
    }
    agg_totals(b.st, L, s.mode, nrec, total);
  }
  child_agg_run<Body, CF>(b, s.rec, s.boff, nrec, total, s.cb, s.mode != 0, s_stage, &s_stage_n, &s_stage_base,
                          s.mode != 0 ? &b.st->child_ticket[b.L & 3] : nullptr);
}

// --------------------------------------------------------------- parent side

template <class Body, int CF>
__device__ __forceinline__ void launch_direct(const BodyArgs& b, int pid, int base, int N, int child_block,
                                              unsigned* s_stat, CtaSink& sink) {
  const int cg = ceil_div(ceil_div(N, child_block), CF);
  child_direct<Body, CF><<<cg, child_block, 0, cudaStreamFireAndForget>>>(b, pid, base, N);
  if (cudaGetLastError() != cudaSuccess) {
    atomicOr(&b.st->error, kErrLaunch);
    atomicAdd(&s_stat[S_LFAIL], 1u);
    run_serial<Body>(b, pid, base, N, sink);
  } else {
    atomicAdd(&s_stat[S_DEVLAUNCH], 1u);
    atomicAdd(&s_stat[S_CBLOCKS], (unsigned)cg);
  }
}

template <class Body, int CF>
__device__ __forceinline__ void launch_aggregated(const BodyArgs& b, const int4* rec, const int* boff, int nrec,
                                                  int total, int child_block, unsigned* s_stat, CtaSink& sink) {
  AggSeg s{rec, boff, nullptr, nullptr, nrec, total, 0, 0, 0, child_block, 0};   // a fixed segment
  child_agg<Body, CF><<<total, child_block, 0, cudaStreamFireAndForget>>>(b, s);
  if (cudaGetLastError() != cudaSuccess) {
    // run the aggregated grid's work in this thread: parent by parent, serially
    atomicOr(&b.st->error, kErrLaunch);
    atomicAdd(&s_stat[S_LFAIL], 1u);
    for (int j = 0; j < nrec; j++) {
      const int4 r = __ldcg(&rec[j]);
      run_serial<Body>(b, r.x, r.y, r.z, sink);
    }
  } else {
    atomicAdd(&s_stat[S_DEVLAUNCH], 1u);
    atomicAdd(&s_stat[S_AGGGRID], 1u);
    atomicAdd(&s_stat[S_CBLOCKS], (unsigned)total);
  }
}

__device__ __forceinline__ void warp_stat(unsigned* s_stat, int k, unsigned v) {
  const unsigned t = __reduce_add_sync(kFull, v);
  if ((threadIdx.x & 31) == 0 && t) atomicAdd(&s_stat[k], t);
}

// The parent kernel of the device-launch forms (CTA tiles). GRAN selects the
// launch scope; CF is the coarsening factor of the child kernel it launches.
// GRAN == G_NODP compiles the same kernel with its launch code left out (every
// parent serialises): set against the G_NONE kernel with a threshold above
// every child count, the only difference is a launch site that never runs
// (the dead-launch-code effect of Section VII-D).
// Per tile: child counts, output offsets (Bezier), the launch decision, the
// aggregation scan, records and launch; the serial children of the parents
// below the threshold come last, so no scan ever waits behind a serial loop.
template <class Body, int GRAN, int CF>
__global__ void NP_PARENT_BOUNDS parent_kernel(Args a) {
  // launched early only as the No-CDP baseline (no launch site); the
  // device-launch forms complete with their children and are never
  if constexpr (GRAN == G_NODP) NP_PDL_ENTRY();
  __shared__ int s_tile;
  __shared__ uint2 s_scan[33];
  __shared__ V3 s_v3;
  __shared__ unsigned s_stat[S_N];
  __shared__ int s_q[kStageSlots];
  __shared__ int s_qn, s_qflush, s_qbase;
  const int tid = threadIdx.x, PB = blockDim.x, lane = tid & 31, warp = tid >> 5;
  LevelState* st = a.st;
  const bool fixed = a.count_fixed >= 0;
  int L = a.L_fixed, count = a.count_fixed;
  if (!fixed) level_of(st, a.k, L, count);
  const unsigned long long epoch = level_epoch(st, L);
  const int slot = L & 3;
  if (!fixed && blockIdx.x == 0 && tid == 0) level_open(st, L, count);
  if (count <= 0) return;
  const int* ids = fixed ? a.ids : ((L & 1) ? a.fr1 : a.fr0);
  BodyArgs b = a.b;
  b.L = L;
  b.next = fixed ? a.next_ovr : ((L & 1) ? a.fr0 : a.fr1);
  b.next_count = fixed ? a.next_count_ovr : &st->count[(L + 1) % 3];
  const int ntiles = ceil_div(count, PB);
  // CTAs beyond the number of tiles have nothing to take: leave at once
  if ((int)blockIdx.x >= ntiles) return;
  const int T = a.threshold < 1 ? 1 : a.threshold;
  const int CB = a.child_block;
  if (tid < S_N) s_stat[tid] = 0;
  CtaSink sink{b.next, b.next_count, s_q, &s_qn};
  __syncthreads();

  for (;;) {
    if (tid == 0) {
      s_tile = atomicAdd(&st->ticket[slot], 1);
      s_qn = 0;
    }
    __syncthreads();
    const int tile = s_tile;
    __syncthreads();
    if (tile >= ntiles) break;
    const int i = tile * PB + tid;
    int pid = 0, base = 0, N = 0;
    if (i < count) pid = ids ? __ldcg(&ids[i]) : i;
    const bool valid = i < count && pid >= 0;   // frontier slots padded with -1 hold no parent
    if (valid) Body::count(a, pid, base, N);
    if constexpr (Body::kOffsets) {
      // output offsets: exclusive scan of N over all parents, in parent order
      unsigned e0, e1, t0, t1;
      block_scan2((unsigned)N, 0u, e0, e1, t0, t1, s_scan);
      if (warp == 0) {
        V3 x = lookback(a.ob_flag, a.ob_agg, a.ob_incl, tile, 0, epoch, V3{t0, 0u, 0u}, st);
        if (lane == 0) s_v3 = x;
      }
      __syncthreads();
      const unsigned tile_base = s_v3.a;
      __syncthreads();
      base = (int)(tile_base + e0);
      if (valid) a.offsets[i] = base;
      if (tile == ntiles - 1 && tid == 0) a.offsets[count] = (int)(tile_base + t0);
      if (valid && (long long)base + N > a.cap) {
        atomicOr(&st->error, kErrCapacity);
        N = 0;
      }
    }
    const bool launch = GRAN != G_NODP && valid && N >= T;
    const bool serial = valid && !launch && N > 0;
    warp_stat(s_stat, S_PARENTS, valid ? 1u : 0u);
    warp_stat(s_stat, S_ITEMS, (unsigned)N);
    warp_stat(s_stat, S_SERIAL, serial ? 1u : 0u);
    if constexpr (GRAN != G_NODP) {
      warp_stat(s_stat, S_LAUNCHP, launch ? 1u : 0u);
      warp_stat(s_stat, S_CITEMS, launch ? (unsigned)N : 0u);
      const unsigned cg = launch ? (unsigned)ceil_div(ceil_div(N, CB), a.cfactor) : 0u;
      if constexpr (GRAN == G_NONE) {
        if (launch) launch_direct<Body, CF>(b, pid, base, N, CB, s_stat, sink);
      } else if constexpr (GRAN == G_WARP) {
        const unsigned m = __ballot_sync(kFull, launch);
        const int np = __popc(m);
        if (np > 0 && np < a.agg_threshold) {
          if (launch) launch_direct<Body, CF>(b, pid, base, N, CB, s_stat, sink);
        } else if (np > 0) {
          unsigned inc = cg;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            unsigned x = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += x;
          }
          const unsigned total = __shfl_sync(kFull, inc, 31);
          const int seg = tile * PB + warp * 32;
          const int slot = __popc(m & lanemask_lt());
          if (launch) {
            a.rec[seg + slot] = make_int4(pid, base, N, 0);
            a.boff[seg + slot] = (int)(inc - cg);
          }
          __threadfence();
          __syncwarp();
          if (lane == 31 - __clz(m))
            launch_aggregated<Body, CF>(b, a.rec + seg, a.boff + seg, np, (int)total, CB, s_stat, sink);
        }
      } else if constexpr (GRAN == G_BLOCK) {
        unsigned ea, eb, ta, tb;
        block_scan2(launch ? 1u : 0u, cg, ea, eb, ta, tb, s_scan);
        if ((int)ta < a.agg_threshold) {
          if (launch) launch_direct<Body, CF>(b, pid, base, N, CB, s_stat, sink);
        } else {
          const int seg = tile * PB;
          if (launch) {
            a.rec[seg + ea] = make_int4(pid, base, N, 0);
            a.boff[seg + ea] = (int)eb;
          }
          __threadfence();
          __syncthreads();
          if (tid == 0 && ta > 0) launch_aggregated<Body, CF>(b, a.rec + seg, a.boff + seg, (int)ta, (int)tb, CB, s_stat, sink);
        }
      } else {
        // multi-block / grid-device granularity: the scope is a group of G tiles
        const int G = a.group_blocks <= 0 ? ntiles : a.group_blocks;
        const int g = tile / G, first = g * G, gsize = min(G, ntiles - first);
        unsigned ea, eb, ta, tb;
        block_scan2(launch ? 1u : 0u, cg, ea, eb, ta, tb, s_scan);
        if (a.scan == 0) {
          if (warp == 0) {
            V3 x = lookback(a.lb_flag, a.lb_agg, a.lb_incl, tile, first, epoch, V3{ta, tb, 0u}, st);
            if (lane == 0) s_v3 = x;
          }
        } else if (tid == 0) {
          const unsigned long long old = atomicAdd(&a.grp_acc[g], ((unsigned long long)ta << 40) | tb);
          s_v3 = V3{(unsigned)(old >> 40), (unsigned)(old & ((1ull << 40) - 1)), 0u};
        }
        __syncthreads();
        const V3 x = s_v3;
        const int seg = first * PB;
        if (launch) {
          a.rec[seg + x.a + ea] = make_int4(pid, base, N, 0);
          a.boff[seg + x.a + ea] = (int)(x.b + eb);
        }
        {
          if (a.scan == 0 && tile == first + gsize - 1 && tid == 0) a.grp_total[g] = make_uint2(x.a + ta, x.b + tb);
          __threadfence();
          __syncthreads();
          if (tid == 0) {
            const int old = atomicAdd(&a.grp_ctr[g], 1);
            if (old == gsize - 1) {
              __threadfence();
              unsigned nrec, nblk;
              if (a.scan == 0) {
                const uint2 t = __ldcg(&a.grp_total[g]);
                nrec = t.x;
                nblk = t.y;
              } else {
                const unsigned long long t = atomicExch(&a.grp_acc[g], 0ull);
                nrec = (unsigned)(t >> 40);
                nblk = (unsigned)(t & ((1ull << 40) - 1));
              }
              a.grp_ctr[g] = 0;
              if (nrec > 0) launch_aggregated<Body, CF>(b, a.rec + seg, a.boff + seg, (int)nrec, (int)nblk, CB, s_stat, sink);
            }
          }
        }
      }
    }
    // serialised children last (thresholding's fallback)
    if (serial) run_serial<Body>(b, pid, base, N, sink);
    __syncthreads();
    if constexpr (Body::kPushes) {
      // flush the tile's staged appends: one atomic on the level counter
      if (tid == 0) {
        const int n = min(s_qn, kStageSlots);
        s_qflush = n;
        s_qbase = n > 0 ? atomicAdd(b.next_count, n) : 0;
      }
      __syncthreads();
      for (int k = tid; k < s_qflush; k += PB) b.next[s_qbase + k] = s_q[k];
    }
  }

  __syncthreads();
  if (tid < S_N && tid != S_LEVELS && tid != S_PUSHES) add_stat(st, tid, s_stat[tid]);
}

// ------------------------------------------------ parent side, warp tiles
//
// The parent kernel of the forms without device launches: no dynamic
// parallelism at all (FORM 0, every parent serialises its children) and
// grid-host aggregation (FORM 1: parents at or above the threshold are
// aggregated into the grid the next stream/graph node runs). Each warp takes
// 32-parent tiles from the level's ticket and works alone: a warp scan and a
// warp-level decoupled look-back over all tiles of the grid give the records'
// slots and block offsets, and the serialised children run in a warp-uniform
// loop (lanes with fewer children idle) that appends through a warp sink. No
// CTA barrier anywhere, so no warp waits for another warp's serial loop.
template <class Body, int FORM>
__device__ __forceinline__ void parent_warp_run(const Args& a, int L, int count, bool fixed, int* s_stage,
                                                int* s_stage_n, int* s_stage_base) {
  const int lane = threadIdx.x & 31;
  LevelState* st = a.st;
  const int slot = L & 3;
  const int ntiles = ceil_div(count, 32);
  // CTAs whose warps would all find no tile leave at once
  if ((int)blockIdx.x * ((int)blockDim.x >> 5) >= ntiles) return;
  if (threadIdx.x == 0) *s_stage_n = 0;
  __syncthreads();
  const unsigned long long epoch = level_epoch(st, L);
  const int* ids = fixed ? a.ids : ((L & 1) ? a.fr1 : a.fr0);
  BodyArgs b = a.b;
  b.L = L;
  b.next = fixed ? a.next_ovr : ((L & 1) ? a.fr0 : a.fr1);
  b.next_count = fixed ? a.next_count_ovr : &st->count[(L + 1) % 3];
  const int T = a.threshold < 1 ? 1 : a.threshold;
  const int CB = a.child_block;
  StageSink sink{b.next, b.next_count, s_stage, s_stage_n};
  unsigned long long n_par = 0, n_items = 0, n_serial = 0, n_launch = 0, n_citems = 0;

  // Without look-back waits (atomic aggregation scan, no output offsets) no
  // tile waits on another, so each warp's first tile is its own index and
  // only later tiles come from the ticket: small levels skip that round trip.
  // With look-back, tiles are taken strictly in ticket order (a wait only ever
  // targets a tile that a running warp holds).
  const bool static_first = a.scan != 0 && !Body::kOffsets;
  const int warps_total = (int)gridDim.x * ((int)blockDim.x >> 5);
  int own_tile = static_first ? (int)blockIdx.x * ((int)blockDim.x >> 5) + ((int)threadIdx.x >> 5) : -1;
  // Bodies with output offsets: the CTA's warps take consecutive tiles on one
  // ticket, combine their tile totals in shared memory, and one warp runs the
  // look-back for the CTA's group. All groups of a level start at once and each
  // walks back until a predecessor has its inclusive prefix, so the chain of
  // look-backs is as many times shorter as the CTA has warps, while every warp
  // still holds one tile. (Two CTA barriers per group; no other form has any.)
  __shared__ unsigned s_off[33];
  __shared__ int s_grp;
  const int nw = (int)blockDim.x >> 5, wid = (int)threadIdx.x >> 5;
  for (;;) {
    int tile = own_tile, grp = 0;
    if constexpr (Body::kOffsets) {
      __syncthreads();   // the previous group's shared words are consumed
      if (threadIdx.x == 0) s_grp = atomicAdd(&st->ticket[slot], 1);
      __syncthreads();
      grp = s_grp;
      if (grp * nw >= ntiles) break;   // uniform over the CTA
      tile = grp * nw + wid;
    } else {
      if (tile < 0) {
        if (lane == 0) tile = atomicAdd(&st->ticket[slot], 1) + (static_first ? warps_total : 0);
        tile = __shfl_sync(kFull, tile, 0);
      }
      own_tile = -1;   // later tiles come from the ticket
      if (tile >= ntiles) break;
    }
    const int i = tile * 32 + lane;
    int pid = 0, base = 0, N = 0;
    if (i < count) pid = ids ? __ldcg(&ids[i]) : i;
    const bool valid = i < count && pid >= 0;   // frontier slots padded with -1 hold no parent
    if (valid) Body::count(a, pid, base, N);
    if constexpr (Body::kOffsets) {
      // output offsets: exclusive scan of N over all parents, in parent order
      int inc = N;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += x;
      }
      if (lane == 31) s_off[wid] = (unsigned)inc;
      __syncthreads();
      if (wid == 0) {
        const unsigned t = lane < nw ? s_off[lane] : 0u;
        unsigned tin = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned x = __shfl_up_sync(kFull, tin, o);
          if (lane >= o) tin += x;
        }
        const unsigned gtot = __shfl_sync(kFull, tin, 31);
        const V3 x = lookback(a.ob_flag, a.ob_agg, a.ob_incl, grp, 0, epoch, V3{gtot, 0u, 0u}, st);
        if (lane < nw) s_off[lane] = x.a + tin - t;   // exclusive prefix of each warp's tile
        if (lane == 0) s_off[32] = x.a + gtot;
      }
      __syncthreads();
      base = (int)(s_off[wid] + (unsigned)(inc - N));
      if (valid) a.offsets[i] = base;
      if ((grp + 1) * nw >= ntiles && threadIdx.x == 0) a.offsets[count] = (int)s_off[32];
      if (valid && (long long)base + N > a.cap) {
        atomicOr(&st->error, kErrCapacity);
        N = 0;
      }
      if (tile >= ntiles) continue;   // past the level's last tile: only the scan above needed this warp
    }
    const bool launch = FORM == 1 && valid && N >= T;
    const bool serial = valid && !launch && N > 0;
    n_par += __popc(__ballot_sync(kFull, valid));
    n_items += __reduce_add_sync(kFull, (unsigned)N);
    n_serial += __popc(__ballot_sync(kFull, serial));
    if constexpr (FORM == 1) {
      const unsigned lm = __ballot_sync(kFull, launch);
      n_launch += __popc(lm);
      n_citems += __reduce_add_sync(kFull, launch ? (unsigned)N : 0u);
      const unsigned cg = launch ? (unsigned)ceil_div(ceil_div(N, CB), a.cfactor) : 0u;
      unsigned inc = cg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned x = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += x;
      }
      const unsigned ta = __popc(lm), tb = __shfl_sync(kFull, inc, 31);
      const unsigned ea = __popc(lm & lanemask_lt()), eb = inc - cg;
      V3 x{0u, 0u, 0u};
      if (a.scan == 0) {
        x = lookback(a.lb_flag, a.lb_agg, a.lb_incl, tile, 0, epoch, V3{ta, tb, 0u}, st);
      } else if (ta > 0) {
        // (a tile without launching parents needs no slots: no atomic round trip)
        unsigned long long old = 0ull;
        if (lane == 0) old = atomicAdd(&st->agg_acc[slot], ((unsigned long long)ta << 40) | tb);
        old = __shfl_sync(kFull, old, 0);
        x = V3{(unsigned)(old >> 40), (unsigned)(old & ((1ull << 40) - 1)), 0u};
      }
      if (launch) {
        a.rec[x.a + ea] = make_int4(pid, base, N, 0);
        a.boff[x.a + ea] = (int)(x.b + eb);
      }
      if (a.scan == 0 && tile == ntiles - 1 && lane == 0) {
        st->agg_records[slot] = (int)(x.a + ta);
        st->agg_blocks[slot] = (int)(x.b + tb);
      }
    }
    const int myN = serial ? N : 0;
    if constexpr (FORM == 1) {
      // Serialised children of the aggregated form, spread over the warp's
      // lanes: the tile's below-threshold children are numbered in parent
      // order, item t goes to lane t % 32, which finds its parent (the first
      // lane whose inclusive count exceeds t) by a shuffle search and takes
      // the parent's fields by shuffle. The work stays in the parent kernel,
      // with every lane busy instead of each lane walking only its own list.
      int incl = myN;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += x;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      if (total > 0) {
        constexpr int KS = NP_SPREAD_BATCH;
        const typename Body::P pm = Body::parent(b, serial ? pid : 0, base, N);
        const int excl = incl - myN;
        for (int t0 = 0; t0 < total; t0 += 32 * KS) {
          typename Body::F f[KS];
          typename Body::P pk[KS];
          bool v[KS];
          int idx[KS];
#pragma unroll
          for (int k = 0; k < KS; k++) {
            const int t = t0 + k * 32 + lane;
            int j = 0;
#pragma unroll
            for (int s2 = 16; s2 > 0; s2 >>= 1) {
              const int x = __shfl_sync(kFull, incl, j + s2 - 1);
              if (x <= t) j += s2;
            }
            j = j > 31 ? 31 : j;
            v[k] = t < total;
            idx[k] = t - __shfl_sync(kFull, excl, j);
            pk[k] = Body::shfl(pm, j);
            f[k] = v[k] ? Body::fetch(b, pk[k], idx[k]) : typename Body::F{};
          }
          bool pf[KS];
          int pv[KS];
          Body::template apply_batch<KS>(b, pk, idx, f, v, pf, pv);
          if constexpr (Body::kPushes) sink.template push<KS>(pf, pv);
        }
      }
    } else {
      // No-CDP form (the paper's baseline): lane l walks its own parent's
      // children in order; lanes with fewer (or none) idle through the tail
      const int maxN = (int)__reduce_max_sync(kFull, (unsigned)myN);
      if (maxN > 0) {
        constexpr int KS = NP_SERIAL_BATCH;
        const typename Body::P p = Body::parent(b, valid ? pid : 0, base, N);
        typename Body::P pk[KS];
#pragma unroll
        for (int k = 0; k < KS; k++) pk[k] = p;
        for (int i0 = 0; i0 < maxN; i0 += KS) {
          typename Body::F f[KS];
          bool v[KS];
          int idx[KS];
#pragma unroll
          for (int k = 0; k < KS; k++) {
            idx[k] = i0 + k;
            v[k] = idx[k] < myN;
            f[k] = v[k] ? Body::fetch(b, p, idx[k]) : typename Body::F{};
          }
          bool pf[KS];
          int pv[KS];
          Body::template apply_batch<KS>(b, pk, idx, f, v, pf, pv);
          if constexpr (Body::kPushes) sink.template push<KS>(pf, pv);
        }
      }
    }
  }
  if constexpr (Body::kPushes) stage_flush(s_stage, s_stage_n, b.next, b.next_count, s_stage_base);
  if (lane == 0) {
    add_stat(st, S_PARENTS, n_par);
    add_stat(st, S_ITEMS, n_items);
    add_stat(st, S_SERIAL, n_serial);
    add_stat(st, S_LAUNCHP, n_launch);
    add_stat(st, S_CITEMS, n_citems);
  }
}

template <class Body, int FORM>
__global__ void NP_PARENT_BOUNDS parent_warp(Args a) {
  NP_PDL_ENTRY();
  __shared__ int s_stage[kCtaStage];
  __shared__ int s_stage_n, s_stage_base;
  LevelState* st = a.st;
  const bool fixed = a.count_fixed >= 0;
  int L = a.L_fixed, count = a.count_fixed;
  if (!fixed) level_of(st, a.k, L, count);
  if (!fixed && blockIdx.x == 0 && threadIdx.x == 0) level_open(st, L, count);
  if (count <= 0) return;   // uniform over the grid
  parent_warp_run<Body, FORM>(a, L, count, fixed, s_stage, &s_stage_n, &s_stage_base);
}

// ------------------------------------------------- persistent level loop
//
// The whole level loop of a form without device launches in one cooperative
// kernel (all CTAs co-resident): per level the warp-tiled parent phase, then
// (grid aggregation) a grid barrier and the aggregated child phase over the
// same CTAs, then a grid barrier before the next level. The barriers stand in
// for the kernel boundaries of the graph drivers; the level state, frontiers
// and records are the same. Every wait is bounded in time: a barrier that
// does not complete within kBarrierNs sets the timeout bit and every CTA
// leaves the loop.
constexpr unsigned long long kBarrierNs = 5000000000ull;   // 5 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Returns false (in every thread of the CTA) once any CTA has timed out.
__device__ __forceinline__ bool grid_barrier(LevelState* st, int* s_ok, unsigned long long limit_ns = kBarrierNs) {
  __syncthreads();
  if (threadIdx.x == 0) {
    bool ok = true;
    const unsigned gen = ld_acquire_u32(&st->bar_gen);
    __threadfence();
    if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
      st->bar_count = 0u;
      __threadfence();
      st_release_u32(&st->bar_gen, gen + 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      unsigned polls = 0;
      while (ld_acquire_u32(&st->bar_gen) == gen) {
        if ((++polls & 63u) == 0u) {
          if (globaltimer_ns() - t0 > limit_ns || (__ldcg(&st->error) & kErrTimeout)) {
            atomicOr(&st->error, kErrTimeout);
            ok = false;
            break;
          }
        }
        __nanosleep(64);
      }
    }
    *s_ok = ok && !(__ldcg(&st->error) & kErrTimeout);
  }
  __syncthreads();
  return *s_ok != 0;
}

template <class Body, int FORM, int CF>
__global__ void __launch_bounds__(1024) level_loop(Args a, int max_levels) {
  __shared__ int s_stage[kCtaStage];
  __shared__ int s_stage_n, s_stage_base, s_ok;
  LevelState* st = a.st;
  int L = __ldcg(&st->base);
  while (L < max_levels) {
    const int count = __ldcg(&st->count[L % 3]);
    if (count <= 0) break;   // uniform: every CTA reads it after the same barrier
    if (blockIdx.x == 0 && threadIdx.x == 0) level_open(st, L, count);
    parent_warp_run<Body, FORM>(a, L, count, false, s_stage, &s_stage_n, &s_stage_base);
    if constexpr (FORM == 1) {
      if (!grid_barrier(st, &s_ok)) break;
      BodyArgs b = a.b;
      b.L = L;
      b.next = (L & 1) ? a.fr0 : a.fr1;
      b.next_count = &st->count[(L + 1) % 3];
      int nrec = 0, total = 0;
      agg_totals(st, L, a.scan == 0 ? 1 : 2, nrec, total);
      child_agg_run<Body, CF>(b, a.rec, a.boff, nrec, total, a.child_block, true, s_stage, &s_stage_n,
                              &s_stage_base, &st->child_ticket[L & 3]);
    }
    if (!grid_barrier(st, &s_ok)) break;
    L++;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->base = L;
}

}  // namespace nestpar
