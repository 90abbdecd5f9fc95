// Constants, build options, the device-resident level state, the argument
// blocks of the kernels, and the synchronisation primitives (decoupled
// look-back, block scans) they share.
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
// Register cap of the warp-tiled parent (spread serial loop) of the graph
// bodies: at 80 it needs no spill and three 256-thread CTAs fit an SM instead
// of two. (Each body states its own cap, kWarpParentRegs.)
#ifndef NP_WARP_PARENT_MAXREG
#define NP_WARP_PARENT_MAXREG 80
#endif
// Register cap of the CTA-tiled grid-host parent: 48, five 256-thread CTAs per
// SM (the tessellation's 36-byte parents take 64, kCtaParentRegs).
#ifndef NP_CTA_PARENT_MAXREG
#define NP_CTA_PARENT_MAXREG 48
#endif

namespace nestpar {

constexpr int kMaxParentBlock = 512;
// Packed serial children: the child grid takes them in chunks of kPackItems
// items (a CTA stages the chunk's parent records in shared memory); a parent
// has fewer than kPackMaxT items, so it meets at most one chunk start.
constexpr int kPackItems = 1024;
constexpr int kPackMaxT = kPackItems;
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
  unsigned long long agg_acc[4]; // slot L % 4: grid-host totals, atomic scan (pair_word(parents, blocks))
  unsigned long long s[S_N];     // counters (np_stats)
  int body_iters;                // conditional-while iterations of this solve (bounded)
  int pad;
  int child_ticket[4];           // slot L % 4: next chunk of aggregated blocks (balanced bodies)
  unsigned bar_count;            // grid barrier of the persistent level loop: arrivals
  unsigned bar_gen;              // and generation
  // Packed serial children (grid-host form): per slot L % 4, the records and
  // items of the parents below the threshold, as the atomic scan's packed
  // accumulator (pair_word(records, items)) or the look-back scan's totals, and
  // the ticket of the child grid's item chunks.
  unsigned long long pack_acc[4];
  int pack_records[4];
  int pack_items[4];
  int pack_ticket[4];
  int pad2[4];
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
  st->pack_acc[s2] = 0ull;
  st->pack_records[s2] = 0;
  st->pack_items[s2] = 0;
  st->pack_ticket[s2] = 0;
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
  int sweep;                     // 1: this level's children reduce, the frontier sweep appends
  // 1: no filter read before a visit's or relaxation's atomic (the one-CTA
  // small-level loop: its atomics are few, and the read would only lengthen
  // each item's chain of round trips)
  int unfiltered;
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
  int pack;                      // 1: children below the threshold go packed to the child grid
  // packed serial children: one record {parent, row start or output offset,
  // N, first item} per parent below the threshold, and per chunk of
  // kPackItems items the record holding the chunk's first item
  int4* prec;
  int* pfirst;
  int small_parents;             // > 0: the while body's one-CTA loop runs levels of at most this many parents
  int n_vertices;                // swept frontier: state elements the sweep visits
  int sweep_parents;             // swept frontier: levels with at least this many parents sweep (0 = none)
  // swept frontier of a serving pool: the sweep skips the chunks of slots
  // that hold no query (slot = element >> sweep_lg, sweep_lg >= 11), or NULL
  int sweep_lg;
  const int* sweep_busy;
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
  int pack;                      // 1: also run the packed serial children (prec, pfirst)
  const int4* prec;
  const int* pfirst;
  int sweep_parents;             // level mode: levels with at least this many parents sweep (0 = none)
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

// The aggregation atomic adds two counters at once in one 64-bit word (the
// paper packs parents and blocks). Each gets 32 bits here: per level both stay
// below 2^31 (a level has fewer than 2^31 parents and, for the counters this
// word carries, fewer than 2^31 children or blocks), whereas a 24-bit parent
// field overflows in one level of a large batch group (tens of millions of
// parents below the threshold), and a wrapped count misplaces records.
__device__ __forceinline__ unsigned long long pair_word(unsigned hi, unsigned lo) {
  return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned pair_hi(unsigned long long w) { return (unsigned)(w >> 32); }
__device__ __forceinline__ unsigned pair_lo(unsigned long long w) { return (unsigned)(w & 0xffffffffull); }

// Up to four counters scanned together (records, blocks, and for packed
// serial children their records and items).
struct V4 {
  unsigned a, b, c, d;
};
__device__ __forceinline__ V4 v4add(V4 x, V4 y) { return V4{x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d}; }
__device__ __forceinline__ V4 warp_sum4(V4 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.a += __shfl_xor_sync(kFull, v.a, o);
    v.b += __shfl_xor_sync(kFull, v.b, o);
    v.c += __shfl_xor_sync(kFull, v.c, o);
    v.d += __shfl_xor_sync(kFull, v.d, o);
  }
  return v;
}

// Decoupled look-back (single-pass prefix scan over tiles): run by one full
// warp; returns the exclusive prefix of tile `tile` within [first, tile].
// Flags hold (epoch << 2) | status, status 1 = aggregate published,
// 2 = inclusive prefix published. Waits are bounded: on expiry the error word
// gets kErrTimeout and the wait is abandoned (result then wrong, never a hang).
__device__ inline V4 lookback(unsigned long long* flag, uint4* agg, uint4* incl, int tile, int first,
                       unsigned long long epoch, V4 mine, LevelState* st) {
  const int lane = threadIdx.x & 31;
  const unsigned long long fA = (epoch << 2) | 1ull, fP = (epoch << 2) | 2ull;
  if (tile == first) {
    if (lane == 0) {
      incl[tile] = make_uint4(mine.a, mine.b, mine.c, mine.d);
      st_release_u64(&flag[tile], fP);
    }
    return V4{0, 0, 0, 0};
  }
  if (lane == 0) {
    agg[tile] = make_uint4(mine.a, mine.b, mine.c, mine.d);
    st_release_u64(&flag[tile], fA);
  }
  V4 excl{0, 0, 0, 0};
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
    V4 v{0, 0, 0, 0};
    if (in && !timed_out) {
      uint4 x = __ldcg(isP ? &incl[idx] : &agg[idx]);
      v = V4{x.x, x.y, x.z, x.w};
    }
    const unsigned pm = __ballot_sync(kFull, isP);
    const int stop = pm ? __ffs(pm) - 1 : 31;
    if (lane > stop) v = V4{0, 0, 0, 0};
    excl = v4add(excl, warp_sum4(v));
    if (pm) break;
    j -= 32;
  }
  if (lane == 0) {
    V4 inc = v4add(excl, mine);
    incl[tile] = make_uint4(inc.a, inc.b, inc.c, inc.d);
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

// Exclusive scan of four counters over the CTA (one warp scan, one scan of the
// warp totals): returns this thread's exclusive values and the CTA totals (in
// all threads). Uses s[0..32].
__device__ __forceinline__ void block_scan4(uint4 v, uint4& ex, uint4& tot, uint4* s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint4 in = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned x0 = __shfl_up_sync(kFull, in.x, o), x1 = __shfl_up_sync(kFull, in.y, o);
    const unsigned x2 = __shfl_up_sync(kFull, in.z, o), x3 = __shfl_up_sync(kFull, in.w, o);
    if (lane >= o) {
      in.x += x0;
      in.y += x1;
      in.z += x2;
      in.w += x3;
    }
  }
  if (lane == 31) s[warp] = in;
  __syncthreads();
  if (warp == 0) {
    const uint4 t = lane < nw ? s[lane] : make_uint4(0u, 0u, 0u, 0u);
    uint4 x = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y0 = __shfl_up_sync(kFull, x.x, o), y1 = __shfl_up_sync(kFull, x.y, o);
      const unsigned y2 = __shfl_up_sync(kFull, x.z, o), y3 = __shfl_up_sync(kFull, x.w, o);
      if (lane >= o) {
        x.x += y0;
        x.y += y1;
        x.z += y2;
        x.w += y3;
      }
    }
    if (lane < nw) s[lane] = make_uint4(x.x - t.x, x.y - t.y, x.z - t.z, x.w - t.w);   // exclusive warp prefix
    if (lane == 31) s[32] = x;                                                          // CTA total
  }
  __syncthreads();
  const uint4 wp = s[warp];
  ex = make_uint4(wp.x + in.x - v.x, wp.y + in.y - v.y, wp.z + in.z - v.z, wp.w + in.w - v.w);
  tot = s[32];
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

}  // namespace nestpar
