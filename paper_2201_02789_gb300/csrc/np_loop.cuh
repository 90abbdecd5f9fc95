// The persistent cooperative level loop and its bounded grid barrier.
#pragma once
#include "np_parent.cuh"

namespace nestpar {

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

namespace nestpar {

// ---------------------------------------------------------- small-level loop
//
// A level with few parents and few children costs mostly fixed latency: two
// kernel boundaries and a dependent chain of L2 round trips in each grid.
// Under the conditional-while driver of the grid-host form this one-CTA kernel
// runs whole levels itself while the frontier holds at most a.small_parents
// (<= 2 * blockDim.x) parents with at most kSmallItems children in all: each
// thread takes two consecutive parents (count, row bounds), a CTA scan gives the
// items' offsets, the parents are staged in shared memory, and the CTA's threads take
// the items, each finding its parent by a binary search over the staged
// offsets; CTA barriers separate the levels. A level whose appends all fit
// the CTA's stage hands them to the next level in shared memory (and to the
// global frontier with plain stores). It keeps the level state as the
// parent and child grids do (slots and the count two levels ahead cleared,
// counts rotated), so the grids continue from the level where it stops: the
// first one too large, or an empty frontier. It runs once before the loop and
// at the end of every body in place of the condition kernel: it moves the base
// on by the body's K levels, runs what it can, and sets the loop's condition
// (iterations counted and capped only at the end of a body).
#ifndef NP_SMALL_ITEMS
#define NP_SMALL_ITEMS 16384
#endif
constexpr int kSmallItems = NP_SMALL_ITEMS;

template <class Body>
__global__ void __launch_bounds__(1024) level_small(Args a, cudaGraphConditionalHandle h, int K, int in_body) {
  NP_PDL_ENTRY();
  constexpr int KS = 4;
  constexpr int PPT = 2;   // parents per thread: thread t takes parents 2t and 2t + 1
  __shared__ int s_first[PPT * 1024];
  __shared__ int s_pid[PPT * 1024];
  __shared__ int s_base[PPT * 1024];
  __shared__ unsigned s_aux[PPT * 1024];
  __shared__ uint2 s_scan[33];
  __shared__ int s_stage[kCtaStage];
  __shared__ int s_stage_n, s_stage_base;
  LevelState* st = a.st;
  const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
  const int limit = a.small_parents < PPT * nt ? a.small_parents : PPT * nt;
  const int max_levels = __ldcg(&st->max_levels);
  const int L0 = __ldcg(&st->base) + K;
  int L = L0;
  unsigned long long n_par = 0, n_items = 0, n_serial = 0;
  // The level's frontier: from global memory at the first level; after a level
  // of this loop whose appends all fit the stage, from the stage itself (the
  // level's count in `staged`, -1 otherwise), so the next level starts without
  // a round trip for its count and ids.
  int staged = -1;
  for (;;) {
    // written before this kernel or by this CTA before the last barrier: the
    // same value in every thread
    const int count = staged >= 0 ? staged : __ldcg(&st->count[L % 3]);
    if (count <= 0 || count > limit || L >= max_levels) break;
    const int* ids = staged >= 0 ? s_stage : ((L & 1) ? a.fr1 : a.fr0);
    int pid[PPT], base[PPT], N[PPT];
    unsigned aux[PPT];
    bool valid[PPT];
    unsigned mine = 0;
    BodyArgs b = a.b;
    b.L = L;
    b.unfiltered = 1;
#pragma unroll
    for (int r = 0; r < PPT; r++) {
      const int i = PPT * tid + r;
      pid[r] = i < count ? (staged >= 0 ? ids[i] : __ldcg(&ids[i])) : 0;
      valid[r] = i < count && pid[r] >= 0;
      base[r] = 0;
      N[r] = 0;
      if (valid[r]) Body::count(a, pid[r], base[r], N[r]);
      // (the value a staged parent carries, loaded beside its row bounds)
      aux[r] = valid[r] ? Body::aux(b, pid[r]) : 0u;
      mine += (unsigned)N[r];
    }
    unsigned e0, e1, items, t1;
    block_scan2(mine, 0u, e0, e1, items, t1, s_scan);
    if (items > (unsigned)kSmallItems) break;   // uniform: the grids take this level
    if (tid == 0) {
      level_open(st, L, count);
      s_stage_n = 0;
    }
    b.next = (L & 1) ? a.fr0 : a.fr1;
    b.next_count = &st->count[(L + 1) % 3];
    {
      // parents without children keep a slot: the search takes the last parent
      // whose first item is <= t, which is the one holding t
      unsigned first = e0;
#pragma unroll
      for (int r = 0; r < PPT; r++) {
        const int i = PPT * tid + r;
        if (i < count) {
          s_first[i] = (int)first;
          s_pid[i] = pid[r];
          s_base[i] = base[r];
          s_aux[i] = aux[r];
        }
        first += (unsigned)N[r];
      }
    }
    __syncthreads();
    StageSink sink{b.next, b.next_count, s_stage, &s_stage_n};
    int top = 1;
    while (top * 2 <= count) top *= 2;
    for (int t0 = 0; t0 < (int)items; t0 += KS * nt) {
      typename Body::F f[KS];
      typename Body::P pk[KS];
      bool v[KS];
      int idx[KS];
#pragma unroll
      for (int k = 0; k < KS; k++) {
        const int t = t0 + k * nt + tid;
        v[k] = t < (int)items;
        int r = 0;
        for (int step = top; step > 0; step >>= 1)
          if (r + step < count && s_first[r + step] <= t) r += step;
        idx[k] = t - s_first[r];
        // (the level-loop bodies do not use N in parent_aux)
        pk[k] = Body::parent_aux(b, s_pid[r], s_base[r], 0, s_aux[r]);
        f[k] = v[k] ? Body::fetch(b, pk[k], idx[k]) : typename Body::F{};
      }
      bool pf[KS];
      int pv[KS];
      Body::template apply_batch<KS>(b, pk, idx, f, v, pf, pv);
      if constexpr (Body::kPushes) sink.template push<KS>(pf, pv);
    }
    // appends reach the next frontier and its count before the next level reads them
    if constexpr (Body::kPushes) {
      __syncthreads();
      const int total = s_stage_n;   // the level's appends, the ones beyond the stage included
      if (total <= kCtaStage) {
        // all in the stage: this CTA made every append to the next frontier,
        // so plain stores place them (for the grids, should they take over)
        // and the next level reads them from the stage
        for (int i = tid; i < total; i += nt) b.next[i] = s_stage[i];
        if (tid == 0) *b.next_count = total;
        staged = total;
      } else {
        // the stage overflowed (those appends reserved their slots at once):
        // reserve the stage's part and copy it out; the next level is too
        // large for this loop
        stage_flush(s_stage, &s_stage_n, b.next, b.next_count, &s_stage_base);
        staged = -1;
      }
    }
#pragma unroll
    for (int r = 0; r < PPT; r++) {
      n_par += valid[r] ? 1u : 0u;
      n_items += (unsigned)N[r];
      n_serial += N[r] > 0 ? 1u : 0u;
    }
    __syncthreads();
    L++;
  }
  if (L != L0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_par += __shfl_xor_sync(kFull, n_par, o);
      n_items += __shfl_xor_sync(kFull, n_items, o);
      n_serial += __shfl_xor_sync(kFull, n_serial, o);
    }
    if ((tid & 31) == 0) {
      add_stat(st, S_PARENTS, n_par);
      add_stat(st, S_ITEMS, n_items);
      add_stat(st, S_SERIAL, n_serial);
    }
  }
  if (tid == 0) {
    st->base = L;
    bool more = __ldcg(&st->count[L % 3]) > 0 && L < max_levels;
    if (in_body) {
      // the iteration cap turns a level loop that failed to terminate into an error
      const int it = ++st->body_iters;
      if (more && it > max_levels + 16) {
        st->error |= kErrTimeout;
        more = false;
      }
    }
    cudaGraphSetConditional(h, more ? 1u : 0u);
  }
}

}  // namespace nestpar

namespace nestpar {

// ------------------------------------------------------------- frontier sweep
//
// After level L of a swept-frontier form (children that only reduce, see
// BfsSweepBody, Sssp64SweepBody): the next frontier is every vertex the level
// reached, level[v] == L + 1 (BFS) or tag(v) == L + 1 (packed SSSP). Each CTA
// takes kSweepVertices consecutive vertices (coalesced loads of the state),
// scans its marks and reserves its part of the frontier with one atomic; ids
// stay in vertex order within a CTA's range up to the interleaving of its
// threads, which keeps the next level's row-bound loads close together.
constexpr int kSweepVertices = 2048;

template <int KIND>
__global__ void __launch_bounds__(256) frontier_sweep_kernel(Args a) {
  NP_PDL_ENTRY();
  constexpr int KV = kSweepVertices / 256;
  __shared__ uint2 s_scan[33];
  __shared__ int s_base;
  LevelState* st = a.st;
  int L = 0, count = 0;
  level_of(st, a.k, L, count);
  // level L did not run, or its children appended the frontier themselves
  if (count <= 0 || count < a.sweep_parents) return;
  const int n = a.n_vertices;
  const unsigned want = (unsigned)(L + 1);
  int* next = (L & 1) ? a.fr0 : a.fr1;
  int* next_count = &st->count[(L + 1) % 3];
  const int* busy = a.sweep_busy;
  // (64-bit range arithmetic: a multi-query state may come close to 2^31 elements)
  for (long long c0 = (long long)blockIdx.x * kSweepVertices; c0 < n; c0 += (long long)gridDim.x * kSweepVertices) {
    // a chunk lies in one slot; an idle slot's state holds no vertex of this level (uniform over the CTA)
    if (busy && !busy[c0 >> a.sweep_lg]) continue;
    bool mark[KV];
    unsigned mine = 0;
#pragma unroll
    for (int k = 0; k < KV; k++) {
      const long long v = c0 + k * 256 + (int)threadIdx.x;
      if (KIND == 0)
        mark[k] = v < n && (unsigned)__ldcg(&a.b.level[v]) == want;
      else
        mark[k] = v < n && (unsigned)__ldcg(&a.b.dtag[v]) == want;
      mine += mark[k] ? 1u : 0u;
    }
    unsigned ex, e1, tot, t1;
    block_scan2(mine, 0u, ex, e1, tot, t1, s_scan);
    if (tot == 0) continue;   // uniform over the CTA
    if (threadIdx.x == 0) s_base = atomicAdd(next_count, (int)tot);
    __syncthreads();
    int pos = s_base + (int)ex;
#pragma unroll
    for (int k = 0; k < KV; k++)
      if (mark[k]) next[pos++] = (int)(c0 + k * 256 + (int)threadIdx.x);   // < n <= INT_MAX
    __syncthreads();   // s_base is rewritten by the next range's reservation
  }
}

}  // namespace nestpar
