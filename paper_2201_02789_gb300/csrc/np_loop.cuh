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
