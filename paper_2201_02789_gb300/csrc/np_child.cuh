// Child side: coarsened child blocks, the serial fallback, device-launched
// child grids and the aggregated child grid (disaggregation).
#pragma once
#include "np_bodies.cuh"

namespace nestpar {

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
    nrec = (int)pair_hi(acc);
    total = (int)pair_lo(acc);
  }
}

// Totals of the packed serial children of level L (look-back or atomic scan).
__device__ __forceinline__ void pack_totals(const LevelState* st, int L, int mode, int& nrec, int& nitems) {
  const int slot = L & 3;
  if (mode == 1) {
    nrec = __ldcg(&st->pack_records[slot]);
    nitems = __ldcg(&st->pack_items[slot]);
  } else {
    const unsigned long long acc = __ldcg(&st->pack_acc[slot]);
    nrec = (int)pair_hi(acc);
    nitems = (int)pair_lo(acc);
  }
}

// Packed serial children: the items of the parents below the threshold,
// numbered in record order (record j holds items [first_j, first_j + N_j)),
// run by the CTAs of the aggregated child grid in chunks of kPackItems items
// taken from the level's pack ticket. Per chunk the CTA stages the records it
// covers in shared memory: records pfirst[c] .. pfirst[c + 1] (the record
// holding the next chunk's first item, or the last record), with their first
// items made chunk-relative and the one value each body needs of its parent
// (SSSP: dist(u), loaded once per record). Each thread then takes items
// t = k * blockDim.x + tid, finds the record holding t by a binary search over
// the staged first items (disaggregation in shared memory, Section II-B), and
// runs the body on KP items at once. Consecutive items of one record are
// consecutive edges, so the edge-list loads of a warp stay coalesced.
#ifndef NP_PACK_BATCH
#define NP_PACK_BATCH 4
#endif
template <class Body>
__device__ __forceinline__ void child_pack_run(const BodyArgs& b, const int4* prec, const int* pfirst, int nrec,
                                               int nitems, int* ticket, int* s_stage, int* s_stage_n,
                                               int* s_stage_base) {
  // (a parent of more than 16 bytes, the tessellation's control points, takes two per thread)
  constexpr int KP = sizeof(typename Body::P) > 16 ? 2 : NP_PACK_BATCH;
  __shared__ int s_chunk;
  __shared__ int s_first[kPackItems + 1];
  __shared__ int4 s_rec[kPackItems + 1];
  const int tid = (int)threadIdx.x, nt = (int)blockDim.x;
  __syncthreads();   // the previous phase has flushed its staged appends
  if (tid == 0) *s_stage_n = 0;
  StageSink sink{b.next, b.next_count, s_stage, s_stage_n};
  const int nchunks = ceil_div(nitems, kPackItems);
  for (;;) {
    if (tid == 0) s_chunk = atomicAdd(ticket, 1);
    __syncthreads();
    const int c = s_chunk;
    if (c >= nchunks) break;   // uniform over the CTA
    const int c0 = c * kPackItems;
    const int j0 = __ldcg(&pfirst[c]);
    const int j1 = c + 1 < nchunks ? __ldcg(&pfirst[c + 1]) : nrec - 1;
    const int nr = j1 - j0 + 1;   // <= kPackItems + 1: every record has at least one item
    for (int r = tid; r < nr; r += nt) {
      const int4 q = __ldcg(&prec[j0 + r]);
      s_first[r] = q.w - c0;
      s_rec[r] = make_int4(q.x, q.y, q.z, (int)Body::aux(b, q.x));
    }
    __syncthreads();
    const int here = min(kPackItems, nitems - c0);
    int top = 1;   // the largest power of two <= nr: the search's first step
    while (top * 2 <= nr) top *= 2;
    for (int t0 = 0; t0 < here; t0 += KP * nt) {
      typename Body::F f[KP];
      typename Body::P pk[KP];
      bool v[KP];
      int idx[KP];
#pragma unroll
      for (int k = 0; k < KP; k++) {
        const int t = t0 + k * nt + tid;
        v[k] = t < here;
        // the last staged record whose first item is <= t (s_first[0] <= 0 <= t)
        int r = 0;
        for (int step = top; step > 0; step >>= 1)
          if (r + step < nr && s_first[r + step] <= t) r += step;
        const int4 q = s_rec[r];
        idx[k] = t - s_first[r];
        pk[k] = Body::parent_aux(b, q.x, q.y, q.z, (unsigned)q.w);
        f[k] = v[k] ? Body::fetch(b, pk[k], idx[k]) : typename Body::F{};
      }
      bool pf[KP];
      int pv[KP];
      Body::template apply_batch<KP>(b, pk, idx, f, v, pf, pv);
      if constexpr (Body::kPushes) sink.template push<KP>(pf, pv);
    }
    __syncthreads();   // the staged records and the chunk word are free again
  }
  if constexpr (Body::kPushes) stage_flush(s_stage, s_stage_n, b.next, b.next_count, s_stage_base);
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
      int count = 0;
      level_of(b.st, s.k, L, count);
      b.L = L;
      b.next = (L & 1) ? s.fr0 : s.fr1;
      b.next_count = &b.st->count[(L + 1) % 3];
      b.sweep = s.sweep_parents > 0 && count >= s.sweep_parents;
    }
    agg_totals(b.st, L, s.mode, nrec, total);
  }
  child_agg_run<Body, CF>(b, s.rec, s.boff, nrec, total, s.cb, s.mode != 0, s_stage, &s_stage_n, &s_stage_base,
                          s.mode != 0 ? &b.st->child_ticket[b.L & 3] : nullptr);
}

}  // namespace nestpar

namespace nestpar {

// The persistent child grid of grid-host aggregation with packed serial
// children: the aggregated blocks of the launching parents (as child_agg),
// then chunks of the packed items of the parents below the threshold, which
// CTAs take from a ticket as they finish their blocks.
template <class Body, int CF>
__global__ void NP_CHILD_AGG_BOUNDS(CF) child_agg_pack(BodyArgs b, AggSeg s) {
  NP_PDL_ENTRY();
  __shared__ int s_stage[kCtaStage];
  __shared__ int s_stage_n, s_stage_base;
  int L = b.L;
  if (s.level_mode) {
    L = __ldcg(&b.st->base) + s.k;
    b.L = L;
    b.next = (L & 1) ? s.fr0 : s.fr1;
    b.next_count = &b.st->count[(L + 1) % 3];
  }
  int nrec = 0, total = 0, prec_n = 0, pitems = 0;
  agg_totals(b.st, L, s.mode, nrec, total);
  pack_totals(b.st, L, s.mode, prec_n, pitems);
  child_agg_run<Body, CF>(b, s.rec, s.boff, nrec, total, s.cb, true, s_stage, &s_stage_n, &s_stage_base,
                          &b.st->child_ticket[L & 3]);
  if (pitems > 0)
    child_pack_run<Body>(b, s.prec, s.pfirst, prec_n, pitems, &b.st->pack_ticket[L & 3], s_stage, &s_stage_n,
                         &s_stage_base);
}

}  // namespace nestpar
