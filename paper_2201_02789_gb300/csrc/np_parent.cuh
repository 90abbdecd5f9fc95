// Parent side: child counts, the threshold test, aggregation scans and
// launches (CTA-tiled parent kernel) and the warp-tiled parent of the forms
// without device launches.
#pragma once
#include "np_child.cuh"

namespace nestpar {

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
  AggSeg s{rec, boff, nullptr, nullptr, nrec, total, 0, 0, 0, child_block, 0, nullptr, nullptr, 0, 0};   // a fixed segment
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
  __shared__ V4 s_v4;
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
  // (INT32_MAX launches nothing, whatever N)
  const int T = a.threshold < 1 ? 1 : a.threshold;
  const bool never = a.threshold == INT_MAX;
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
        V4 x = lookback(a.ob_flag, a.ob_agg, a.ob_incl, tile, 0, epoch, V4{t0, 0u, 0u, 0u}, st);
        if (lane == 0) s_v4 = x;
      }
      __syncthreads();
      const unsigned tile_base = s_v4.a;
      __syncthreads();
      base = (int)(tile_base + e0);
      if (valid) a.offsets[i] = base;
      if (tile == ntiles - 1 && tid == 0) a.offsets[count] = (int)(tile_base + t0);
      if (valid && (long long)base + N > a.cap) {
        atomicOr(&st->error, kErrCapacity);
        N = 0;
      }
    }
    const bool launch = GRAN != G_NODP && valid && !never && N >= T;
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
            V4 x = lookback(a.lb_flag, a.lb_agg, a.lb_incl, tile, first, epoch, V4{ta, tb, 0u, 0u}, st);
            if (lane == 0) s_v4 = x;
          }
        } else if (tid == 0) {
          const unsigned long long old = atomicAdd(&a.grp_acc[g], pair_word(ta, tb));
          s_v4 = V4{pair_hi(old), pair_lo(old), 0u, 0u};
        }
        __syncthreads();
        const V4 x = s_v4;
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
                nrec = pair_hi(t);
                nblk = pair_lo(t);
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
  // the CTA's counters (np_stats), in shared memory: no registers held across the tile loop
  __shared__ unsigned long long s_cnt[5];
  if (threadIdx.x == 0) *s_stage_n = 0;
  if (threadIdx.x < 5) s_cnt[threadIdx.x] = 0ull;
  __syncthreads();
  const unsigned long long epoch = level_epoch(st, L);
  const int* ids = fixed ? a.ids : ((L & 1) ? a.fr1 : a.fr0);
  BodyArgs b = a.b;
  b.L = L;
  b.next = fixed ? a.next_ovr : ((L & 1) ? a.fr0 : a.fr1);
  b.next_count = fixed ? a.next_count_ovr : &st->count[(L + 1) % 3];
  b.sweep = !fixed && a.sweep_parents > 0 && count >= a.sweep_parents;
  // (INT32_MAX launches nothing, whatever N)
  const int T = a.threshold < 1 ? 1 : a.threshold;
  const bool never = a.threshold == INT_MAX;
  const int CB = a.child_block;
  StageSink sink{b.next, b.next_count, s_stage, s_stage_n};

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
        const V4 x = lookback(a.ob_flag, a.ob_agg, a.ob_incl, grp, 0, epoch, V4{gtot, 0u, 0u, 0u}, st);
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
    const bool launch = FORM == 1 && valid && !never && N >= T;
    const bool serial = valid && !launch && N > 0;
    {
      const unsigned c_par = __popc(__ballot_sync(kFull, valid)), c_items = __reduce_add_sync(kFull, (unsigned)N);
      const unsigned c_serial = __popc(__ballot_sync(kFull, serial));
      if (lane == 0) {
        atomicAdd(&s_cnt[0], (unsigned long long)c_par);
        atomicAdd(&s_cnt[1], (unsigned long long)c_items);
        atomicAdd(&s_cnt[2], (unsigned long long)c_serial);
      }
    }
    if constexpr (FORM == 1) {
      const unsigned lm = __ballot_sync(kFull, launch);
      {
        const unsigned c_citems = __reduce_add_sync(kFull, launch ? (unsigned)N : 0u);
        if (lane == 0 && lm) {
          atomicAdd(&s_cnt[3], (unsigned long long)__popc(lm));
          atomicAdd(&s_cnt[4], (unsigned long long)c_citems);
        }
      }
      const unsigned cg = launch ? (unsigned)ceil_div(ceil_div(N, CB), a.cfactor) : 0u;
      unsigned inc = cg;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned x = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += x;
      }
      const unsigned ta = __popc(lm), tb = __shfl_sync(kFull, inc, 31);
      const unsigned ea = __popc(lm & lanemask_lt()), eb = inc - cg;
      V4 x{0u, 0u, 0u, 0u};
      if (a.scan == 0) {
        x = lookback(a.lb_flag, a.lb_agg, a.lb_incl, tile, 0, epoch, V4{ta, tb, 0u, 0u}, st);
      } else if (ta > 0) {
        // (a tile without launching parents needs no slots: no atomic round trip)
        unsigned long long old = 0ull;
        if (lane == 0) old = atomicAdd(&st->agg_acc[slot], pair_word(ta, tb));
        old = __shfl_sync(kFull, old, 0);
        x = V4{pair_hi(old), pair_lo(old), 0u, 0u};
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
    if constexpr (FORM == 1) {
      // Serialised children of the aggregated form. The work stays in the
      // parent kernel, with every lane busy instead of each lane walking only
      // its own list.
      if (__ballot_sync(kFull, serial) == 0u) continue;   // (uniform) no serialised children in this tile
      const typename Body::P pm = Body::parent(b, serial ? pid : 0, base, N);
      // Bodies with kWarpLoop: a parent with at least 32 serialised children
      // runs them with the whole warp, one parent at a time: child j on lane
      // j % 32, coalesced, the parent's fields taken by shuffle once.
      const int wideN = Body::kWarpLoop && serial && N >= 32 ? N : 0;
      const int myN = serial && wideN == 0 ? N : 0;
      if constexpr (Body::kWarpLoop) {
        for (unsigned wm = __ballot_sync(kFull, wideN > 0); wm; wm &= wm - 1) {
          const int src = __ffs(wm) - 1;
          const int n = __shfl_sync(kFull, wideN, src);
          const typename Body::P p = Body::shfl(pm, src);
          for (int j0 = 0; j0 < n; j0 += 32) {
            typename Body::F f[1];
            typename Body::P pk[1] = {p};
            bool v[1] = {j0 + lane < n};
            int idx[1] = {j0 + lane};
            f[0] = v[0] ? Body::fetch(b, p, idx[0]) : typename Body::F{};
            bool pf[1];
            int pv[1];
            Body::template apply_batch<1>(b, pk, idx, f, v, pf, pv);
            if constexpr (Body::kPushes) sink.template push<1>(pf, pv);
          }
        }
      }
      // The others are spread over the warp's lanes: their children are
      // numbered in parent order, item t goes to lane t % 32, which finds its
      // parent (the first lane whose inclusive count exceeds t) by a shuffle
      // search and takes the parent's fields by shuffle.
      int incl = myN;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += x;
      }
      const int total = __shfl_sync(kFull, incl, 31);
      if (total > 0) {
        // (the tessellation's 36-byte parents take two items per lane)
        constexpr int KS = sizeof(typename Body::P) > 16 ? 2 : NP_SPREAD_BATCH;
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
      const int myN = serial ? N : 0;
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
  __syncthreads();
  if (threadIdx.x == 0) {
    add_stat(st, S_PARENTS, s_cnt[0]);
    add_stat(st, S_ITEMS, s_cnt[1]);
    add_stat(st, S_SERIAL, s_cnt[2]);
    add_stat(st, S_LAUNCHP, s_cnt[3]);
    add_stat(st, S_CITEMS, s_cnt[4]);
  }
}

// --------------------------------------- parent side, CTA-tiled grid-host
//
// The parent kernel of grid-host aggregation with CTA tiles. Per tile of
// blockDim.x parents: child counts, one CTA scan of four counters (launching
// parents, their coarsened blocks, parents below the threshold, their items),
// then the paper's packed 64-bit atomic per counter pair (or one decoupled
// look-back over the tiles, which keeps records in parent order):
//   N >= T     rec / boff, for the aggregated child grid;
//   0 < N < T  serialised children (Section III-A), in one of two ways:
//     a.pack == 0  they stay in this kernel, spread over the CTA: the tile's
//                  parents below the threshold are staged in shared memory
//                  ({parent, start, N, the value the body stages}, first item
//                  from the scan) and every thread takes items
//                  t = k * blockDim.x + tid, finds its parent by a binary
//                  search over the staged first items and runs the body on
//                  NP_CTA_SPREAD_BATCH items at once;
//     a.pack == 1  they go packed to the child grid: prec = {parent, start, N,
//                  first item} and pfirst[k] = that record when it holds item
//                  k * kPackItems (N < kPackItems: at most one chunk start).
// Capped at Body::kCtaParentRegs registers (48 for the graph bodies: five
// 256-thread CTAs per SM).
#ifndef NP_CTA_SPREAD_BATCH
#define NP_CTA_SPREAD_BATCH 4
#endif
template <class Body>
__global__ void __maxnreg__(Body::kCtaParentRegs) parent_cta(Args a) {
  NP_PDL_ENTRY();
  // items per thread per round of the CTA-wide serial loop (the tessellation's
  // 32-byte parent takes two)
  constexpr int KS = sizeof(typename Body::P) > 16 ? 2 : NP_CTA_SPREAD_BATCH;
  __shared__ int s_tile;
  __shared__ uint4 s_scan[33];
  __shared__ uint2 s_scan2[33];
  __shared__ V4 s_x;
  __shared__ int s_first[kMaxParentBlock];
  __shared__ int4 s_rec[kMaxParentBlock];
  __shared__ int s_stage[Body::kPushes ? kCtaStage : 1];
  __shared__ int s_stage_n, s_stage_base;
  const int tid = (int)threadIdx.x, PB = (int)blockDim.x, lane = tid & 31, warp = tid >> 5;
  LevelState* st = a.st;
  const bool fixed = a.count_fixed >= 0;
  int L = a.L_fixed, count = a.count_fixed;
  if (!fixed) level_of(st, a.k, L, count);
  if (!fixed && blockIdx.x == 0 && tid == 0) level_open(st, L, count);
  if (count <= 0) return;   // uniform over the grid
  const int ntiles = ceil_div(count, PB);
  if ((int)blockIdx.x >= ntiles) return;
  const unsigned long long epoch = level_epoch(st, L);
  const int slot = L & 3;
  const int* ids = fixed ? a.ids : ((L & 1) ? a.fr1 : a.fr0);
  BodyArgs b = a.b;
  b.L = L;
  b.next = fixed ? a.next_ovr : ((L & 1) ? a.fr0 : a.fr1);
  b.next_count = fixed ? a.next_count_ovr : &st->count[(L + 1) % 3];
  // (INT32_MAX launches nothing, whatever N)
  const int T = a.threshold < 1 ? 1 : a.threshold;
  const bool never = a.threshold == INT_MAX;
  const int CB = a.child_block;
  if (tid == 0) s_stage_n = 0;
  StageSink sink{b.next, b.next_count, s_stage, &s_stage_n};
  // Without look-back waits no tile waits on another, so a CTA's first tile is
  // its own index and only later tiles come from the ticket.
  const bool static_first = a.scan != 0 && !Body::kOffsets;
  int own = static_first ? (int)blockIdx.x : -1;
  unsigned n_par = 0, n_serial = 0, n_launch = 0;
  unsigned long long n_items = 0, n_citems = 0;
  for (;;) {
    int tile = own;
    if (tile < 0) {
      // s_tile is read before the next write: thread 0 rewrites it only after
      // the CTA barriers of this tile's scan
      if (tid == 0) s_tile = atomicAdd(&st->ticket[slot], 1) + (static_first ? (int)gridDim.x : 0);
      __syncthreads();
      tile = s_tile;
    }
    own = -1;
    if (tile >= ntiles) break;   // uniform over the CTA
    const int i = tile * PB + tid;
    int pid = 0, base = 0, N = 0;
    if (i < count) pid = ids ? __ldcg(&ids[i]) : i;
    const bool valid = i < count && pid >= 0;   // frontier slots padded with -1 hold no parent
    if (valid) Body::count(a, pid, base, N);
    if constexpr (Body::kOffsets) {
      // output offsets: exclusive scan of N over all parents, in parent order
      unsigned e0, e1, t0, t1;
      block_scan2((unsigned)N, 0u, e0, e1, t0, t1, s_scan2);
      if (warp == 0) {
        const V4 x = lookback(a.ob_flag, a.ob_agg, a.ob_incl, tile, 0, epoch, V4{t0, 0u, 0u, 0u}, st);
        if (lane == 0) s_x = x;
      }
      __syncthreads();
      const unsigned tile_base = s_x.a;
      __syncthreads();
      base = (int)(tile_base + e0);
      if (valid) a.offsets[i] = base;
      if (tile == ntiles - 1 && tid == 0) a.offsets[count] = (int)(tile_base + t0);
      if (valid && (long long)base + N > a.cap) {
        atomicOr(&st->error, kErrCapacity);
        N = 0;
      }
    }
    const bool launch = valid && !never && N >= T;
    const bool small = valid && !launch && N > 0;
    const unsigned cg = launch ? (unsigned)ceil_div(ceil_div(N, CB), a.cfactor) : 0u;
    uint4 ex, tot;
    block_scan4(make_uint4(launch ? 1u : 0u, cg, small ? 1u : 0u, small ? (unsigned)N : 0u), ex, tot, s_scan);
    // only packed children need places beyond this tile
    const V4 mine{tot.x, tot.y, a.pack ? tot.z : 0u, a.pack ? tot.w : 0u};
    if (a.scan == 0) {
      if (warp == 0) {
        const V4 x = lookback(a.lb_flag, a.lb_agg, a.lb_incl, tile, 0, epoch, mine, st);
        if (lane == 0) s_x = x;
      }
    } else if (tid == 0) {
      // (no atomic round trip for a counter pair the tile leaves at zero)
      unsigned long long o1 = 0ull, o2 = 0ull;
      if (mine.a) o1 = atomicAdd(&st->agg_acc[slot], pair_word(mine.a, mine.b));
      if (mine.c) o2 = atomicAdd(&st->pack_acc[slot], pair_word(mine.c, mine.d));
      s_x = V4{pair_hi(o1), pair_lo(o1), pair_hi(o2), pair_lo(o2)};
    }
    if (small && !a.pack) {
      s_first[ex.z] = (int)ex.w;
      s_rec[ex.z] = make_int4(pid, base, N, (int)Body::aux(b, pid));
    }
    __syncthreads();
    const V4 x = s_x;
    if (launch) {
      a.rec[x.a + ex.x] = make_int4(pid, base, N, 0);
      a.boff[x.a + ex.x] = (int)(x.b + ex.y);
    }
    if (small && a.pack) {
      const int j = (int)(x.c + ex.z);
      const int first = (int)(x.d + ex.w);
      a.prec[j] = make_int4(pid, base, N, first);
      const int k = ceil_div(first, kPackItems);   // the first chunk start at or after `first`
      if (k * kPackItems < first + N) a.pfirst[k] = j;
    }
    if (a.scan == 0 && tile == ntiles - 1 && tid == 0) {
      st->agg_records[slot] = (int)(x.a + tot.x);
      st->agg_blocks[slot] = (int)(x.b + tot.y);
      st->pack_records[slot] = (int)(x.c + mine.c);
      st->pack_items[slot] = (int)(x.d + mine.d);
    }
    n_par += valid ? 1u : 0u;
    n_items += (unsigned)N;
    n_serial += small ? 1u : 0u;
    n_launch += launch ? 1u : 0u;
    n_citems += launch ? (unsigned)N : 0u;
    if (!a.pack && tot.w > 0) {   // uniform over the CTA
      const int nr = (int)tot.z, items = (int)tot.w;
      int top = 1;   // the largest power of two <= nr: the search's first step
      while (top * 2 <= nr) top *= 2;
      for (int t0 = 0; t0 < items; t0 += KS * PB) {
        typename Body::F f[KS];
        typename Body::P pk[KS];
        bool v[KS];
        int idx[KS];
#pragma unroll
        for (int k = 0; k < KS; k++) {
          const int t = t0 + k * PB + tid;
          v[k] = t < items;
          // the last staged parent whose first item is <= t (s_first[0] = 0)
          int r = 0;
          for (int step = top; step > 0; step >>= 1)
            if (r + step < nr && s_first[r + step] <= t) r += step;
          const int4 q = s_rec[r];
          idx[k] = t - s_first[r];
          pk[k] = Body::parent_aux(b, q.x, q.y, q.z, (unsigned)q.w);
          f[k] = v[k] ? Body::fetch(b, pk[k], idx[k]) : typename Body::F{};
        }
        bool pf[KS];
        int pv[KS];
        Body::template apply_batch<KS>(b, pk, idx, f, v, pf, pv);
        if constexpr (Body::kPushes) sink.template push<KS>(pf, pv);
      }
    }
    // s_x, s_first and s_rec are rewritten only after the next tile's scan
    // barriers: no barrier here
  }
  if constexpr (Body::kPushes) stage_flush(s_stage, &s_stage_n, b.next, b.next_count, &s_stage_base);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n_par += __shfl_xor_sync(kFull, n_par, o);
    n_items += __shfl_xor_sync(kFull, n_items, o);
    n_serial += __shfl_xor_sync(kFull, n_serial, o);
    n_launch += __shfl_xor_sync(kFull, n_launch, o);
    n_citems += __shfl_xor_sync(kFull, n_citems, o);
  }
  if (lane == 0) {
    add_stat(st, S_PARENTS, n_par);
    add_stat(st, S_ITEMS, n_items);
    add_stat(st, S_SERIAL, n_serial);
    add_stat(st, S_LAUNCHP, n_launch);
    add_stat(st, S_CITEMS, n_citems);
  }
}

template <class Body, int FORM>
__global__ void __maxnreg__(Body::kWarpParentRegs) parent_warp(Args a) {
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

}  // namespace nestpar
