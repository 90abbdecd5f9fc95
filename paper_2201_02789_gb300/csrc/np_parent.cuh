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

}  // namespace nestpar
