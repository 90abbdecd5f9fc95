// Child bodies: the child count of a parent and the work of one child item
// for BFS, SSSP, triangle counting and Bezier tessellation.
#pragma once
#include "np_sinks.cuh"

namespace nestpar {

// ------------------------------------------------------------------- bodies
//
// A body gives the child count of a parent (count), what every child of a
// parent shares (parent, or parent_aux from a staged record that carries the
// one 32-bit value aux loads for it), the loads of one child item (fetch) and
// the effect of a batch of K items of one thread (apply_batch), which reports the
// vertices to append to the next frontier. A batch issues all its loads, then
// all its atomics, before it uses any of their results, so a thread keeps K
// memory operations in flight.

// BFS (Section VII): child item = out-edge u->v; claims v for level L+1.
struct BfsBody {
  static constexpr bool kOffsets = false;
  static constexpr bool kPushes = true;
  static constexpr bool kBalance = false;   // child blocks cost the same: static ranges
  static constexpr int kStage = 1;          // edge lists the child can stage: col
  static constexpr bool kWarpLoop = false;
  static constexpr int kWarpParentRegs = NP_WARP_PARENT_MAXREG;
  static constexpr int kCtaParentRegs = NP_CTA_PARENT_MAXREG;
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
  __device__ static unsigned aux(const BodyArgs&, int) { return 0u; }
  __device__ static P parent_aux(const BodyArgs& b, int pid, int base, int N, unsigned) {
    return parent(b, pid, base, N);
  }
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
      cur[k] = 0;
      if (valid[k]) cur[k] = b.unfiltered ? -1 : NP_FILTER_LOAD(&b.level[v[k]]);
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
  static constexpr bool kWarpLoop = false;
  static constexpr int kWarpParentRegs = 96;   // (the stamp form spills at 80)
  static constexpr int kCtaParentRegs = NP_CTA_PARENT_MAXREG;
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
  // what a staged parent record carries besides {parent, base, N}: dist(u)
  __device__ static unsigned aux(const BodyArgs& b, int pid) { return __ldcg(&b.dist[pid]); }
  __device__ static P parent_aux(const BodyArgs& b, int pid, int base, int, unsigned du) {
    return P{base, du, pid & ~b.vmask};
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
  static constexpr bool kWarpLoop = false;
  static constexpr int kWarpParentRegs = NP_WARP_PARENT_MAXREG;
  static constexpr int kCtaParentRegs = NP_CTA_PARENT_MAXREG;
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
  __device__ static unsigned aux(const BodyArgs&, int) { return 0u; }
  __device__ static P parent_aux(const BodyArgs& b, int pid, int base, int N, unsigned) {
    return parent(b, pid, base, N);
  }
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
  static constexpr bool kWarpLoop = false;
  static constexpr int kWarpParentRegs = NP_WARP_PARENT_MAXREG;
  static constexpr int kCtaParentRegs = NP_CTA_PARENT_MAXREG;
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
  // what a staged parent record carries besides {parent, base, N}: dist(u)
  __device__ static unsigned aux(const BodyArgs& b, int pid) { return (unsigned)(__ldcg(&b.dtag[pid]) >> 32); }
  __device__ static P parent_aux(const BodyArgs& b, int pid, int base, int, unsigned du) {
    return P{base, du, pid & ~b.vmask};
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
      cur[k] = (valid[k] && live[k]) ? (b.unfiltered ? ~0ull : NP_FILTER_LOAD(&b.dtag[v[k]])) : 0ull;
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

// ------------------------------------------------ bodies of the swept frontier
//
// In a level with b.sweep set, the next frontier is rebuilt after the level
// from the vertex state (a sweep over the vertices, see frontier_sweep_kernel)
// instead of appended by the children. Nothing then waits on an atomic's
// return: a child item's effect is a fire-and-forget reduction (red.min), and
// the state alone tells which vertices level L reached: level[v] == L + 1
// (BFS), tag(v) == L + 1 (packed SSSP: the last level that lowered dist(v)).
// In other levels these bodies append as the queue bodies do.
__device__ __forceinline__ void red_min_u32(unsigned* p, unsigned v) {
  asm volatile("red.relaxed.gpu.global.min.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_min_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.relaxed.gpu.global.min.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// BFS: level[] read as unsigned (unreached -1 = the largest value), so a claim
// is min(level[v], L + 1): a vertex reached in an earlier level keeps its level,
// whatever a stale filter read said.
struct BfsSweepBody : BfsBody {
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&p)[K], const int (&i)[K], const F (&f)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
    if (!b.sweep) {
      BfsBody::apply_batch<K>(b, p, i, f, valid, push, v);
      return;
    }
    int cur[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      v[k] = f[k].v;
      push[k] = false;
      cur[k] = valid[k] ? NP_FILTER_LOAD(&b.level[v[k]]) : 0;
    }
#pragma unroll
    for (int k = 0; k < K; k++)
      if (valid[k] && cur[k] == -1) red_min_u32(reinterpret_cast<unsigned*>(&b.level[v[k]]), (unsigned)(b.L + 1));
  }
};

// SSSP, packed form: the 64-bit min of (nd << 32 | L + 1) as a reduction; an
// equal distance keeps the older, smaller tag, as in Sssp64Body.
struct Sssp64SweepBody : Sssp64Body {
  template <int K>
  __device__ static void apply_batch(const BodyArgs& b, const P (&p)[K], const int (&i)[K], const F (&f)[K],
                                     const bool (&valid)[K], bool (&push)[K], int (&v)[K]) {
    if (!b.sweep) {
      Sssp64Body::apply_batch<K>(b, p, i, f, valid, push, v);
      return;
    }
    const unsigned tag = (unsigned)(b.L + 1);
    unsigned long long nd[K], cur[K];
    bool live[K];
#pragma unroll
    for (int k = 0; k < K; k++) {
      v[k] = f[k].v;
      push[k] = false;
      live[k] = p[k].du != 0xffffffffu;
      const unsigned long long s = (unsigned long long)p[k].du + f[k].w;
      nd[k] = ((s >= 0xffffffffull ? 0xfffffffeull : s) << 32) | tag;
      cur[k] = (valid[k] && live[k]) ? NP_FILTER_LOAD(&b.dtag[v[k]]) : 0ull;
    }
#pragma unroll
    for (int k = 0; k < K; k++)
      if (valid[k] && live[k] && (nd[k] >> 32) < (cur[k] >> 32)) red_min_u64(&b.dtag[v[k]], nd[k]);
  }
};

// BT (Section VII): parent = quadratic curve; child item j = point j.
struct BezierBody {
  static constexpr bool kOffsets = true;
  static constexpr bool kPushes = false;
  static constexpr bool kBalance = false;
  static constexpr int kStage = 0;
  // serialised curves of 32 points or more run with the whole parent warp (a
  // point only stores: one parent at a time beats spreading several)
  static constexpr bool kWarpLoop = true;
  static constexpr int kWarpParentRegs = 64;   // (no spill: two 512-thread CTAs per SM)
  // (64 still fits two 512-thread CTAs per SM, as 48 does; 48 spills)
  static constexpr int kCtaParentRegs = 64;
  struct P {
    float x0, y0, x1, y1, x2, y2;
    int base;
    float inv;   // 1 / (N - 1), correctly rounded
    float nm1;   // N - 1 (exact)
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
    const float nm1 = (float)(N - 1);
    return P{__ldg(c), __ldg(c + 1), __ldg(c + 2), __ldg(c + 3), __ldg(c + 4), __ldg(c + 5), base, 1.0f / nm1, nm1};
  }
  __device__ static unsigned aux(const BodyArgs&, int) { return 0u; }
  __device__ static P parent_aux(const BodyArgs& b, int pid, int base, int N, unsigned) {
    return parent(b, pid, base, N);
  }
  __device__ static P shfl(const P& p, int src) {
    return P{__shfl_sync(kFull, p.x0, src), __shfl_sync(kFull, p.y0, src), __shfl_sync(kFull, p.x1, src),
             __shfl_sync(kFull, p.y1, src), __shfl_sync(kFull, p.x2, src), __shfl_sync(kFull, p.y2, src),
             __shfl_sync(kFull, p.base, src), __shfl_sync(kFull, p.inv, src), __shfl_sync(kFull, p.nm1, src)};
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
      // t = j / (N - 1) and u = 1 - t = (N - 1 - j) / (N - 1), each from the
      // exact integer numerator times the parent's reciprocal: no division per
      // point, and u keeps its relative accuracy near t = 1, where 1 - t would
      // cancel
      const P& q = p[k];
      const float t = (float)idx[k] * q.inv;
      const float u = (q.nm1 - (float)idx[k]) * q.inv;
      const float b0 = u * u, b1 = 2.0f * u * t, b2 = t * t;
      b.points[q.base + idx[k]] =
          make_float2(b0 * q.x0 + b1 * q.x1 + b2 * q.x2, b0 * q.y0 + b1 * q.y1 + b2 * q.y2);
    }
  }
};

}  // namespace nestpar
