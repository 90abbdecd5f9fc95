// Frontier sinks: how child and parent threads append vertices to the next
// frontier.
#pragma once
#include "np_state.cuh"

namespace nestpar {

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

}  // namespace nestpar
