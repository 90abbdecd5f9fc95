// Instantiates every kernel of one body and fills its table.
#pragma once
#include "np_device.cuh"
#include "np_kernels.h"

namespace nestpar {

template <class Body, int G>
inline void fill_parent_row(const void* (&row)[kNumCF]) {
  row[0] = (const void*)parent_kernel<Body, G, 1>;
  row[1] = (const void*)parent_kernel<Body, G, 2>;
  row[2] = (const void*)parent_kernel<Body, G, 4>;
  row[3] = (const void*)parent_kernel<Body, G, 8>;
  row[4] = (const void*)parent_kernel<Body, G, 16>;
}

template <class Body>
inline BodyKernels make_table() {
  BodyKernels t{};
  t.parent_nodp = (const void*)parent_warp<Body, 0>;
  t.parent_grid_host = (const void*)parent_warp<Body, 1>;
  t.parent_nodp_cta = (const void*)parent_kernel<Body, G_NODP, 1>;
  fill_parent_row<Body, G_NONE>(t.parent[0]);
  fill_parent_row<Body, G_WARP>(t.parent[1]);
  fill_parent_row<Body, G_BLOCK>(t.parent[2]);
  fill_parent_row<Body, G_MULTIBLOCK>(t.parent[3]);
  t.child_direct[0] = (const void*)child_direct<Body, 1>;
  t.child_direct[1] = (const void*)child_direct<Body, 2>;
  t.child_direct[2] = (const void*)child_direct<Body, 4>;
  t.child_direct[3] = (const void*)child_direct<Body, 8>;
  t.child_direct[4] = (const void*)child_direct<Body, 16>;
  t.child_agg[0] = (const void*)child_agg<Body, 1>;
  t.child_agg[1] = (const void*)child_agg<Body, 2>;
  t.child_agg[2] = (const void*)child_agg<Body, 4>;
  t.child_agg[3] = (const void*)child_agg<Body, 8>;
  t.child_agg[4] = (const void*)child_agg<Body, 16>;
  t.level_loop_nodp = (const void*)level_loop<Body, 0, 1>;
  t.level_loop_agg[0] = (const void*)level_loop<Body, 1, 1>;
  t.level_loop_agg[1] = (const void*)level_loop<Body, 1, 2>;
  t.level_loop_agg[2] = (const void*)level_loop<Body, 1, 4>;
  t.level_loop_agg[3] = (const void*)level_loop<Body, 1, 8>;
  t.level_loop_agg[4] = (const void*)level_loop<Body, 1, 16>;
  t.parent_cta = (const void*)parent_cta<Body>;
  t.child_agg_pack[0] = (const void*)child_agg_pack<Body, 1>;
  t.child_agg_pack[1] = (const void*)child_agg_pack<Body, 2>;
  t.child_agg_pack[2] = (const void*)child_agg_pack<Body, 4>;
  t.child_agg_pack[3] = (const void*)child_agg_pack<Body, 8>;
  t.child_agg_pack[4] = (const void*)child_agg_pack<Body, 16>;
  // level loops only: bodies that append to the next frontier
  t.level_small = Body::kPushes ? (const void*)level_small<Body> : nullptr;
  return t;
}

// Adds the swept-frontier kernels of body S (state kind KIND) to a table.
template <class S, int KIND>
inline BodyKernels with_sweep(BodyKernels t) {
  t.parent_sweep = (const void*)parent_warp<S, 1>;
  t.child_sweep[0] = (const void*)child_agg<S, 1>;
  t.child_sweep[1] = (const void*)child_agg<S, 2>;
  t.child_sweep[2] = (const void*)child_agg<S, 4>;
  t.child_sweep[3] = (const void*)child_agg<S, 8>;
  t.child_sweep[4] = (const void*)child_agg<S, 16>;
  t.frontier_sweep = (const void*)frontier_sweep_kernel<KIND>;
  return t;
}

}  // namespace nestpar
