// Host-visible table of the kernels instantiated for one child body.
#pragma once

namespace nestpar {

constexpr int kNumCF = 5;                     // coarsening factors 1, 2, 4, 8, 16
inline int cf_index(int cf) {
  switch (cf) {
    case 1: return 0;
    case 2: return 1;
    case 4: return 2;
    case 8: return 3;
    case 16: return 4;
    default: return -1;
  }
}

struct BodyKernels {
  const void* parent_nodp;                    // parent_warp<Body, 0>
  const void* parent_grid_host;               // parent_warp<Body, 1>
  const void* parent_nodp_cta;                // parent_kernel<Body, G_NODP, 1>: CTA tiles, no launch code
  const void* parent[4][kNumCF];              // [NONE, WARP, BLOCK, MULTIBLOCK/GRID_DEVICE][cf]
  const void* child_direct[kNumCF];
  const void* child_agg[kNumCF];
  const void* level_loop_nodp;                // level_loop<Body, 0, 1>: persistent no-DP level loop
  const void* level_loop_agg[kNumCF];         // level_loop<Body, 1, cf>: persistent grid-aggregation loop
  const void* parent_cta;                     // parent_cta<Body>: grid-host, CTA tiles (serial modes BLOCK, PACKED)
  const void* child_agg_pack[kNumCF];         // child_agg_pack<Body, cf>: the child grid of PACKED
  const void* level_small;                    // level_small<Body>: one-CTA loop over small levels (or NULL)
  // swept frontier (BFS and packed SSSP only, else NULL): the grid-host parent and
  // child grids of the reducing body, and the sweep that rebuilds the frontier
  const void* parent_sweep;
  const void* child_sweep[kNumCF];
  const void* frontier_sweep;
};

const BodyKernels& bfs_kernels();
const BodyKernels& sssp_kernels();
const BodyKernels& sssp64_kernels();
const BodyKernels& bezier_kernels();
const BodyKernels& tc_kernels();

}  // namespace nestpar
