// Kernels of the bfs child body (see np_bodies.cuh).
#include "np_table.cuh"

namespace nestpar {
const BodyKernels& bfs_kernels() {
  static const BodyKernels t = with_sweep<BfsSweepBody, 0>(make_table<BfsBody>());
  return t;
}
}  // namespace nestpar
