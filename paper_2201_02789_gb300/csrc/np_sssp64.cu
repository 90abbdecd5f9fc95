// Kernels of the packed-distance SSSP child body (see np_bodies.cuh).
#include "np_table.cuh"

namespace nestpar {
const BodyKernels& sssp64_kernels() {
  static const BodyKernels t = with_sweep<Sssp64SweepBody, 1>(make_table<Sssp64Body>());
  return t;
}
}  // namespace nestpar
