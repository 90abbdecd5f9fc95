// Kernels of the sssp child body (see np_bodies.cuh).
#include "np_table.cuh"

namespace nestpar {
const BodyKernels& sssp_kernels() {
  static const BodyKernels t = make_table<SsspBody>();
  return t;
}
}  // namespace nestpar
