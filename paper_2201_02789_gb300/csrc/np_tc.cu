// Kernels of the triangle-counting child body (see np_bodies.cuh).
#include "np_table.cuh"

namespace nestpar {
const BodyKernels& tc_kernels() {
  static const BodyKernels t = make_table<TcBody>();
  return t;
}
}  // namespace nestpar
