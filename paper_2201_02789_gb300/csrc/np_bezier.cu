// Kernels of the bezier child body (see np_bodies.cuh).
#include "np_table.cuh"

namespace nestpar {
const BodyKernels& bezier_kernels() {
  static const BodyKernels t = make_table<BezierBody>();
  return t;
}
}  // namespace nestpar
