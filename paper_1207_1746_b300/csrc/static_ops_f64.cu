// Compile-time operators (static_ops.h) instantiated for double storage; one
// translation unit per dtype so the build compiles them in parallel.
#include "sweep_kernel.cuh"

namespace gscl {

gscl_status launch_static_f64(const Plan &pl, int red, cudaStream_t stream, int *occupancy_only) {
  return launch_static_t<double>(pl, red, stream, occupancy_only);
}

}  // namespace gscl
