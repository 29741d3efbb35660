// Compile-time operators (static_ops.h) instantiated for FP64 grids in pair
// arithmetic (pair64.cuh); one translation unit per storage type so the
// build compiles them in parallel.
#include "sweep_kernel.cuh"

namespace gscl {

gscl_status launch_static_f64pair(const Plan &pl, int red, cudaStream_t stream, int *occupancy_only) {
  return launch_static_t<f64pair>(pl, red, stream, occupancy_only);
}

}  // namespace gscl
