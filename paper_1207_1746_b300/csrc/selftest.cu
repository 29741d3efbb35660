// A self-test of the device-side failure path: one thread waits, with the
// library's bounded wait, on an mbarrier that nothing arrives on.  The wait
// gives up after its cycle limit (about 2 s), the kernel sets bit 0 of the
// device error word and returns; the next gscl_sync reports GSCL_ERR_TIMEOUT
// and the context stays usable.  Nothing faults, traps or hangs.
#include "sweep_kernel.cuh"

namespace gscl {
namespace {

__global__ void bounded_wait_selftest_kernel(int *err) {
  __shared__ uint64_t bar;
  mbar_init(&bar, 1);
  fence_mbar_init();
  if (!mbar_wait_bounded(&bar, 0u)) atomicOr(err, 1);  // phase 0 never completes
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" gscl_status gscl_selftest_bounded_wait(void *stream) {
  int *err = device_error_word();
  if (!err) return fail(GSCL_ERR_CUDA, "device error word unavailable");
  bounded_wait_selftest_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(err);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "self-test launch");
}
