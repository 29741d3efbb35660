// FMA throughput microbenchmark: the measured denominator of the ALU
// roofline for sweeps bound by the FP64 pipe (not part of the paper's
// method; a measurement aid for the rooflines the sweeps are reported on).
//
// Every thread runs CH independent chains a <- a * b + c (|b| < 1, so the
// chains stay bounded and normal), CTAs fill every SM at full occupancy, and
// the elapsed time of `iters` rounds comes from CUDA events on the caller's
// stream after one warm-up launch.
#include "gscl_internal.h"

namespace gscl {
namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T b, T c, T *sink) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x + 1 + i) * T(1e-3);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(-1)) sink[0] = s;  // never true (the chains converge to c / (1 - b) > 0): keeps them live
}

template <typename T>
gscl_status measure(int iters, double *flops_per_s, cudaStream_t st) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T>, kThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy query");
  const int blocks = sm_count() * (per_sm > 0 ? per_sm : 1);
  T *sink = nullptr;
  if ((e = cudaMallocAsync(&sink, sizeof(T), st)) != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const T b = T(0.9999), c = T(1e-4);
  fma_chain_kernel<T><<<blocks, kThreads, 0, st>>>(iters, b, c, sink);  // warm-up
  cudaEventRecord(e0, st);
  fma_chain_kernel<T><<<blocks, kThreads, 0, st>>>(iters, b, c, sink);
  cudaEventRecord(e1, st);
  e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "FMA microbenchmark");
  *flops_per_s = 2.0 * kChains * (double)iters * blocks * kThreads / (ms * 1e-3);
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" gscl_status gscl_fma_throughput(int32_t dtype, int32_t iters, double *flops_per_s, void *stream) {
  if (!flops_per_s) return fail(GSCL_ERR_INVALID, "flops_per_s is NULL");
  if (iters < 1) return fail(GSCL_ERR_INVALID, "iters must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  switch (dtype) {
    case GSCL_F64: return measure<double>(iters, flops_per_s, st);
    case GSCL_F32: return measure<float>(iters, flops_per_s, st);
  }
  return fail(GSCL_ERR_DTYPE, "FMA microbenchmark is for FP64 and FP32");
}
