// FMA throughput microbenchmark: the measured denominator of the ALU
// roofline for sweeps bound by the FP64 pipe (not part of the paper's
// method; a measurement aid for the rooflines the sweeps are reported on).
//
// Every thread runs CH independent chains a <- a * b + c (|b| < 1, so the
// chains stay bounded and normal), CTAs fill every SM at full occupancy, and
// the elapsed time comes from CUDA events on the caller's stream.  Several
// chain counts and block sizes are timed (best of three launches each, after
// a warm-up) and the fastest is reported.
#include <algorithm>

#include "gscl_internal.h"

namespace gscl {
namespace {

template <typename T, int CH, int NT>
__global__ void __launch_bounds__(NT) fma_chain_kernel(int iters, T b, T c, T *sink) {
  T a[CH];
#pragma unroll
  for (int i = 0; i < CH; ++i) a[i] = T(threadIdx.x + 1 + i) * T(1e-3);
#pragma unroll 4
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < CH; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < CH; ++i) s += a[i];
  if (s == T(-1)) sink[0] = s;  // never true (the chains converge to c / (1 - b) > 0): keeps them live
}

// Best of three timed launches (after one warm-up) of one chain count and
// block size, at full occupancy; FLOP/s, or a negative value on failure.
template <typename T, int CH, int NT>
double time_config(int iters, T *sink, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_chain_kernel<T, CH, NT>, NT, 0) != cudaSuccess)
    return -1.0;
  const int blocks = sm_count() * (per_sm > 0 ? per_sm : 1);
  const int it = std::max(1, iters * 8 / CH);  // the same FMA count per thread for every chain count
  const T b = T(0.9999), c = T(1e-4);
  fma_chain_kernel<T, CH, NT><<<blocks, NT, 0, st>>>(it, b, c, sink);
  float best = 1e30f;
  for (int rep = 0; rep < 3; ++rep) {
    cudaEventRecord(e0, st);
    fma_chain_kernel<T, CH, NT><<<blocks, NT, 0, st>>>(it, b, c, sink);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return -1.0;
    best = std::min(best, ms);
  }
  return 2.0 * CH * (double)it * blocks * NT / (best * 1e-3);
}

template <typename T>
gscl_status measure(int iters, double *flops_per_s, cudaStream_t st) {
  T *sink = nullptr;
  cudaError_t e = cudaMallocAsync(&sink, sizeof(T), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double r[] = {time_config<T, 4, 256>(iters, sink, st, e0, e1), time_config<T, 8, 256>(iters, sink, st, e0, e1),
                      time_config<T, 16, 256>(iters, sink, st, e0, e1), time_config<T, 8, 128>(iters, sink, st, e0, e1),
                      time_config<T, 16, 512>(iters, sink, st, e0, e1)};
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "FMA microbenchmark");
  double best = -1.0;
  for (double v : r) best = std::max(best, v);
  if (best <= 0.0) return fail(GSCL_ERR_CUDA, "FMA microbenchmark: no configuration ran");
  *flops_per_s = best;
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
