// Mixed-precision grid update dst = alpha * src (+ dst): the casts and the
// correction step of mixed-precision iterative refinement (an FP64 iterate
// corrected by an FP32 solve, an FP64 residual handed to an FP32 solve).
// Elementwise and bandwidth-bound: one coalesced row pass, no staging.
#include <cuda_bf16.h>

#include "sweep_host.h"

namespace gscl {
namespace {

__device__ __forceinline__ double load_d(const double *p) { return *p; }
__device__ __forceinline__ double load_d(const float *p) { return (double)*p; }
__device__ __forceinline__ double load_d(const __nv_bfloat16 *p) { return (double)__bfloat162float(*p); }
__device__ __forceinline__ void store_d(double *p, double v) { *p = v; }
__device__ __forceinline__ void store_d(float *p, double v) { *p = __double2float_rn(v); }
__device__ __forceinline__ void store_d(__nv_bfloat16 *p, double v) { *p = __double2bfloat16(v); }

struct ConvertArgs {
  char *dst;
  const char *src;
  int64_t dst_pitch, dst_plane, src_pitch, src_plane;  // elements
  int64_t lo[3], n[3];
  double alpha;
};

// blockIdx.x: 256-wide x chunks, blockIdx.y: rows, blockIdx.z: planes.
// Arithmetic in FP64, one rounding to the destination type.
template <typename TD, typename TS, bool ACC>
__global__ void __launch_bounds__(256) convert_kernel(const ConvertArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n[0]) return;
  const int64_t x = a.lo[0] + i, y = a.lo[1] + blockIdx.y, z = a.lo[2] + blockIdx.z;
  TD *d = reinterpret_cast<TD *>(a.dst) + z * a.dst_plane + y * a.dst_pitch + x;
  const TS *s = reinterpret_cast<const TS *>(a.src) + z * a.src_plane + y * a.src_pitch + x;
  double v = a.alpha * load_d(s);
  if (ACC) v += load_d(d);
  store_d(d, v);
}

template <typename TD, typename TS>
gscl_status launch_convert(const ConvertArgs &a, bool acc, cudaStream_t st) {
  dim3 grid((unsigned)((a.n[0] + 255) / 256), (unsigned)a.n[1], (unsigned)a.n[2]);
  if (acc) convert_kernel<TD, TS, true><<<grid, 256, 0, st>>>(a);
  else convert_kernel<TD, TS, false><<<grid, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "convert kernel launch");
}

template <typename TD>
gscl_status dispatch_src(int src_dtype, const ConvertArgs &a, bool acc, cudaStream_t st) {
  switch (src_dtype) {
    case GSCL_F64: return launch_convert<TD, double>(a, acc, st);
    case GSCL_F32: return launch_convert<TD, float>(a, acc, st);
    case GSCL_BF16: return launch_convert<TD, __nv_bfloat16>(a, acc, st);
  }
  return fail(GSCL_ERR_DTYPE, "unknown source dtype");
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" gscl_status gscl_convert(gscl_grid dst, gscl_grid src, double alpha, int32_t accumulate,
                                    const gscl_range *range, void *stream) {
  Grid d, s;
  if (gscl_status e = lookup(dst, &d)) return e;
  if (gscl_status e = lookup(src, &s)) return e;
  if (d.ndim != s.ndim || d.n[0] != s.n[0] || d.n[1] != s.n[1] || d.n[2] != s.n[2])
    return fail(GSCL_ERR_SHAPE, "convert needs grids of one interior extent");
  if (overlaps(d, s) && (d.buf != s.buf || d.dtype != s.dtype))
    return fail(GSCL_ERR_ALIAS, "convert between overlapping storage of different layout");
  ConvertArgs a{};
  for (int ax = 0; ax < 3; ++ax) {
    const int64_t lo = range ? range->lo[ax] : 0, hi = range ? range->hi[ax] : d.n[ax];
    if (lo < 0 || hi > d.n[ax] || lo > hi) return fail(GSCL_ERR_RANGE, "convert range outside the interior");
    a.lo[ax] = lo;
    a.n[ax] = hi - lo;
  }
  if (a.n[0] == 0 || a.n[1] == 0 || a.n[2] == 0) return GSCL_OK;
  if (a.n[1] > 65535 || a.n[2] > 65535) return fail(GSCL_ERR_UNSUPPORTED, "convert range taller than 65535 rows");
  a.dst = d.elem_ptr(0, 0, 0);
  a.src = s.elem_ptr(0, 0, 0);
  a.dst_pitch = d.pitch;
  a.dst_plane = d.plane;
  a.src_pitch = s.pitch;
  a.src_plane = s.plane;
  a.alpha = alpha;
  cudaStream_t st = (cudaStream_t)stream;
  switch (d.dtype) {
    case GSCL_F64: return dispatch_src<double>(s.dtype, a, accumulate != 0, st);
    case GSCL_F32: return dispatch_src<float>(s.dtype, a, accumulate != 0, st);
    case GSCL_BF16: return dispatch_src<__nv_bfloat16>(s.dtype, a, accumulate != 0, st);
  }
  return fail(GSCL_ERR_DTYPE, "unknown destination dtype");
}
