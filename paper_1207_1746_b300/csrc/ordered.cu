// Ordered iteration spaces (Section 3): do_j_inc / do_j_dec / do_k_inc /
// do_k_dec visit (i, j-1, k) / (i, j+1, k) / (i, j, k-1) / (i, j, k+1)
// before (i, j, k).  The operator is a term list as for do_all; an output
// bound also as an input is read at the element just visited (a recurrence:
// running sums, bidiagonal forward and backward substitution, upwind
// integration along a column).
//
// One thread per column of the ordered axis, columns laid out x-fastest so
// that a warp's loads and stores are 32 consecutive elements; each thread
// walks its column in order and keeps the element just written in registers
// (the recurrence never goes through memory).  The term list is interpreted
// at run time.  The ordered axis must be y or z: columns along x would put a
// warp's accesses a whole row apart.
#include "sweep_host.h"
#include "sweep_kernel.cuh"

namespace gscl {
namespace {

constexpr int kOrdThreads = 128;

struct OrdTerm {
  int16_t in;    // input grid, or -1: the operator's value
  int16_t coef;  // coefficient grid, or -1
  int16_t out;   // output, or -1: a term of the value
  int16_t prev;  // >= 0: reads output `prev` at the element just visited (from registers)
  int16_t nc;    // the input is not written by this call (read-only cache path)
  int16_t cnc;   // the same for the coefficient grid
  int16_t dx, dy, dz;
  float wf;
  double wd;
};

struct OrdParams {
  const char *in[kMaxIn];
  int64_t in_pitch[kMaxIn], in_plane[kMaxIn];  // elements
  char *out[kMaxOut_];
  int64_t out_pitch[kMaxOut_], out_plane[kMaxOut_];
  OrdTerm terms[kMaxTerms];
  int32_t n_terms, n_out;
  int32_t need_prev[kMaxOut_];  // some term reads this output's previous element
  int64_t lo[3], hi[3];
};

__device__ __forceinline__ double ord_weight(const OrdTerm &t, double) { return t.wd; }
__device__ __forceinline__ float ord_weight(const OrdTerm &t, float) { return t.wf; }

template <typename T>
__device__ __forceinline__ typename Arith<T>::A ord_load(const char *base, int64_t idx, bool nc) {
  const T *p = reinterpret_cast<const T *>(base) + idx;
  return to_arith(nc ? __ldg(p) : *p);
}

// AXIS: 1 (y) or 2 (z); INC: increasing along it.
template <typename T, int AXIS, bool INC>
__global__ void __launch_bounds__(kOrdThreads) ordered_kernel(const __grid_constant__ OrdParams P) {
  using A = typename Arith<T>::A;
  constexpr int OTHER = AXIS == 2 ? 1 : 2;
  const int64_t nx = P.hi[0] - P.lo[0], no = P.hi[OTHER] - P.lo[OTHER];
  const int64_t col = (int64_t)blockIdx.x * kOrdThreads + threadIdx.x;
  if (col >= nx * no) return;
  int64_t p[3];
  p[0] = P.lo[0] + col % nx;
  p[OTHER] = P.lo[OTHER] + col / nx;
  const int64_t len = P.hi[AXIS] - P.lo[AXIS];
  auto index = [&](int64_t pitch, int64_t plane, int dx, int dy, int dz) {
    return (p[2] + dz) * plane + (p[1] + dy) * pitch + (p[0] + dx);
  };
  A prev[kMaxOut_];
#pragma unroll
  for (int m = 0; m < kMaxOut_; ++m) {
    prev[m] = A(0);
    if (m < P.n_out && P.need_prev[m]) {
      p[AXIS] = INC ? P.lo[AXIS] - 1 : P.hi[AXIS];
      prev[m] = to_arith(reinterpret_cast<const T *>(P.out[m])[index(P.out_pitch[m], P.out_plane[m], 0, 0, 0)]);
    }
  }
  for (int64_t s = 0; s < len; ++s) {
    p[AXIS] = INC ? P.lo[AXIS] + s : P.hi[AXIS] - 1 - s;
    A v = A(0);
    A o[kMaxOut_];
#pragma unroll
    for (int m = 0; m < kMaxOut_; ++m) o[m] = A(0);
    for (int t = 0; t < P.n_terms; ++t) {  // value terms come first
      const OrdTerm &tm = P.terms[t];
      A x;
      if (tm.in < 0) {
        x = v;
      } else if (tm.prev >= 0) {
        x = prev[0];
#pragma unroll
        for (int m = 1; m < kMaxOut_; ++m)
          if (tm.prev == m) x = prev[m];
      } else {
        x = ord_load<T>(P.in[tm.in], index(P.in_pitch[tm.in], P.in_plane[tm.in], tm.dx, tm.dy, tm.dz), tm.nc);
      }
      if (tm.coef >= 0)
        x = x * ord_load<T>(P.in[tm.coef], index(P.in_pitch[tm.coef], P.in_plane[tm.coef], 0, 0, 0), tm.cnc);
      const A w = ord_weight(tm, A(0));
      if (tm.out < 0) {
        v = fma(w, x, v);
      } else {
#pragma unroll
        for (int m = 0; m < kMaxOut_; ++m)
          if (tm.out == m) o[m] = fma(w, x, o[m]);
      }
    }
    // every output of this element is computed before any is stored
#pragma unroll
    for (int m = 0; m < kMaxOut_; ++m) {
      if (m < P.n_out) {
        reinterpret_cast<T *>(P.out[m])[index(P.out_pitch[m], P.out_plane[m], 0, 0, 0)] = from_arith<T>(o[m]);
        prev[m] = to_arith(from_arith<T>(o[m]));  // the stored (rounded) value feeds the recurrence
      }
    }
  }
}

template <typename T>
gscl_status launch_ordered_t(const OrdParams &P, int axis, bool inc, long long cols, cudaStream_t st) {
  const unsigned blocks = (unsigned)((cols + kOrdThreads - 1) / kOrdThreads);
  if (axis == 2) {
    if (inc) ordered_kernel<T, 2, true><<<blocks, kOrdThreads, 0, st>>>(P);
    else ordered_kernel<T, 2, false><<<blocks, kOrdThreads, 0, st>>>(P);
  } else {
    if (inc) ordered_kernel<T, 1, true><<<blocks, kOrdThreads, 0, st>>>(P);
    else ordered_kernel<T, 1, false><<<blocks, kOrdThreads, 0, st>>>(P);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "ordered kernel launch");
}

}  // namespace
}  // namespace gscl

using namespace gscl;

extern "C" gscl_status gscl_do_ordered(int32_t order, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                                       const gscl_grid *out, int32_t n_out, const gscl_range *range, void *stream) {
  if (order < GSCL_I_INC || order > GSCL_K_DEC) return fail(GSCL_ERR_INVALID, "unknown order %d", order);
  const int axis = order / 2;
  const bool inc = order % 2 == 0;
  if (axis == 0)
    return fail(GSCL_ERR_UNSUPPORTED, "ordered iteration along x is not built (columns must run along y or z)");
  if (!op) return fail(GSCL_ERR_INVALID, "do_ordered needs an operator");
  if (n_out < 1) return fail(GSCL_ERR_INVALID, "do_ordered needs an output");
  Bound b;
  if (gscl_status s = bind(op, false, in, n_in, out, n_out, range, &b, axis, inc ? -1 : 1)) return s;
  if (b.empty) return GSCL_OK;
  OrdParams P;
  memset(&P, 0, sizeof P);
  int alias[kMaxIn];
  for (int a = 0; a < n_in; ++a) {
    const Grid &g = b.in[a];
    alias[a] = -1;
    for (int m = 0; m < n_out; ++m)
      if (overlaps(g, b.out[m])) alias[a] = m;  // bind has checked it is the same grid
    P.in[a] = g.elem_ptr(0, 0, 0);
    P.in_pitch[a] = g.pitch;
    P.in_plane[a] = g.plane;
  }
  for (int m = 0; m < n_out; ++m) {
    P.out[m] = b.out[m].elem_ptr(0, 0, 0);
    P.out_pitch[m] = b.out[m].pitch;
    P.out_plane[m] = b.out[m].plane;
  }
  // value terms first, then the outputs' terms, each group in descriptor order
  int nt = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int t = 0; t < op->n_terms; ++t) {
      const gscl_term &tm = op->terms[t];
      if ((tm.out == GSCL_VALUE) != (pass == 0)) continue;
      OrdTerm &d = P.terms[nt++];
      d.in = tm.in == GSCL_VALUE ? -1 : (int16_t)tm.in;
      d.coef = tm.coef == GSCL_NONE ? -1 : (int16_t)tm.coef;
      d.out = tm.out == GSCL_VALUE ? -1 : (int16_t)tm.out;
      d.dx = tm.dx;
      d.dy = tm.dy;
      d.dz = tm.dz;
      d.prev = -1;
      if (d.in >= 0 && alias[d.in] >= 0 && (tm.dx || tm.dy || tm.dz)) {
        d.prev = (int16_t)alias[d.in];  // bind allowed only the element just visited
        P.need_prev[d.prev] = 1;
      }
      d.nc = (int16_t)(d.in >= 0 && alias[d.in] < 0);
      d.cnc = (int16_t)(d.coef >= 0 && alias[d.coef] < 0);
      d.wf = (float)tm.w;
      d.wd = tm.w;
    }
  P.n_terms = nt;
  P.n_out = n_out;
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = b.lo[a];
    P.hi[a] = b.hi[a];
  }
  const int other = axis == 2 ? 1 : 2;
  const long long cols = (long long)(b.hi[0] - b.lo[0]) * (b.hi[other] - b.lo[other]);
  cudaStream_t st = (cudaStream_t)stream;
  switch (b.in[0].dtype) {
    case GSCL_F64: return launch_ordered_t<double>(P, axis, inc, cols, st);
    case GSCL_F32: return launch_ordered_t<float>(P, axis, inc, cols, st);
    case GSCL_BF16: return launch_ordered_t<__nv_bfloat16>(P, axis, inc, cols, st);
  }
  return fail(GSCL_ERR_DTYPE, "unknown dtype");
}
