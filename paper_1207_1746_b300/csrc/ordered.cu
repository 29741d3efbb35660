// Ordered iteration spaces (Section 3): do_i_inc / do_i_dec / do_j_inc /
// do_j_dec / do_k_inc / do_k_dec visit (i-1, j, k) / (i+1, j, k) /
// (i, j-1, k) / (i, j+1, k) / (i, j, k-1) / (i, j, k+1) before (i, j, k).  The operator is a term list as for do_all; an output
// bound also as an input is read at the element just visited (a recurrence:
// running sums, bidiagonal forward and backward substitution, upwind
// integration along a column).
//
// One thread per column of the ordered axis, columns laid out x-fastest so
// that a warp's loads and stores are 32 consecutive elements; each thread
// walks its column in order and keeps the element just written in registers
// (the recurrence never goes through memory).  The term list is interpreted
// at run time.  Operators with at most kLoads distinct element loads per
// step take a pipelined path: every load of the element kAhead steps ahead is
// issued together into a register ring, so a column waits for memory once
// per kAhead steps instead of once per term and step.  The ring lives in
// shared memory, one private column of slots per thread, filled by cp.async
// (one commit group per step; a thread waits only for its own copies), so
// slots can be indexed at run time.  FP32 / FP64 storage (cp.async moves 4 or
// 8 bytes); BF16 takes the simple path.  Along x (do_i_inc / do_i_dec) a
// thread per row would put a warp's accesses a whole row apart, so rows go
// through shared memory in chunks of 16 to 64 steps (ordered_x_kernel and
// ordered_x_pair_kernel below).
//
// The common recurrences (running sums, first-order recurrences, bidiagonal
// substitution) are also compiled: their shape (which load, output or value
// each term reads, and in what order) is a constant, the step loop is
// unrolled by the look-ahead so the ring is a register array with constant
// slots, and a step costs its loads, its multiply-adds and its stores.
// Grids, offsets, direction and weights stay runtime values, and the
// arithmetic is the interpreted loop's, operation for operation.
#include "sweep_host.h"
#include "sweep_kernel.cuh"

namespace gscl {
namespace {

constexpr int kOrdThreads = 128;
constexpr int kLoads = 8;   // distinct element loads per step on the pipelined path
constexpr int kAheadFew = 16;  // steps of look-ahead for operators with at most kFewLoads loads
constexpr int kAheadMany = 4;  // ... and for the others (up to kLoads)
constexpr int kFewLoads = 3;

struct OrdLoad {
  int16_t grid, nc, dx, dy, dz, pad;
  int64_t start;  // element offset of the read at the column's first step, without the column's base
  int64_t step;   // element offset from one step to the next (signed)
};

struct OrdTerm {
  int16_t in;    // input grid, or -1: the operator's value
  int16_t coef;  // coefficient grid, or -1
  int16_t out;   // output, or -1: a term of the value
  int16_t prev;  // >= 0: reads output `prev` at the element just visited (from registers)
  int16_t nc;    // the input is not written by this call (read-only cache path)
  int16_t cnc;   // the same for the coefficient grid
  int16_t dx, dy, dz;
  int16_t xslot;  // pipelined path: ring slot of the input value (-1: value or previous element)
  int16_t cslot;  // ring slot of the coefficient (-1: none)
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
  OrdLoad loads[kLoads];        // pipelined path: the distinct loads (n_loads <= kLoads)
  int32_t n_loads;              // > kLoads: the simple path
  int64_t out_start[kMaxOut_], out_step[kMaxOut_];  // the outputs' element at the first step, step offset
};

__device__ __forceinline__ double ord_weight(const OrdTerm &t, double) { return t.wd; }
__device__ __forceinline__ float ord_weight(const OrdTerm &t, float) { return t.wf; }

template <typename T>
__device__ __forceinline__ typename Arith<T>::A ord_load(const char *base, int64_t idx, bool nc) {
  const T *p = reinterpret_cast<const T *>(base) + idx;
  return to_arith(nc ? __ldg(p) : *p);
}

__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Copies the pipelined path's loads of step `step` into ring slot `slot` of
// this thread (element [slot][l][threadIdx.x] of the ring); src[l] points at
// load l's element of the column's first step.
template <typename T>
__device__ __forceinline__ void issue_loads(const OrdParams &P, const T *const (&src)[kLoads], int64_t step, T *ring,
                                            int slot) {
  T *dst = ring + (int64_t)slot * P.n_loads * kOrdThreads + threadIdx.x;
#pragma unroll
  for (int l = 0; l < kLoads; ++l)
    if (l < P.n_loads) cp_async(dst + l * kOrdThreads, src[l] + step * P.loads[l].step, (int)sizeof(T));
}

// AXIS: 1 (y) or 2 (z); INC: increasing along it; AHEAD: look-ahead of the
// pipelined path (0: the simple path), whose ring is the dynamic shared
// memory (AHEAD x n_loads x kOrdThreads elements).
template <typename T, int AXIS, bool INC, int AHEAD>
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
  if constexpr (AHEAD > 0) {
    // pipelined path: ring slot s % AHEAD holds the loads of step s
    extern __shared__ __align__(16) unsigned char ord_smem[];
    T *ring = reinterpret_cast<T *>(ord_smem);
    // the column's base in each grid (x and the non-ordered coordinate)
    auto colbase = [&](int64_t pitch, int64_t plane) { return p[0] + p[OTHER] * (OTHER == 1 ? pitch : plane); };
    const T *src[kLoads];
#pragma unroll
    for (int l = 0; l < kLoads; ++l) {
      src[l] = nullptr;
      if (l < P.n_loads) {
        const OrdLoad &ld = P.loads[l];
        src[l] = reinterpret_cast<const T *>(P.in[ld.grid]) + colbase(P.in_pitch[ld.grid], P.in_plane[ld.grid]) +
                 ld.start;
      }
    }
    T *dst[kMaxOut_];
#pragma unroll
    for (int m = 0; m < kMaxOut_; ++m)
      dst[m] = m < P.n_out ? reinterpret_cast<T *>(P.out[m]) + colbase(P.out_pitch[m], P.out_plane[m]) + P.out_start[m]
                           : nullptr;
#pragma unroll
    for (int d = 0; d < AHEAD; ++d) {
      if (d < len) issue_loads<T>(P, src, d, ring, d);
      cp_async_commit();
    }
    for (int64_t s = 0; s < len; ++s) {
      cp_async_wait<AHEAD - 1>();  // this thread's copies of step s have landed
      const int slot = (int)(s % AHEAD);
      const T *r = ring + (int64_t)slot * P.n_loads * kOrdThreads + threadIdx.x;
      A v = A(0);
      A o[kMaxOut_];
#pragma unroll
      for (int m = 0; m < kMaxOut_; ++m) o[m] = A(0);
      for (int t = 0; t < P.n_terms; ++t) {
        const OrdTerm &tm = P.terms[t];
        A x = v;
        if (tm.prev >= 0) {
          x = prev[0];
#pragma unroll
          for (int m = 1; m < kMaxOut_; ++m)
            if (tm.prev == m) x = prev[m];
        } else if (tm.xslot >= 0) {
          x = to_arith(r[tm.xslot * kOrdThreads]);
        }
        if (tm.cslot >= 0) x = x * to_arith(r[tm.cslot * kOrdThreads]);
        const A w = ord_weight(tm, A(0));
        if (tm.out < 0) {
          v = fma(w, x, v);
        } else {
#pragma unroll
          for (int m = 0; m < kMaxOut_; ++m)
            if (tm.out == m) o[m] = fma(w, x, o[m]);
        }
      }
#pragma unroll
      for (int m = 0; m < kMaxOut_; ++m) {
        if (m < P.n_out) {
          dst[m][s * P.out_step[m]] = from_arith<T>(o[m]);
          prev[m] = to_arith(from_arith<T>(o[m]));
        }
      }
      // the slot just used takes the element AHEAD steps on (issued after this
      // element's stores; that element is written only at its own step)
      if (s + AHEAD < len) issue_loads<T>(P, src, s + AHEAD, ring, slot);
      cp_async_commit();
    }
    cp_async_wait<0>();
  } else {
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
}

// ------------------------------------------------------------ compiled shapes
// A term of a compiled shape: where its input value comes from (xs: a load
// slot 0..kLoads-1, kSrcValue for the operator's value, kSrcPrev + m for
// output m at the element just visited), its coefficient slot (cs, -1: none)
// and where it adds (out, -1: the value).  Slots are numbered in the order
// the terms first use them, as the host numbers the loads.
constexpr int kSrcValue = -1;
constexpr int kSrcPrev = 16;
struct OrdShapeTerm {
  int xs, cs, out;
};
template <int N>
struct OrdShapeTable {
  OrdShapeTerm t[N];
};

enum OrdShapeId { ORD_ROWS_X = -3, ORD_INTERPRETED = -1, ORD_SIMPLE = -2, ORD_RUNSUM_PREV_FIRST = 0, ORD_RUNSUM, ORD_BIDIAG,
                  ORD_BIDIAG_PREV_FIRST, ORD_AXPY2, ORD_SHAPES };

struct OrdRunSumPrevFirst {  // x = a x(prev) + b f
  static constexpr int NL = 1, NT = 2, NOUT = 1;
  static constexpr OrdShapeTable<NT> table = {{{kSrcPrev, -1, 0}, {0, -1, 0}}};
};
struct OrdRunSum {  // x = b f + a x(prev)
  static constexpr int NL = 1, NT = 2, NOUT = 1;
  static constexpr OrdShapeTable<NT> table = {{{0, -1, 0}, {kSrcPrev, -1, 0}}};
};
struct OrdBidiag {  // x = a g + b m x(prev): forward / backward substitution
  static constexpr int NL = 2, NT = 2, NOUT = 1;
  static constexpr OrdShapeTable<NT> table = {{{0, -1, 0}, {kSrcPrev, 1, 0}}};
};
struct OrdBidiagPrevFirst {  // x = b m x(prev) + a g
  static constexpr int NL = 2, NT = 2, NOUT = 1;
  static constexpr OrdShapeTable<NT> table = {{{kSrcPrev, 0, 0}, {1, -1, 0}}};
};
struct OrdAxpy2 {  // x = a f + b g + c x(prev): upwind integration with two sources
  static constexpr int NL = 2, NT = 3, NOUT = 1;
  static constexpr OrdShapeTable<NT> table = {{{0, -1, 0}, {1, -1, 0}, {kSrcPrev, -1, 0}}};
};

template <class S>
GSCL_HD constexpr bool shape_reads_prev(int m) {
  for (int t = 0; t < S::NT; ++t)
    if (S::table.t[t].xs == kSrcPrev + m) return true;
  return false;
}

// One thread per column as above; the step loop is unrolled by AHEAD so that
// ring slot j (registers) always holds the loads of steps = j mod AHEAD.  At
// each step the loads of the element AHEAD steps on are issued after this
// element's stores (that element is written only at its own step).
template <typename T, int AXIS, bool INC, class S, int AHEAD>
__global__ void __launch_bounds__(kOrdThreads) ordered_compiled_kernel(const __grid_constant__ OrdParams P) {
  using A = typename Arith<T>::A;
  constexpr int NL = S::NL, NT = S::NT, NO = S::NOUT;
  constexpr int OTHER = AXIS == 2 ? 1 : 2;
  const int64_t nx = P.hi[0] - P.lo[0], no = P.hi[OTHER] - P.lo[OTHER];
  const int64_t col = (int64_t)blockIdx.x * kOrdThreads + threadIdx.x;
  if (col >= nx * no) return;
  const int64_t x0 = P.lo[0] + col % nx, y0 = P.lo[OTHER] + col / nx;
  const int len = (int)(P.hi[AXIS] - P.lo[AXIS]);
  const T *q[NL];  // the next element each load fetches
  int64_t qs[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    const OrdLoad &ld = P.loads[l];
    q[l] = reinterpret_cast<const T *>(P.in[ld.grid]) + x0 +
           y0 * (OTHER == 1 ? P.in_pitch[ld.grid] : P.in_plane[ld.grid]) + ld.start;
    qs[l] = ld.step;
  }
  T *d[NO];
  int64_t ds[NO];
  A prev[NO];
#pragma unroll
  for (int m = 0; m < NO; ++m) {
    d[m] = reinterpret_cast<T *>(P.out[m]) + x0 + y0 * (OTHER == 1 ? P.out_pitch[m] : P.out_plane[m]) +
           P.out_start[m];
    ds[m] = P.out_step[m];
    prev[m] = A(0);
  }
  static_for<NO>([&](auto mc) {
    constexpr int m = decltype(mc)::value;
    if constexpr (shape_reads_prev<S>(m)) prev[m] = to_arith(d[m][-ds[m]]);
  });
  T r[AHEAD][NL];
#pragma unroll
  for (int j = 0; j < AHEAD; ++j) {
    if (j < len) {
#pragma unroll
      for (int l = 0; l < NL; ++l) r[j][l] = q[l][j * qs[l]];
    }
  }
#pragma unroll
  for (int l = 0; l < NL; ++l) q[l] += AHEAD * qs[l];
  auto element = [&](const T (&rj)[NL]) {
    A v = A(0);
    A o[NO];
#pragma unroll
    for (int m = 0; m < NO; ++m) o[m] = A(0);
    static_for<NT>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      constexpr OrdShapeTerm st = S::table.t[t];
      A x;
      if constexpr (st.xs == kSrcValue) x = v;
      else if constexpr (st.xs >= kSrcPrev) x = prev[st.xs - kSrcPrev];
      else x = to_arith(rj[st.xs]);
      if constexpr (st.cs >= 0) x = x * to_arith(rj[st.cs]);
      const A w = ord_weight(P.terms[t], A(0));
      if constexpr (st.out < 0) v = fma(w, x, v);
      else o[st.out] = fma(w, x, o[st.out]);
    });
#pragma unroll
    for (int m = 0; m < NO; ++m) {
      const T y = from_arith<T>(o[m]);
      *d[m] = y;
      d[m] += ds[m];
      prev[m] = to_arith(y);
    }
  };
  int s0 = 0;
  for (; s0 + AHEAD <= len; s0 += AHEAD) {
    static_for<AHEAD>([&](auto jc) {
      constexpr int j = decltype(jc)::value;
      element(r[j]);
      if (s0 + j + AHEAD < len) {
#pragma unroll
        for (int l = 0; l < NL; ++l) r[j][l] = *q[l];
      }
#pragma unroll
      for (int l = 0; l < NL; ++l) q[l] += qs[l];
    });
  }
  // the last len mod AHEAD steps: their loads are in slots 0.. already
  static_for<AHEAD>([&](auto jc) {
    constexpr int j = decltype(jc)::value;
    if (s0 + j < len) element(r[j]);
  });
}

struct OrdShapeDesc {
  int id, nl, nt, nout;
  const OrdShapeTerm *t;
};

template <class S>
OrdShapeDesc shape_desc(int id) {
  return OrdShapeDesc{id, S::NL, S::NT, S::NOUT, S::table.t};
}

const std::vector<OrdShapeDesc> &ord_shapes() {
  static const std::vector<OrdShapeDesc> v = {
      shape_desc<OrdRunSumPrevFirst>(ORD_RUNSUM_PREV_FIRST), shape_desc<OrdRunSum>(ORD_RUNSUM),
      shape_desc<OrdBidiag>(ORD_BIDIAG), shape_desc<OrdBidiagPrevFirst>(ORD_BIDIAG_PREV_FIRST),
      shape_desc<OrdAxpy2>(ORD_AXPY2)};
  return v;
}

// The compiled shape the prepared parameters have, else ORD_INTERPRETED
// (pipelined term loop) or ORD_SIMPLE (per-term loads).
int ordered_shape(const OrdParams &P, gscl_dtype dt) {
  const bool ring_dtype = dt == GSCL_F32 || dt == GSCL_F64;
  if (P.n_loads > kLoads) return ORD_SIMPLE;
  const char *env = getenv("GSCL_GENERIC_ONLY");
  const bool generic = env && env[0] && env[0] != '0';
  if (!generic) {
    for (const OrdShapeDesc &d : ord_shapes()) {
      if (d.nl != P.n_loads || d.nt != P.n_terms || d.nout != P.n_out) continue;
      bool ok = true;
      for (int t = 0; t < d.nt && ok; ++t) {
        const OrdTerm &tm = P.terms[t];
        const int xs = tm.prev >= 0 ? kSrcPrev + tm.prev : tm.in < 0 ? kSrcValue : tm.xslot;
        ok = xs == d.t[t].xs && tm.cslot == d.t[t].cs && tm.out == d.t[t].out;
      }
      if (ok) return d.id;
    }
  }
  return ring_dtype ? ORD_INTERPRETED : ORD_SIMPLE;
}

template <typename T, int AXIS, bool INC, class S>
gscl_status launch_compiled(const OrdParams &P, long long cols, cudaStream_t st) {
  const unsigned blocks = (unsigned)((cols + kOrdThreads - 1) / kOrdThreads);
  ordered_compiled_kernel<T, AXIS, INC, S, kAheadFew><<<blocks, kOrdThreads, 0, st>>>(P);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "ordered kernel launch");
}

template <typename T, int AXIS, bool INC>
gscl_status launch_shape(const OrdParams &P, int shape, long long cols, cudaStream_t st) {
  switch (shape) {
    case ORD_RUNSUM_PREV_FIRST: return launch_compiled<T, AXIS, INC, OrdRunSumPrevFirst>(P, cols, st);
    case ORD_RUNSUM: return launch_compiled<T, AXIS, INC, OrdRunSum>(P, cols, st);
    case ORD_BIDIAG: return launch_compiled<T, AXIS, INC, OrdBidiag>(P, cols, st);
    case ORD_BIDIAG_PREV_FIRST: return launch_compiled<T, AXIS, INC, OrdBidiagPrevFirst>(P, cols, st);
    case ORD_AXPY2: return launch_compiled<T, AXIS, INC, OrdAxpy2>(P, cols, st);
  }
  return fail(GSCL_ERR_INVALID, "unknown ordered shape %d", shape);
}

template <typename T, int AXIS, bool INC>
gscl_status launch_ordered_dir(const OrdParams &P, int shape, long long cols, cudaStream_t st) {
  if (shape >= 0) return launch_shape<T, AXIS, INC>(P, shape, cols, st);
  const unsigned blocks = (unsigned)((cols + kOrdThreads - 1) / kOrdThreads);
  if constexpr (sizeof(T) >= 4) {
    if (shape == ORD_INTERPRETED) {
      const bool few = P.n_loads <= kFewLoads;
      const size_t smem = (size_t)(few ? kAheadFew : kAheadMany) * P.n_loads * kOrdThreads * sizeof(T);
      if (few) ordered_kernel<T, AXIS, INC, kAheadFew><<<blocks, kOrdThreads, smem, st>>>(P);
      else ordered_kernel<T, AXIS, INC, kAheadMany><<<blocks, kOrdThreads, smem, st>>>(P);
      cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "ordered kernel launch");
    }
  }
  ordered_kernel<T, AXIS, INC, 0><<<blocks, kOrdThreads, 0, st>>>(P);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "ordered kernel launch");
}

// ------------------------------------------------------------ ordered along x
// do_i_inc / do_i_dec: rows along x are walked in order, one lane per row,
// 32 rows at a time.  A lane walking its row through global memory would put
// a warp's accesses a whole row apart, so rows go through shared memory in
// chunks: every distinct load of a chunk is staged for the 32 rows with
// coalesced row reads (every row of every load in flight at once), the lanes
// walk their rows through the transposed tile (a row stride of chunk + 1
// elements keeps the banks apart) keeping each output's element just written
// in registers, and the outputs of the chunk go back through a transposed
// output tile with coalesced row stores.  Staging runs ahead of the compute:
// an output read as an input is read only at the element itself, which no
// chunk writes for a later one, so early staging reads the right values.
// The compiled recurrences and the interpreted term loop compute the same
// operations in the same order as on the other axes.  Two kernels:
//  - ordered_x_pair_kernel (8-byte elements): blocks of two warps, one
//    computing and one moving data.  The FP64 recurrence is long (its chain
//    of dependent FP64-pipe operations), and the second warp takes the
//    staging and the stores off it.
//  - ordered_x_kernel (4- and 2-byte elements): one warp per block, which
//    stages chunk c + 1 before computing and storing chunk c.  Its longer
//    chunks (64 steps, in the shared memory a warp pair would need for 32)
//    measured faster where the recurrence itself is cheap.
struct OrdInterpretedX {};

// One warp per block: load tiles double-buffered, one output tile; the row
// offsets of every load and output are computed once per lane and shared
// through shared memory.
template <typename T>
struct XChunkWarp {
  static constexpr int value = sizeof(T) == 8 ? 32 : 64;
};

// Dynamic shared memory of one block (one warp): two buffers of load tiles
// and one tile per output, 32 rows of XChunkWarp + 1 elements each.
template <typename T>
size_t ordered_x_smem(int n_loads, int n_out) {
  return (size_t)(2 * n_loads + n_out) * 32 * (XChunkWarp<T>::value + 1) * sizeof(T);
}

template <typename T, bool INC, class S>
__global__ void __launch_bounds__(32) ordered_x_kernel(const __grid_constant__ OrdParams P) {
  using A = typename Arith<T>::A;
  constexpr int KC = XChunkWarp<T>::value;
  constexpr int TS = KC + 1;     // row stride of a tile
  constexpr int TILE = 32 * TS;  // one load's or one output's tile: 32 rows
  extern __shared__ __align__(16) unsigned char ox_smem[];
  // element offset of row r's first element (x = 0) in load l's grid, with
  // the load's offset, at [l][r]; output m's at [kLoads + m][r]
  __shared__ int64_t rbase[kLoads + kMaxOut_][32];
  const int lane = threadIdx.x;
  const int nl = P.n_loads, no = P.n_out;
  T *lt = reinterpret_cast<T *>(ox_smem);  // load tiles: [buffer][load]
  T *ot = lt + (size_t)2 * nl * TILE;      // output tiles
  const int64_t ny = P.hi[1] - P.lo[1], rows = ny * (P.hi[2] - P.lo[2]);
  const int64_t row0 = (int64_t)blockIdx.x * 32;
  if (row0 >= rows) return;  // the whole warp
  const int64_t my = row0 + lane;
  const bool live = my < rows;
  const int64_t yl = live ? P.lo[1] + my % ny : 0, zl = live ? P.lo[2] + my / ny : 0;
  const int64_t len = P.hi[0] - P.lo[0];
  for (int l = 0; l < nl; ++l) {
    const OrdLoad &ld = P.loads[l];
    rbase[l][lane] = (zl + ld.dz) * P.in_plane[ld.grid] + (yl + ld.dy) * P.in_pitch[ld.grid] + ld.dx;
  }
  for (int m = 0; m < no; ++m) rbase[kLoads + m][lane] = zl * P.out_plane[m] + yl * P.out_pitch[m];
  A prev[kMaxOut_];
#pragma unroll
  for (int m = 0; m < kMaxOut_; ++m) {
    prev[m] = A(0);
    if (live && m < no && P.need_prev[m])
      prev[m] = to_arith(reinterpret_cast<const T *>(P.out[m])[zl * P.out_plane[m] + yl * P.out_pitch[m] +
                                                                 (INC ? P.lo[0] - 1 : P.hi[0])]);
  }
  __syncwarp();
  const int nrows = (int)min((int64_t)32, rows - row0);
  const int64_t nchunks = (len + KC - 1) / KC;
  // chunk c: its length and its lowest x; step j of the chunk is element
  // e = j (increasing) or e = clen - 1 - j (decreasing) of it
  auto chunk = [&](int64_t c, int &clen) -> int64_t {
    const int64_t c0 = c * KC;
    clen = (int)min((int64_t)KC, len - c0);
    return INC ? P.lo[0] + c0 : P.hi[0] - c0 - clen;
  };
  // stages chunk c of every load into buffer c & 1 (one commit group)
  auto issue = [&](int64_t c) {
    int clen;
    const int64_t xs = chunk(c, clen);
    T *buf = lt + (size_t)(c & 1) * nl * TILE;
    for (int l = 0; l < nl; ++l) {
      const T *g = reinterpret_cast<const T *>(P.in[P.loads[l].grid]) + xs;
      T *tl = buf + l * TILE;
#pragma unroll 8
      for (int rr = 0; rr < nrows; ++rr) {
        const T *src = g + rbase[l][rr];
#pragma unroll
        for (int k = 0; k < KC / 32; ++k) {
          const int e = lane + 32 * k;
          if (e < clen) {
            T *d = tl + rr * TS + (INC ? e : clen - 1 - e);
            if constexpr (sizeof(T) >= 4) cp_async(d, src + e, (int)sizeof(T));
            else *d = src[e];
          }
        }
      }
    }
    if constexpr (sizeof(T) >= 4) cp_async_commit();
  };
  issue(0);
  for (int64_t c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      issue(c + 1);
      if constexpr (sizeof(T) >= 4) cp_async_wait<1>();  // chunk c has landed
    } else if constexpr (sizeof(T) >= 4) {
      cp_async_wait<0>();
    }
    __syncwarp();
    int clen;
    const int64_t xs = chunk(c, clen);
    if (live) {
      const T *r = lt + (size_t)(c & 1) * nl * TILE + lane * TS;
      T *o_t = ot + lane * TS;
      if constexpr (!std::is_same<S, OrdInterpretedX>::value) {
        // compiled recurrence: every term's slot a constant.  One step reads
        // the staged value of load slot l as val(l) and leaves output m's
        // element in y[m].
        auto step = [&](auto val, T (&y)[S::NOUT]) {
          A v = A(0);
          A o[S::NOUT];
#pragma unroll
          for (int m = 0; m < S::NOUT; ++m) o[m] = A(0);
          static_for<S::NT>([&](auto tc) {
            constexpr int t = decltype(tc)::value;
            constexpr OrdShapeTerm st = S::table.t[t];
            A x;
            if constexpr (st.xs == kSrcValue) x = v;
            else if constexpr (st.xs >= kSrcPrev) x = prev[st.xs - kSrcPrev];
            else x = val(st.xs);
            if constexpr (st.cs >= 0) x = x * val(st.cs);
            const A wgt = ord_weight(P.terms[t], A(0));
            if constexpr (st.out < 0) v = fma(wgt, x, v);
            else o[st.out] = fma(wgt, x, o[st.out]);
          });
#pragma unroll
          for (int m = 0; m < S::NOUT; ++m) {
            y[m] = from_arith<T>(o[m]);
            prev[m] = to_arith(y[m]);
          }
        };
        if (clen == KC) {
          // groups of G steps: the next group's staged values are read into
          // registers before this group is computed (the reads are not held
          // behind this group's output writes), and a group's outputs are
          // written to the tile together
          constexpr int G = 8;
          A cur[S::NL][G], nxt[S::NL][G];
          auto fetch = [&](int s0, A(&d)[S::NL][G]) {
#pragma unroll
            for (int l = 0; l < S::NL; ++l)
#pragma unroll
              for (int g = 0; g < G; ++g) d[l][g] = to_arith(r[l * TILE + s0 + g]);
          };
          fetch(0, cur);
#pragma unroll
          for (int s0 = 0; s0 < KC; s0 += G) {
            if (s0 + G < KC) fetch(s0 + G, nxt);
            T ys[G][S::NOUT];
#pragma unroll
            for (int g = 0; g < G; ++g) step([&](int l) { return cur[l][g]; }, ys[g]);
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
              for (int m = 0; m < S::NOUT; ++m) o_t[m * TILE + s0 + g] = ys[g][m];
#pragma unroll
            for (int l = 0; l < S::NL; ++l)
#pragma unroll
              for (int g = 0; g < G; ++g) cur[l][g] = nxt[l][g];
          }
        } else {
          for (int s = 0; s < clen; ++s) {
            T y[S::NOUT];
            step([&](int l) { return to_arith(r[l * TILE + s]); }, y);
#pragma unroll
            for (int m = 0; m < S::NOUT; ++m) o_t[m * TILE + s] = y[m];
          }
        }
      } else {
        for (int s = 0; s < clen; ++s) {
          A v = A(0);
          A o[kMaxOut_];
#pragma unroll
          for (int m = 0; m < kMaxOut_; ++m) o[m] = A(0);
          for (int t = 0; t < P.n_terms; ++t) {
            const OrdTerm &tm = P.terms[t];
            A x = v;
            if (tm.prev >= 0) {
              x = prev[0];
#pragma unroll
              for (int m = 1; m < kMaxOut_; ++m)
                if (tm.prev == m) x = prev[m];
            } else if (tm.xslot >= 0) {
              x = to_arith(r[tm.xslot * TILE + s]);
            }
            if (tm.cslot >= 0) x = x * to_arith(r[tm.cslot * TILE + s]);
            const A wgt = ord_weight(tm, A(0));
            if (tm.out < 0) {
              v = fma(wgt, x, v);
            } else {
#pragma unroll
              for (int m = 0; m < kMaxOut_; ++m)
                if (tm.out == m) o[m] = fma(wgt, x, o[m]);
            }
          }
#pragma unroll
          for (int m = 0; m < kMaxOut_; ++m) {
            if (m < no) {
              const T y = from_arith<T>(o[m]);
              o_t[m * TILE + s] = y;
              prev[m] = to_arith(y);
            }
          }
        }
      }
    }
    __syncwarp();
    for (int m = 0; m < no; ++m) {
      T *g = reinterpret_cast<T *>(P.out[m]) + xs;
      const T *to = ot + m * TILE;
#pragma unroll 8
      for (int rr = 0; rr < nrows; ++rr) {
        T *dst = g + rbase[kLoads + m][rr];
#pragma unroll
        for (int k = 0; k < KC / 32; ++k) {
          const int e = lane + 32 * k;
          if (e < clen) dst[e] = to[rr * TS + (INC ? e : clen - 1 - e)];
        }
      }
    }
    __syncwarp();  // the tiles of chunk c are read before chunk c + 2 is staged
  }
}

// Two warps per block: the first walks the rows, the second moves data.
// While chunk c is computed the mover has chunk c + 1 staged, is staging
// chunk c + 2 and is storing chunk c - 1; one block barrier per chunk hands
// the buffers over (three load buffers, two output buffers).
template <typename T>
struct XChunkPair {
  static constexpr int value = sizeof(T) == 8 ? 16 : 32;
};
constexpr int kXLoadBufs = 3;

// Dynamic shared memory of one block: kXLoadBufs buffers of load tiles and
// two of output tiles, 32 rows of XChunkPair + 1 elements each.
template <typename T>
size_t ordered_x_pair_smem(int n_loads, int n_out) {
  return (size_t)(kXLoadBufs * n_loads + 2 * n_out) * 32 * (XChunkPair<T>::value + 1) * sizeof(T);
}

template <typename T, bool INC, class S>
__global__ void __launch_bounds__(64) ordered_x_pair_kernel(const __grid_constant__ OrdParams P) {
  using A = typename Arith<T>::A;
  constexpr int KC = XChunkPair<T>::value;
  constexpr int TS = KC + 1;     // row stride of a tile
  constexpr int TILE = 32 * TS;  // one load's or one output's tile: 32 rows
  constexpr int RPI = 32 / KC;   // rows covered by one copy instruction of the mover
  extern __shared__ __align__(16) unsigned char oxp_smem[];
  // element offset of row r's first element (x = 0) in load l's grid, with
  // the load's offset, at [l][r]; output m's at [kLoads + m][r]
  __shared__ int64_t rbase[kLoads + kMaxOut_][32];
  const int lane = threadIdx.x & 31;
  const bool mover = threadIdx.x >= 32;
  const int nl = P.n_loads, no = P.n_out;
  T *lt = reinterpret_cast<T *>(oxp_smem);          // load tiles: [buffer][load]
  T *ot = lt + (size_t)kXLoadBufs * nl * TILE;     // output tiles: [buffer][output]
  const int64_t ny = P.hi[1] - P.lo[1], rows = ny * (P.hi[2] - P.lo[2]);
  const int64_t row0 = (int64_t)blockIdx.x * 32;
  if (row0 >= rows) return;  // the whole block
  const int64_t my = row0 + lane;
  const bool live = my < rows;
  const int64_t yl = live ? P.lo[1] + my % ny : 0, zl = live ? P.lo[2] + my / ny : 0;
  const int64_t len = P.hi[0] - P.lo[0];
  A prev[kMaxOut_];
#pragma unroll
  for (int m = 0; m < kMaxOut_; ++m) prev[m] = A(0);
  if (mover) {
    for (int l = 0; l < nl; ++l) {
      const OrdLoad &ld = P.loads[l];
      rbase[l][lane] = (zl + ld.dz) * P.in_plane[ld.grid] + (yl + ld.dy) * P.in_pitch[ld.grid] + ld.dx;
    }
    for (int m = 0; m < no; ++m) rbase[kLoads + m][lane] = zl * P.out_plane[m] + yl * P.out_pitch[m];
    __syncwarp();
  } else {
#pragma unroll
    for (int m = 0; m < kMaxOut_; ++m)
      if (live && m < no && P.need_prev[m])
        prev[m] = to_arith(reinterpret_cast<const T *>(P.out[m])[zl * P.out_plane[m] + yl * P.out_pitch[m] +
                                                                   (INC ? P.lo[0] - 1 : P.hi[0])]);
  }
  const int nrows = (int)min((int64_t)32, rows - row0);
  const int64_t nchunks = (len + KC - 1) / KC;
  // chunk c: its length and its lowest x; step j of the chunk is element
  // e = j (increasing) or e = clen - 1 - j (decreasing) of it
  auto chunk = [&](int64_t c, int &clen) -> int64_t {
    const int64_t c0 = c * KC;
    clen = (int)min((int64_t)KC, len - c0);
    return INC ? P.lo[0] + c0 : P.hi[0] - c0 - clen;
  };
  // mover lane: row rr0 + lane / KC of a group of RPI rows, element lane % KC
  const int lr = lane / KC, le = lane % KC;
  // mover: stages chunk c of every load into load buffer c % kXLoadBufs (one
  // commit group)
  auto issue = [&](int64_t c) {
    int clen;
    const int64_t xs = chunk(c, clen);
    T *buf = lt + (size_t)(c % kXLoadBufs) * nl * TILE;
    for (int l = 0; l < nl; ++l) {
      const T *g = reinterpret_cast<const T *>(P.in[P.loads[l].grid]) + xs;
      T *tl = buf + l * TILE;
#pragma unroll 8
      for (int r0 = 0; r0 < nrows; r0 += RPI) {
        const int rr = r0 + lr;
        if (rr < nrows && le < clen) {
          const T *src = g + rbase[l][rr] + le;
          T *d = tl + rr * TS + (INC ? le : clen - 1 - le);
          if constexpr (sizeof(T) >= 4) cp_async(d, src, (int)sizeof(T));
          else *d = *src;
        }
      }
    }
    if constexpr (sizeof(T) >= 4) cp_async_commit();
  };
  // mover: writes chunk c of every output back from output buffer c & 1
  auto store = [&](int64_t c) {
    int clen;
    const int64_t xs = chunk(c, clen);
    const T *buf = ot + (size_t)(c & 1) * no * TILE;
    for (int m = 0; m < no; ++m) {
      T *g = reinterpret_cast<T *>(P.out[m]) + xs;
      const T *to = buf + m * TILE;
#pragma unroll 8
      for (int r0 = 0; r0 < nrows; r0 += RPI) {
        const int rr = r0 + lr;
        if (rr < nrows && le < clen) g[rbase[kLoads + m][rr] + le] = to[rr * TS + (INC ? le : clen - 1 - le)];
      }
    }
  };
  if (mover) {
    issue(0);
    if (nchunks > 1) {
      issue(1);
      if constexpr (sizeof(T) >= 4) cp_async_wait<1>();  // chunk 0 has landed
    } else if constexpr (sizeof(T) >= 4) {
      cp_async_wait<0>();
    }
  }
  __syncthreads();
  // Both warps pass the same barriers: one before the loop and one per chunk.
  for (int64_t c = 0; c < nchunks; ++c) {
    int clen;
    chunk(c, clen);
    if (mover) {
      // load buffer (c + 2) % 3 was last read by the compute of chunk c - 1,
      // output buffer (c - 1) & 1 written by it: both finished before the
      // barrier that ended the previous chunk
      if (c + 2 < nchunks) issue(c + 2);
      if (c >= 1) store(c - 1);
      if constexpr (sizeof(T) >= 4) {
        if (c + 2 < nchunks) cp_async_wait<1>();  // chunk c + 1 has landed
        else cp_async_wait<0>();
      }
    } else {
      if (live) {
        const T *r = lt + (size_t)(c % kXLoadBufs) * nl * TILE + lane * TS;
        T *o_t = ot + (size_t)(c & 1) * no * TILE + lane * TS;
        if constexpr (!std::is_same<S, OrdInterpretedX>::value) {
          // compiled recurrence: every term's slot a constant.  One step reads
          // the staged value of load slot l as val(l) and leaves output m's
          // element in y[m].
          auto step = [&](auto val, T (&y)[S::NOUT]) {
            A v = A(0);
            A o[S::NOUT];
#pragma unroll
            for (int m = 0; m < S::NOUT; ++m) o[m] = A(0);
            static_for<S::NT>([&](auto tc) {
              constexpr int t = decltype(tc)::value;
              constexpr OrdShapeTerm st = S::table.t[t];
              A x;
              if constexpr (st.xs == kSrcValue) x = v;
              else if constexpr (st.xs >= kSrcPrev) x = prev[st.xs - kSrcPrev];
              else x = val(st.xs);
              if constexpr (st.cs >= 0) x = x * val(st.cs);
              const A wgt = ord_weight(P.terms[t], A(0));
              if constexpr (st.out < 0) v = fma(wgt, x, v);
              else o[st.out] = fma(wgt, x, o[st.out]);
            });
#pragma unroll
            for (int m = 0; m < S::NOUT; ++m) {
              y[m] = from_arith<T>(o[m]);
              prev[m] = to_arith(y[m]);
            }
          };
          if (clen == KC) {
            // groups of G steps: the next group's staged values are read into
            // registers before this group is computed (the reads are not held
            // behind this group's output writes), and a group's outputs are
            // written to the tile together
            constexpr int G = 8;
            A cur[S::NL][G], nxt[S::NL][G];
            auto fetch = [&](int s0, A(&d)[S::NL][G]) {
#pragma unroll
              for (int l = 0; l < S::NL; ++l)
#pragma unroll
                for (int g = 0; g < G; ++g) d[l][g] = to_arith(r[l * TILE + s0 + g]);
            };
            fetch(0, cur);
#pragma unroll
            for (int s0 = 0; s0 < KC; s0 += G) {
              if (s0 + G < KC) fetch(s0 + G, nxt);
              T ys[G][S::NOUT];
#pragma unroll
              for (int g = 0; g < G; ++g) step([&](int l) { return cur[l][g]; }, ys[g]);
#pragma unroll
              for (int g = 0; g < G; ++g)
#pragma unroll
                for (int m = 0; m < S::NOUT; ++m) o_t[m * TILE + s0 + g] = ys[g][m];
#pragma unroll
              for (int l = 0; l < S::NL; ++l)
#pragma unroll
                for (int g = 0; g < G; ++g) cur[l][g] = nxt[l][g];
            }
          } else {
            for (int s = 0; s < clen; ++s) {
              T y[S::NOUT];
              step([&](int l) { return to_arith(r[l * TILE + s]); }, y);
#pragma unroll
              for (int m = 0; m < S::NOUT; ++m) o_t[m * TILE + s] = y[m];
            }
          }
        } else {
          for (int s = 0; s < clen; ++s) {
            A v = A(0);
            A o[kMaxOut_];
#pragma unroll
            for (int m = 0; m < kMaxOut_; ++m) o[m] = A(0);
            for (int t = 0; t < P.n_terms; ++t) {
              const OrdTerm &tm = P.terms[t];
              A x = v;
              if (tm.prev >= 0) {
                x = prev[0];
#pragma unroll
                for (int m = 1; m < kMaxOut_; ++m)
                  if (tm.prev == m) x = prev[m];
              } else if (tm.xslot >= 0) {
                x = to_arith(r[tm.xslot * TILE + s]);
              }
              if (tm.cslot >= 0) x = x * to_arith(r[tm.cslot * TILE + s]);
              const A wgt = ord_weight(tm, A(0));
              if (tm.out < 0) {
                v = fma(wgt, x, v);
              } else {
#pragma unroll
                for (int m = 0; m < kMaxOut_; ++m)
                  if (tm.out == m) o[m] = fma(wgt, x, o[m]);
              }
            }
#pragma unroll
            for (int m = 0; m < kMaxOut_; ++m) {
              if (m < no) {
                const T y = from_arith<T>(o[m]);
                o_t[m * TILE + s] = y;
                prev[m] = to_arith(y);
              }
            }
          }
        }
      }
    }
    __syncthreads();
  }
  if (mover && nchunks > 0) store(nchunks - 1);
}

template <typename T, class S>
gscl_status launch_ordered_x_s(const OrdParams &P, bool inc, long long rows, cudaStream_t st) {
  const unsigned blocks = (unsigned)((rows + 31) / 32);
  size_t smem;
  int threads;
  void (*kern)(const OrdParams);
  if constexpr (sizeof(T) == 8) {
    smem = ordered_x_pair_smem<T>(P.n_loads, P.n_out);
    threads = 64;
    kern = inc ? ordered_x_pair_kernel<T, true, S> : ordered_x_pair_kernel<T, false, S>;
  } else {
    smem = ordered_x_smem<T>(P.n_loads, P.n_out);
    threads = 32;
    kern = inc ? ordered_x_kernel<T, true, S> : ordered_x_kernel<T, false, S>;
  }
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "ordered kernel set-up");
  }
  kern<<<blocks, threads, smem, st>>>(P);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GSCL_OK : cuda_fail(e, "ordered kernel launch");
}

// shape: a compiled recurrence (>= 0) or the interpreted term loop
template <typename T>
gscl_status launch_ordered_x(const OrdParams &P, int shape, bool inc, long long rows, cudaStream_t st) {
  if (P.n_loads > kLoads)
    return fail(GSCL_ERR_UNSUPPORTED, "ordered iteration along x takes at most %d distinct loads per element", kLoads);
  switch (shape) {
    case ORD_RUNSUM_PREV_FIRST: return launch_ordered_x_s<T, OrdRunSumPrevFirst>(P, inc, rows, st);
    case ORD_RUNSUM: return launch_ordered_x_s<T, OrdRunSum>(P, inc, rows, st);
    case ORD_BIDIAG: return launch_ordered_x_s<T, OrdBidiag>(P, inc, rows, st);
    case ORD_BIDIAG_PREV_FIRST: return launch_ordered_x_s<T, OrdBidiagPrevFirst>(P, inc, rows, st);
    case ORD_AXPY2: return launch_ordered_x_s<T, OrdAxpy2>(P, inc, rows, st);
  }
  return launch_ordered_x_s<T, OrdInterpretedX>(P, inc, rows, st);
}

template <typename T>
gscl_status launch_ordered_t(const OrdParams &P, int shape, int axis, bool inc, long long cols, cudaStream_t st) {
  if (axis == 0) return launch_ordered_x<T>(P, shape, inc, cols, st);
  if (axis == 2)
    return inc ? launch_ordered_dir<T, 2, true>(P, shape, cols, st) : launch_ordered_dir<T, 2, false>(P, shape, cols, st);
  return inc ? launch_ordered_dir<T, 1, true>(P, shape, cols, st) : launch_ordered_dir<T, 1, false>(P, shape, cols, st);
}

// Binds the call and fills the kernel parameters (shared by gscl_do_ordered
// and gscl_ordered_specialization).
struct OrdCall {
  OrdParams P;
  int axis;
  bool inc, empty;
  long long cols;
  gscl_dtype dtype;
};


}  // namespace
}  // namespace gscl

using namespace gscl;

namespace gscl {
namespace {

gscl_status prepare_ordered(int32_t order, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                            const gscl_grid *out, int32_t n_out, const gscl_range *range, OrdCall *c) {
  if (order < GSCL_I_INC || order > GSCL_K_DEC) return fail(GSCL_ERR_INVALID, "unknown order %d", order);
  const int axis = order / 2;
  const bool inc = order % 2 == 0;
  if (!op) return fail(GSCL_ERR_INVALID, "do_ordered needs an operator");
  if (n_out < 1) return fail(GSCL_ERR_INVALID, "do_ordered needs an output");
  Bound b;
  if (gscl_status s = bind(op, false, in, n_in, out, n_out, range, &b, axis, inc ? -1 : 1)) return s;
  memset(c, 0, sizeof *c);
  c->axis = axis;
  c->inc = inc;
  c->empty = b.empty;
  c->dtype = (gscl_dtype)b.in[0].dtype;
  if (b.empty) return GSCL_OK;
  OrdParams &P = c->P;
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
  // distinct element loads of one step (inputs at their offsets, coefficients
  // at the element) for the pipelined path
  int nl = 0;
  auto slot_of = [&](int grid, int dx, int dy, int dz, int nc) -> int {
    for (int l = 0; l < nl && l < kLoads; ++l) {
      const OrdLoad &q = P.loads[l];
      if (q.grid == grid && q.dx == dx && q.dy == dy && q.dz == dz) return l;
    }
    if (nl < kLoads) P.loads[nl] = OrdLoad{(int16_t)grid, (int16_t)nc, (int16_t)dx, (int16_t)dy, (int16_t)dz, 0};
    return nl++;
  };
  for (int t = 0; t < nt; ++t) {
    OrdTerm &d = P.terms[t];
    d.xslot = (d.in >= 0 && d.prev < 0) ? (int16_t)slot_of(d.in, d.dx, d.dy, d.dz, d.nc) : (int16_t)-1;
    d.cslot = d.coef >= 0 ? (int16_t)slot_of(d.coef, 0, 0, 0, d.cnc) : (int16_t)-1;
  }
  P.n_loads = nl;
  // element offsets along the column: first step a0, direction +-1 per step
  const int64_t a0 = inc ? b.lo[axis] : b.hi[axis] - 1, dir = inc ? 1 : -1;
  for (int l = 0; l < nl && l < kLoads; ++l) {
    OrdLoad &ld = P.loads[l];
    const Grid &g = b.in[ld.grid];
    const int64_t S = axis == 2 ? g.plane : g.pitch;
    ld.start = (int64_t)ld.dz * g.plane + (int64_t)ld.dy * g.pitch + ld.dx + a0 * S;
    ld.step = dir * S;
  }
  for (int m = 0; m < n_out; ++m) {
    const Grid &g = b.out[m];
    const int64_t S = axis == 2 ? g.plane : g.pitch;
    P.out_start[m] = a0 * S;
    P.out_step[m] = dir * S;
  }
  for (int a = 0; a < 3; ++a) {
    P.lo[a] = b.lo[a];
    P.hi[a] = b.hi[a];
  }
  const int other = axis == 2 ? 1 : 2;
  c->cols = axis == 0 ? (long long)(b.hi[1] - b.lo[1]) * (b.hi[2] - b.lo[2])  // rows along x
                      : (long long)(b.hi[0] - b.lo[0]) * (b.hi[other] - b.lo[other]);
  return GSCL_OK;
}

}  // namespace
}  // namespace gscl

extern "C" gscl_status gscl_do_ordered(int32_t order, const gscl_stencil *op, const gscl_grid *in, int32_t n_in,
                                       const gscl_grid *out, int32_t n_out, const gscl_range *range, void *stream) {
  OrdCall c;
  if (gscl_status s = prepare_ordered(order, op, in, n_in, out, n_out, range, &c)) return s;
  if (c.empty) return GSCL_OK;
  const int shape = ordered_shape(c.P, c.dtype);
  cudaStream_t st = (cudaStream_t)stream;
  switch (c.dtype) {
    case GSCL_F64: return launch_ordered_t<double>(c.P, shape, c.axis, c.inc, c.cols, st);
    case GSCL_F32: return launch_ordered_t<float>(c.P, shape, c.axis, c.inc, c.cols, st);
    case GSCL_BF16: return launch_ordered_t<__nv_bfloat16>(c.P, shape, c.axis, c.inc, c.cols, st);
  }
  return fail(GSCL_ERR_DTYPE, "unknown dtype");
}

extern "C" gscl_status gscl_ordered_specialization(int32_t order, const gscl_stencil *op, const gscl_grid *in,
                                                   int32_t n_in, const gscl_grid *out, int32_t n_out,
                                                   int32_t *shape) {
  if (!shape) return fail(GSCL_ERR_INVALID, "shape is NULL");
  OrdCall c;
  if (gscl_status s = prepare_ordered(order, op, in, n_in, out, n_out, nullptr, &c)) return s;
  if (c.axis == 0 && c.P.n_loads > kLoads)
    return fail(GSCL_ERR_UNSUPPORTED, "ordered iteration along x takes at most %d distinct loads per element", kLoads);
  const int sh = ordered_shape(c.P, c.dtype);
  *shape = c.axis == 0 && sh < 0 ? ORD_ROWS_X : sh;
  return GSCL_OK;
}
