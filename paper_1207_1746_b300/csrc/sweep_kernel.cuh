// Device side of the do_all / do_reduce sweep (Section 3 iteration spaces).
//
// One kernel serves every dtype, operator and grid shape.  A CTA owns an
// xy tile of TX x TY core elements (TX = 32 * VX, VY adjacent rows per warp,
// lane l of a warp computing x = l, l + 32, ..., so every shared-memory read
// of a term is 32 consecutive elements: conflict-free) and streams along z
// through a chunk of planes (2.5D blocking).  For every input grid it keeps
// a ring of R plane boxes of (TX + 2 AX) x (TY + 2 RY) elements in shared
// memory, filled by TMA (cp.async.bulk.tensor) from HBM ahead of use and
// completed on one mbarrier per ring slot; R = 2 rz + 1 + prefetch.  Each
// input is therefore read from HBM once per sweep (plus the halo overlap
// between tiles, which L2 absorbs), outputs are written once with coalesced
// stores, and the operator's returned value is reduced in registers without
// touching memory (fused sweep + reduce).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include <mutex>
#include <type_traits>
#include <utility>

#include "fp64_int.cuh"
#include "gscl_internal.h"
#include "pair64.cuh"
#include "static_ops.h"

namespace gscl {

constexpr int kMaxTerms = GSCL_MAX_TERMS;
constexpr int kMaxIn = GSCL_MAX_IN;
constexpr int kMaxOut_ = GSCL_MAX_OUT;
constexpr int kBarBytes = 256;                   // up to 32 ring-slot mbarriers
constexpr int kMaxRing = kBarBytes / 8 - 2;      // the last two serve the centre ring
constexpr long long kWaitCycles = 4000000000LL;  // ~2 s at 2 GHz: bounded mbarrier waits
constexpr int kMaxReduceCtas = 65536;
constexpr int64_t kWorkspaceBytes = 256 + 16LL * kMaxReduceCtas;

enum RedKind { RED_NONE = 0, RED_SUM = 1, RED_MAXABS = 2, RED_L2 = 3 };

// A term as the kernel sees it: ring indices instead of grid ids, and the
// read offset pre-folded into an element offset inside one ring slot.
struct DevTerm {
  int16_t in;    // input ring, or -1: the operator's value
  int16_t coef;  // input ring of the coefficient, or -1
  int16_t dz;
  int16_t pad;
  int32_t toff;  // (RY_in + dy) * BW_in + AX_in + dx, in the read input's box
  float wf;
  double wd;
  float wl;      // pair arithmetic: the weight's low part, wd - (double)wf
  int32_t pad2;
};

struct OutDesc {
  char *base;     // address of interior element (0,0,0)
  int64_t pitch;  // elements
  int64_t plane;  // elements
};

// Everything that differs between grid sets of one operator: a single-grid
// launch carries one in its parameters, a batched launch a device table of
// them (one per instance).  Aligned as strictly as its tensor maps.
struct InstDesc {
  CUtensorMap tmap[kMaxIn];
  OutDesc out[kMaxOut_];
  OutDesc in[kMaxIn];        // the inputs' interior (0,0,0) addresses, for direct loads
  int64_t lo[3], hi[3];
  int64_t x_base, y_base;
  int32_t tiles_x, tiles_y;  // xy tiles covering the range
  int32_t cx_add[kMaxIn], cy_add[kMaxIn], cz_add[kMaxIn];
};

// One entry of a batched launch's work-list: planes [zoff, zoff + zlen) of
// tile column `col` of instance `inst`.
struct Segment {
  int32_t inst, col, zoff, zlen;
};

// The term weights of one instance of a batch, in the order of the launch's
// term table (a batch's instances share the operator's structure; coloured
// batches give each instance its own weights, e.g. its own SOR factor).
struct InstWeights {
  double wd[kMaxTerms];
  float wf[kMaxTerms];
  float wl[kMaxTerms];  // pair arithmetic: wd - (double)wf
  int32_t eq;           // equal axial weights: the axial-sum evaluation (StaticOp<Def, XS, true>)
};

struct SweepParams {
  InstDesc inst;             // single-grid launches
  DevTerm terms[kMaxTerms];
  int32_t n_in, n_out, n_value_terms;
  int32_t out_begin[kMaxOut_ + 1];
  int32_t R, rz;      // ring slots (planes) per input, z reach of the operator
  // per input: plane box width / height, x apron (rounded to 16 bytes), y
  // reach, element offset of its ring in shared memory and slot size
  int32_t in_bw[kMaxIn], in_bh[kMaxIn], in_ax[kMaxIn], in_ry[kMaxIn], in_base[kMaxIn], in_se[kMaxIn];
  uint32_t tx_bytes;  // bytes one plane delivers over all ring inputs
  // centre-ring inputs (read only at the core element; compile-time operators):
  // two slots of one TX x TY box each, at in_base[a] + slot * in_se[a]
  uint32_t cmask;
  uint32_t ctx_bytes;  // bytes one centre-ring slot receives over all such inputs
  int32_t zalt;       // launch a whole multiple of the tile columns (one z range per CTA)
  // batched launches: CTA b runs segments [cta_seg[b], cta_seg[b + 1])
  const InstDesc *insts;
  const InstWeights *inst_w; // one row of weights per instance
  const Segment *segs;
  const int32_t *cta_seg;
  double *seg_partials;      // batched reduce: one (s, c) pair per segment
  unsigned char *workspace;  // single reduce: ticket at +0, partials at +256
  double *result;            // single reduce: where the last CTA writes the value
  double within;             // >= 0: MAXABS reports 1 if max |value| <= within, else 0
  int32_t color;             // 0 / 1: outputs written only where (i + j + k) % 2 == color; -1: everywhere
  int *err;                  // device error word
};

template <typename T> struct Arith;
template <> struct Arith<double> { using A = double; };
template <> struct Arith<float> { using A = float; };
template <> struct Arith<__nv_bfloat16> { using A = float; };
template <> struct Arith<f64pair> { using A = Df64; };

// Storage types held as FP64 in memory (IEEE or pair arithmetic).
template <typename T> struct IsFp64Storage { static constexpr bool value = false; };
template <> struct IsFp64Storage<double> { static constexpr bool value = true; };
template <> struct IsFp64Storage<f64pair> { static constexpr bool value = true; };

__device__ __forceinline__ double to_arith(double x) { return x; }
__device__ __forceinline__ float to_arith(float x) { return x; }
__device__ __forceinline__ float to_arith(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ Df64 to_arith(f64pair x) { return split_f64(x.v); }

template <typename T> __device__ __forceinline__ T from_arith(typename Arith<T>::A x);
template <> __device__ __forceinline__ double from_arith<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_arith<float>(float x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_arith<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ f64pair from_arith<f64pair>(Df64 x) { return f64pair{combine_f64(x)}; }

__device__ __forceinline__ double term_weight(const DevTerm &t, double) { return t.wd; }
__device__ __forceinline__ float term_weight(const DevTerm &t, float) { return t.wf; }
__device__ __forceinline__ Df64 term_weight(const DevTerm &t, Df64) { return Df64(t.wf, t.wl); }
__device__ __forceinline__ double inst_weight(const InstWeights &w, int i, double) { return w.wd[i]; }
__device__ __forceinline__ float inst_weight(const InstWeights &w, int i, float) { return w.wf[i]; }
__device__ __forceinline__ Df64 inst_weight(const InstWeights &w, int i, Df64) { return Df64(w.wf[i], w.wl[i]); }

// Where the operator's weights come from.  Single-grid launches read them
// from the launch parameters.  Batched launches read the row of the
// instance being swept, once per segment: into registers for compile-time
// operators (N terms, constant indices), through a pointer for the
// interpreted term list.
template <typename A>
struct ParamWeights {
  __device__ __forceinline__ void load(const InstWeights *) {}
  __device__ __forceinline__ A operator()(const SweepParams &P, int i) const { return term_weight(P.terms[i], A(0)); }
  // single grids: the axial-sum kernel is launched only for equal weights
  __device__ static constexpr bool eq() { return true; }
};
template <typename A, int N, bool DYN = false>
struct RegWeights {
  A v[N];
  bool e;
  __device__ __forceinline__ void load(const InstWeights *w) {
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = inst_weight(*w, i, A(0));
    if constexpr (DYN) e = w->eq != 0;
  }
  __device__ __forceinline__ A operator()(const SweepParams &, int i) const { return v[i]; }
  // the group evaluation: per instance (DYN: a coloured batch mixing
  // instances whose weights allow it and instances whose weights do not),
  // else for every instance of the batch
  __device__ __forceinline__ bool eq() const {
    if constexpr (DYN) return e;
    else return true;
  }
};
template <typename A>
struct RowWeights {
  const InstWeights *w = nullptr;
  __device__ __forceinline__ void load(const InstWeights *row) { w = row; }
  __device__ __forceinline__ A operator()(const SweepParams &, int i) const { return inst_weight(*w, i, A(0)); }
};

// ------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete; gives up after
// kWaitCycles and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > kWaitCycles) return false;
  }
  return true;
}

// Programmatic dependent launch: a grid launched with the programmatic
// serialisation attribute may start while the previous grid on its stream is
// still running.  launch_dependents lets the next grid begin launching;
// wait blocks until every prerequisite grid has completed and its memory is
// visible (a no-op for a grid launched without the attribute).
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Calls f(std::integral_constant<int, i>) for i = 0 .. N-1 (a loop whose
// index is a compile-time constant in the body).
template <class F, int... I>
__device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F &&f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// --------------------------------------------------------------- reduction
// FP64 accumulation of the per-element values.  Within one z-step a thread
// first adds its VX values in plain FP64, then folds that group sum into a
// Kahan-compensated running sum (s, c) whose true value is s - c; threads
// and CTAs are merged with Knuth's error-free TwoSum so the compensation
// survives the tree.
struct Compensated {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double y = x - c;
    const double t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// (s, c) += (s2, c2) for values s - c and s2 - c2.
__device__ __forceinline__ void combine_pair(double &s, double &c, double s2, double c2) {
  const double t = s + s2;
  const double bp = t - s;
  const double err = (s - (t - bp)) + (s2 - bp);  // t + err == s + s2 exactly
  s = t;
  c = (c + c2) - err;
}

// Knuth's TwoSum: t + err == a + b exactly.  The _rn intrinsics are never
// contracted into FMAs, which would break the error-free steps.
__device__ __forceinline__ void two_sum(float a, float b, float &t, float &err) {
  t = __fadd_rn(a, b);
  const float bp = __fsub_rn(t, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bp)), __fsub_rn(b, bp));
}

// Knuth's TwoSum on two independent lanes at once (the sm_100-family packed
// FP32 add, each lane exactly one __fadd_rn).  Subtraction is an add of the
// negated operand, which is exact.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &t, float2 &err) {
  t = __fadd2_rn(a, b);
  const float2 bp = __fadd2_rn(t, neg2(a));
  err = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(b, neg2(bp)));
}

// Sum of squares of FP32 values on the FP32 pipe (the L2 reduction of FP32 /
// BF16 sweeps), as two unevaluated pairs hi + lo (even and odd elements of a
// group, two independent chains held as the two lanes of packed registers).
// Each square is formed exactly as p + pe (the product, and its rounding
// error from one FMA: exact while |x| lies in [2^-50, 2^50], which the
// caller checks) and added with Knuth's error-free TwoSum, the errors going
// to lo.  The products are scalar, non-contractible intrinsics, and the sums
// packed adds, so no multiply can be fused into an error-free step.
// renormalize() keeps |lo| within an ulp of hi; the pairs are folded chain
// to chain, across the warp and into FP64 only at the end of a reduction,
// so the narrow FP64 pipe sees a few operations per warp instead of one FMA
// per element.  Relative error of a sum of n squares: about (3 + n) 2^-48.
struct SquareSum32 {
  float2 hi = make_float2(0.0f, 0.0f), lo = make_float2(0.0f, 0.0f);
  __device__ __forceinline__ void add_squares(float a, float b) {
    const float pa = __fmul_rn(a, a), pb = __fmul_rn(b, b);
    const float2 p = make_float2(pa, pb);
    const float2 pe = make_float2(__fmaf_rn(a, a, -pa), __fmaf_rn(b, b, -pb));
    float2 t, err;
    two_sum2(hi, p, t, err);
    hi = t;
    lo = __fadd2_rn(lo, __fadd2_rn(err, pe));
  }
  __device__ __forceinline__ void renormalize() {
    const float2 t = __fadd2_rn(hi, lo);
    lo = __fadd2_rn(lo, neg2(__fadd2_rn(t, neg2(hi))));
    hi = t;
  }
  // folds chain 1 into chain 0
  __device__ __forceinline__ void fold_lanes() {
    float t, err;
    two_sum(hi.x, hi.y, t, err);
    hi.x = t;
    lo.x = __fadd_rn(__fadd_rn(lo.x, lo.y), err);
    hi.y = lo.y = 0.0f;
  }
  // FP64 values split as v = h + e (split_double): h^2 exactly as p + pe,
  // the cross term 2 h e rounded to a float and added with the errors;
  // e^2 < 2^-46 h^2 is dropped.  With e = 0 (every FP64 value of at most 24
  // significant bits, integers below 2^24 among them) this is add_squares.
  __device__ __forceinline__ void add_split_squares(float ha, float ea, float hb, float eb) {
    const float pa = __fmul_rn(ha, ha), pb = __fmul_rn(hb, hb);
    const float2 p = make_float2(pa, pb);
    const float2 pe = make_float2(__fmaf_rn(ha, ha, -pa), __fmaf_rn(hb, hb, -pb));
    const float2 c = make_float2(__fmul_rn(__fadd_rn(ha, ha), ea), __fmul_rn(__fadd_rn(hb, hb), eb));
    float2 t, err;
    two_sum2(hi, p, t, err);
    hi = t;
    lo = __fadd2_rn(lo, __fadd2_rn(__fadd2_rn(err, pe), c));
  }
  // adds another sum h + l into chain 0
  __device__ __forceinline__ void add_sum(float h, float l) {
    float t, err;
    two_sum(hi.x, h, t, err);
    hi.x = t;
    lo.x = __fadd_rn(lo.x, __fadd_rn(l, err));
  }
};

// FP64 values on the FP32 pipe (the L2 reduction of IEEE FP64 sweeps, whose
// FP64 pipe binds): v = h + e with h its 24 leading significand bits (the
// truncation, a float, exact) and e the rest rounded to a float (relative
// error 2^-24 of a term below 2^-23 |v|), both taken apart with integer
// operations.  In range when 2^-50 <= |v| < 2^50 (biased exponent 973 ..
// 1072, so h, e and the squares' error terms stay representable) or v == 0;
// other values (an infinity, a NaN, a subnormal) take the FP64 chain.
__device__ __forceinline__ bool split_in_range(double v) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const uint32_t ex = (hi >> 20) & 0x7ffu;
  return ex - 973u < 100u || ((hi & 0x7fffffffu) | lo) == 0u;
}
__device__ __forceinline__ void split_double(double v, float &h, float &e) {
  const uint32_t hi = (uint32_t)__double2hiint(v), lo = (uint32_t)__double2loint(v);
  const uint32_t ex = (hi >> 20) & 0x7ffu, sign = hi & 0x80000000u;
  // float exponent field ex - 896 (bias 1023 -> 127); 23 fraction bits: the
  // double's top 20 and 3 more
  const float hv = __uint_as_float(sign | ((ex - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
  // the remaining 29 bits, times 2^(ex - 1075) (exponent field ex - 948)
  const float ev = __uint_as_float(
      __float_as_uint(__fmul_rn(__uint2float_rn(lo & 0x1fffffffu), __uint_as_float((ex - 948u) << 23))) | sign);
  h = ex != 0u ? hv : 0.0f;
  e = ex != 0u ? ev : 0.0f;
}

__device__ __forceinline__ double max_abs_bits(double a, double b) {
  return __longlong_as_double(
      (long long)max((unsigned long long)__double_as_longlong(a), (unsigned long long)__double_as_longlong(b)));
}

// ---------------------------------------------------------------- operators
// An operator policy evaluates the operator for the VX points a thread owns
// at the current z step: v receives the returned value, o[m] output m.
// ring: shared-memory ring of input planes; smod: ring slot of the current
// plane; thr: this thread's element offset inside a slot.

// Runtime term list (any descriptor the ABI accepts).
struct GenericOp {
  static constexpr int kMaxOut = kMaxOut_;
  static constexpr int kQueue = 1;  // no z register queue (size of the unused array)
  static constexpr int kXStep = 1;  // a thread's columns: lane + 32 e
  static constexpr int kGroup = 1;  // columns strided by 32, not grouped (see StaticOpV)
  static constexpr int kRowsPerSlot = 1;
  static constexpr int kTerms = kMaxTerms;
  template <typename A, bool BATCH>
  using Weights = typename std::conditional<BATCH, RowWeights<A>, ParamWeights<A>>::type;
  __device__ static int n_out(const SweepParams &P) { return P.n_out; }

  template <typename T, int VX, int VY>
  __device__ static __forceinline__ void advance_queue(const SweepParams &, const T *, int, int, int, bool,
                                                       typename Arith<T>::A (&)[kQueue][VY][VX]) {}

  template <typename T, int VX, int VY, int r, class WS>
  __device__ static __forceinline__ void eval_row(const SweepParams &P, const WS &ws, const T *ring, int smod,
                                                  int cslot, int row0, int lane,
                                                  const typename Arith<T>::A (&)[kQueue][VY][VX],
                                                  typename Arith<T>::A (&v)[VX],
                                                  typename Arith<T>::A (&o)[kMaxOut][VX]) {
    eval<T, VX>(P, ws, ring, smod, cslot, row0 + r, lane, v, o);
  }

  template <typename T, int VX, class WS>
  __device__ static __forceinline__ void term(const SweepParams &P, const WS &ws, int ti, const T *ring, int smod,
                                              int row, int lane, const typename Arith<T>::A (&v)[VX],
                                              typename Arith<T>::A (&acc)[VX]) {
    using A = typename Arith<T>::A;
    const int R = P.R;
    const DevTerm &tm = P.terms[ti];
    const A w = ws(P, ti);
    A x[VX];
    if (tm.in < 0) {
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = v[e];
    } else {
      int slot = smod + tm.dz;
      slot = slot >= R ? slot - R : (slot < 0 ? slot + R : slot);
      const T *p = ring + P.in_base[tm.in] + slot * P.in_se[tm.in] + row * P.in_bw[tm.in] + lane + tm.toff;
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = to_arith(p[32 * e]);
    }
    if (tm.coef >= 0) {
      const int c = tm.coef;
      const T *cp = ring + P.in_base[c] + smod * P.in_se[c] + (row + P.in_ry[c]) * P.in_bw[c] + P.in_ax[c] + lane;
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = x[e] * to_arith(cp[32 * e]);
    }
#pragma unroll
    for (int e = 0; e < VX; ++e) acc[e] = fma(w, x[e], acc[e]);
  }

  template <typename T, int VX, class WS>
  __device__ static __forceinline__ void eval(const SweepParams &P, const WS &ws, const T *ring, int smod, int,
                                              int row, int lane, typename Arith<T>::A (&v)[VX],
                                              typename Arith<T>::A (&o)[kMaxOut][VX]) {
    for (int t = 0; t < P.n_value_terms; ++t) term<T, VX>(P, ws, t, ring, smod, row, lane, v, v);
#pragma unroll
    for (int m = 0; m < kMaxOut; ++m)
      if (m < P.n_out)
        for (int t = P.out_begin[m]; t < P.out_begin[m + 1]; ++t)
          term<T, VX>(P, ws, t, ring, smod, row, lane, v, o[m]);
  }
};

// Compile-time term table (static_ops.h).  Term i's weight is P.terms[i]:
// the host stores the matched descriptor's weights in table order.
//
// XS = 2 is the colour-compacted evaluation of red-black sweeps (FP64): a
// warp covers 64 VX columns and a thread only the elements of the launch's
// colour, x = x0 + col + 64 e with col = 2 lane + the row's parity offset.
// The kernel passes col for the warp's first row as `lane`; row r flips its
// low bit (the warp's rows start at an even row).  The column changes from
// plane to plane, so there is no z register queue and no centre ring.
//
// EQ = true (IEEE FP64 grids, XS = 1, chosen on the host when the axial
// group's six weights are bit-identical): the group is evaluated as its
// weight times axial_sum, w (sum of six) instead of six FMAs; two of the
// sum's five additions run on the integer pipe, so a point of the heat
// operator takes six FP64 operations instead of eight.
template <class Def, int XS = 1, bool EQ = false, bool DYN = false>
struct StaticOp {
  static constexpr int kXStep = XS;
  static constexpr int kAxial = EQ ? axial_group<Def>() : -1;
  // the group is evaluated after the last coefficient-free term of its
  // destination's block, so the other terms accumulate while its integer
  // additions run and one FMA follows the sum
  __host__ __device__ static constexpr int axial_at() {
    if (kAxial < 0) return -1;
    int j = kAxial + 5;
    while (j + 1 < Def::NT && Def::table.t[j + 1].out == Def::table.t[kAxial].out && Def::table.t[j + 1].coef < 0 &&
           Def::table.t[j + 1].in >= 0)
      ++j;
    return j;
  }
  static constexpr int kAxialAt = axial_at();
  static_assert(!EQ || has_groups<Def>(), "the group evaluation needs a term group");
  static constexpr int kGroup = 1;
  static constexpr int kRowsPerSlot = 1;
  static constexpr int kTerms = Def::NT;
  static constexpr int kMaxOut = Def::NOUT > 0 ? Def::NOUT : 1;
  template <typename A, bool BATCH>
  using Weights = typename std::conditional<BATCH, RegWeights<A, Def::NT, DYN>, ParamWeights<A>>::type;
  __device__ static constexpr int n_out(const SweepParams &) { return Def::NOUT; }

  // reach of the terms reading input `in` (-1: every input) along `axis`
  __host__ __device__ static constexpr int radius(int axis, int in = -1) {
    int r = 0;
    for (int i = 0; i < Def::NT; ++i) {
      const OpTerm &t = Def::table.t[i];
      if (t.in < 0 || (in >= 0 && t.in != in)) continue;
      const int d = axis == 0 ? t.dx : axis == 1 ? t.dy : t.dz;
      r = d > r ? d : (-d > r ? -d : r);
    }
    return r;
  }
  static constexpr int RZ = radius(2);

  // The z register queue: the one ring input whose centre column is read at
  // z offsets (the star / heat family's u) keeps that column for planes
  // z - RZ .. z + RZ in registers, so each step loads one new plane centre
  // from shared memory instead of 2 RZ + 1, and the y neighbours of a
  // thread's inner rows are its other rows' centres.  Operators with several
  // such inputs (the climate operator) read them all from shared memory.
  __host__ __device__ static constexpr int queue_input() {
    int found = -1, count = 0;
    for (int a = 0; a < Def::NIN; ++a) {
      bool zcol = false;
      for (int i = 0; i < Def::NT; ++i) {
        const OpTerm &t = Def::table.t[i];
        if (t.in == a && t.dx == 0 && t.dy == 0 && t.dz != 0) zcol = true;
      }
      if (zcol) {
        found = a;
        ++count;
      }
    }
    return count == 1 ? found : -1;
  }
  static constexpr int ZQ = XS == 1 ? queue_input() : -1;
  static constexpr int kQueue = ZQ >= 0 ? 2 * RZ + 1 : 1;

  // this thread's first column in tile row row0 + r (see XS above)
  __device__ static __forceinline__ int column(int lane, int r) { return XS == 1 ? lane : (lane ^ (r & 1)); }

  // centre of the queue input at ring slot `sl`, tile row row0 + r
  template <typename T, int VX>
  __device__ static __forceinline__ typename Arith<T>::A queue_load(const SweepParams &P, const T *ring, int sl,
                                                                    int row, int lane, int e) {
    constexpr int vec = 16 / (int)sizeof(T);
    constexpr int AXq = (radius(0, ZQ) + vec - 1) / vec * vec;
    constexpr int RYq = radius(1, ZQ);
    constexpr int BWq = 32 * VX + 2 * AXq;
    return to_arith(ring[P.in_base[ZQ] + sl * P.in_se[ZQ] + (row + RYq) * BWq + AXq + lane + 32 * e]);
  }

  // Step start: the queue holds planes z - RZ .. z + RZ (all loaded on the
  // first step of a z range, then shifted by one plane per step).
  template <typename T, int VX, int VY>
  __device__ static __forceinline__ void advance_queue(const SweepParams &P, const T *ring, int smod, int row0,
                                                       int lane, bool first,
                                                       typename Arith<T>::A (&zq)[kQueue][VY][VX]) {
    if constexpr (ZQ >= 0) {
      const int R = P.R;
      if (first) {
#pragma unroll
        for (int k = 0; k <= 2 * RZ; ++k) {
          int sl = smod + k - RZ;
          sl = sl >= R ? sl - R : (sl < 0 ? sl + R : sl);
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int e = 0; e < VX; ++e) zq[k][r][e] = queue_load<T, VX>(P, ring, sl, row0 + r, lane, e);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 2 * RZ; ++k)
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int e = 0; e < VX; ++e) zq[k][r][e] = zq[k + 1][r][e];
        int sl = smod + RZ;
        sl = sl >= R ? sl - R : sl;
#pragma unroll
        for (int r = 0; r < VY; ++r)
#pragma unroll
          for (int e = 0; e < VX; ++e) zq[2 * RZ][r][e] = queue_load<T, VX>(P, ring, sl, row0 + r, lane, e);
      }
    }
  }

  // A run: consecutive table terms with one coefficient grid and one
  // destination.  Its terms are summed first and the sum is multiplied by the
  // coefficient once (sum_t w_t X_t C = C sum_t w_t X_t): one multiply per run
  // instead of one per term.
  __host__ __device__ static constexpr bool same_run(int i, int j) {
    return Def::table.t[i].coef >= 0 && Def::table.t[i].coef == Def::table.t[j].coef &&
           Def::table.t[i].out == Def::table.t[j].out;
  }
  __host__ __device__ static constexpr bool run_first(int i) { return i == 0 || !same_run(i - 1, i); }
  __host__ __device__ static constexpr bool run_last(int i) { return i == Def::NT - 1 || !same_run(i, i + 1); }

  // Centre ring for every storage, and for IEEE FP64 only for operators with
  // kCentreFp64Min or more centre-only inputs (static_ops.h; the host planner
  // makes the same choice).
  template <typename T>
  __host__ __device__ static constexpr bool in_centre_ring(int in) {
    return XS == 1 && (!std::is_same<T, double>::value || centre_count<Def>() >= kCentreFp64Min) &&
           centre_only<Def>(in);
  }

  // element (row, lane) of centre-ring input `in` in slot cslot
  template <typename T, int VX>
  __device__ static __forceinline__ const T *centre_ptr(const SweepParams &P, const T *ring, int in, int cslot,
                                                        int row, int lane) {
    return ring + P.in_base[in] + cslot * P.in_se[in] + row * (32 * VX) + lane;
  }

  // The values term I reads at tile row row0 + r of this thread's VY rows
  // (v: the operator's value so far, for a term of the value).
  template <typename T, int VX, int VY, int r, int I>
  __device__ static __forceinline__ void load_x(const SweepParams &P, const T *ring, int smod, int cslot, int row0,
                                                int lane, const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                                const typename Arith<T>::A (&v)[VX],
                                                typename Arith<T>::A (&x)[VX]) {
    const int row = row0 + r;
    const int col = column(lane, r);
    constexpr int ES = 32 * XS;  // element stride of a thread's columns
    constexpr OpTerm t = Def::table.t[I];
    constexpr int vec = 16 / (int)sizeof(T);
    const int R = P.R;
    if constexpr (t.in < 0) {
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = v[e];
    } else if constexpr (in_centre_ring<T>(t.in)) {
      const T *p = centre_ptr<T, VX>(P, ring, t.in, cslot, row, lane);
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = to_arith(p[32 * e]);
    } else if constexpr (t.in == ZQ && t.dx == 0 && t.dy == 0) {
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = zq[t.dz + RZ][r][e];
    } else if constexpr (t.in == ZQ && t.dx == 0 && t.dz == 0 && r + t.dy >= 0 && r + t.dy < VY) {
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = zq[RZ][r + t.dy][e];
    } else {
      constexpr int RX = radius(0, t.in), RY = radius(1, t.in);
      constexpr int AX = (RX + vec - 1) / vec * vec;
      constexpr int BW = ES * VX + 2 * AX;
      constexpr int toff = (RY + t.dy) * BW + AX + t.dx;
      int slot = smod + t.dz;
      if constexpr (t.dz > 0) slot = slot >= R ? slot - R : slot;
      if constexpr (t.dz < 0) slot = slot < 0 ? slot + R : slot;
      const T *p = ring + P.in_base[t.in] + slot * P.in_se[t.in] + row * BW + col + toff;
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = to_arith(p[ES * e]);
    }
  }

  // The axial group's six values summed as ((x+ + x-) + (y+ + y-)) + (z+ + z-)
  // in table order of the pairs; the first two pair sums run on the integer
  // pipe (exact IEEE additions, fp64_int.cuh), the rest on the FP64 pipe.
  template <typename T, int VX, int VY, int r>
  __device__ static __forceinline__ void axial_sum(const SweepParams &P, const T *ring, int smod, int cslot, int row0,
                                                   int lane, const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                                   const typename Arith<T>::A (&v)[VX],
                                                   typename Arith<T>::A (&x)[VX]) {
    using A = typename Arith<T>::A;
    A x0[VX], x1[VX], x2[VX], x3[VX], x4[VX], x5[VX];
    load_x<T, VX, VY, r, kAxial + 0>(P, ring, smod, cslot, row0, lane, zq, v, x0);
    load_x<T, VX, VY, r, kAxial + 1>(P, ring, smod, cslot, row0, lane, zq, v, x1);
    load_x<T, VX, VY, r, kAxial + 2>(P, ring, smod, cslot, row0, lane, zq, v, x2);
    load_x<T, VX, VY, r, kAxial + 3>(P, ring, smod, cslot, row0, lane, zq, v, x3);
    load_x<T, VX, VY, r, kAxial + 4>(P, ring, smod, cslot, row0, lane, zq, v, x4);
    load_x<T, VX, VY, r, kAxial + 5>(P, ring, smod, cslot, row0, lane, zq, v, x5);
#pragma unroll
    for (int e = 0; e < VX; ++e) x[e] = (fp64_add_int(x0[e], x1[e]) + fp64_add_int(x2[e], x3[e])) + (x4[e] + x5[e]);
  }

  // A coefficient group's values combined: four as (x0 + x1) + (x2 + x3), a
  // pair as x0 - x1; the first addition (the difference) runs on the integer
  // pipe (exact IEEE arithmetic, fp64_int.cuh).
  template <typename T, int VX, int VY, int r, int G, int N>
  __device__ static __forceinline__ void coef_group_sum(const SweepParams &P, const T *ring, int smod, int cslot,
                                                        int row0, int lane,
                                                        const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                                        const typename Arith<T>::A (&v)[VX],
                                                        typename Arith<T>::A (&x)[VX]) {
    using A = typename Arith<T>::A;
    A x0[VX], x1[VX];
    load_x<T, VX, VY, r, G + 0>(P, ring, smod, cslot, row0, lane, zq, v, x0);
    load_x<T, VX, VY, r, G + 1>(P, ring, smod, cslot, row0, lane, zq, v, x1);
    if constexpr (N == 2) {
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = fp64_add_int(x0[e], -x1[e]);
    } else {
      A x2[VX], x3[VX];
      load_x<T, VX, VY, r, G + 2>(P, ring, smod, cslot, row0, lane, zq, v, x2);
      load_x<T, VX, VY, r, G + 3>(P, ring, smod, cslot, row0, lane, zq, v, x3);
#pragma unroll
      for (int e = 0; e < VX; ++e) x[e] = fp64_add_int(x0[e], x1[e]) + (x2[e] + x3[e]);
    }
  }

  // Term I at tile row row0 + r of this thread's VY rows.
  template <typename T, int VX, int VY, int r, int I, class WS>
  __device__ static __forceinline__ void term(const SweepParams &P, const WS &ws, const T *ring, int smod, int cslot,
                                              int row0, int lane, const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                              typename Arith<T>::A (&v)[VX],
                                              typename Arith<T>::A (&o)[kMaxOut][VX],
                                              typename Arith<T>::A (&g)[VX]) {
    using A = typename Arith<T>::A;
    constexpr int cg = EQ ? coef_group_start<Def>(I) : -1;
    if constexpr (cg >= 0) {
      // a coefficient group: one weighted sum (or difference) at its first
      // term; a batch instance whose weights do not allow it takes the terms
      // one by one, as its single-grid call does
      if (!ws.eq()) {
        term_body<T, VX, VY, r, I>(P, ws, ring, smod, cslot, row0, lane, zq, v, o, g);
      } else if constexpr (I == cg) {
        constexpr int n = coef_group_len<Def>(cg);
        A x[VX];
        coef_group_sum<T, VX, VY, r, cg, n>(P, ring, smod, cslot, row0, lane, zq, v, x);
        accumulate<T, VX, r, cg, cg + n - 1>(P, ring, smod, cslot, row0, lane, ws(P, cg), x, v, o, g);
      }
    } else if constexpr (kAxial >= 0 && I >= kAxial && I < kAxial + 6) {
      // the axial group: its six terms are one weighted sum at kAxialAt; a
      // batch instance with unequal weights takes them in table order, as
      // its single-grid call does
      if (!ws.eq()) term_body<T, VX, VY, r, I>(P, ws, ring, smod, cslot, row0, lane, zq, v, o, g);
    } else {
      term_body<T, VX, VY, r, I>(P, ws, ring, smod, cslot, row0, lane, zq, v, o, g);
    }
    if constexpr (kAxialAt >= 0 && I == kAxialAt) {
      if (!ws.eq()) return;
      constexpr int out = Def::table.t[kAxial].out;
      const A w = ws(P, kAxial);
      A x[VX];
      axial_sum<T, VX, VY, r>(P, ring, smod, cslot, row0, lane, zq, v, x);
#pragma unroll
      for (int e = 0; e < VX; ++e) {
        if constexpr (out < 0) v[e] = fma(w, x[e], v[e]);
        else o[out][e] = fma(w, x[e], o[out][e]);
      }
    }
  }

  // One term's contribution (a term outside the axial group).
  template <typename T, int VX, int VY, int r, int I, class WS>
  __device__ static __forceinline__ void term_body(const SweepParams &P, const WS &ws, const T *ring, int smod,
                                                   int cslot, int row0, int lane,
                                                   const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                                   typename Arith<T>::A (&v)[VX],
                                                   typename Arith<T>::A (&o)[kMaxOut][VX],
                                                   typename Arith<T>::A (&g)[VX]) {
    using A = typename Arith<T>::A;
    const A w = ws(P, I);
    A x[VX];
    load_x<T, VX, VY, r, I>(P, ring, smod, cslot, row0, lane, zq, v, x);
    accumulate<T, VX, r, I, I>(P, ring, smod, cslot, row0, lane, w, x, v, o, g);
  }

  // w x added for table terms IF .. IL (one term, or a group summed into x):
  // into the run's sum g (then times the coefficient at the run's last
  // term), or into the destination.
  template <typename T, int VX, int r, int IF, int IL>
  __device__ static __forceinline__ void accumulate(const SweepParams &P, const T *ring, int smod, int cslot,
                                                    int row0, int lane, typename Arith<T>::A w,
                                                    const typename Arith<T>::A (&x)[VX],
                                                    typename Arith<T>::A (&v)[VX],
                                                    typename Arith<T>::A (&o)[kMaxOut][VX],
                                                    typename Arith<T>::A (&g)[VX]) {
    const int row = row0 + r;
    const int col = column(lane, r);
    constexpr int ES = 32 * XS;  // element stride of a thread's columns
    constexpr OpTerm t = Def::table.t[IL];
    constexpr int vec = 16 / (int)sizeof(T);
    if constexpr (t.coef >= 0) {
#pragma unroll
      for (int e = 0; e < VX; ++e) g[e] = run_first(IF) ? w * x[e] : fma(w, x[e], g[e]);
      if constexpr (run_last(IL)) {
        constexpr int RXc = radius(0, t.coef), RYc = radius(1, t.coef);
        constexpr int AXc = (RXc + vec - 1) / vec * vec;
        constexpr int BWc = ES * VX + 2 * AXc;
        const T *cp = in_centre_ring<T>(t.coef)
                          ? centre_ptr<T, VX>(P, ring, t.coef, cslot, row, lane)
                          : ring + P.in_base[t.coef] + smod * P.in_se[t.coef] + row * BWc + col + (RYc * BWc + AXc);
#pragma unroll
        for (int e = 0; e < VX; ++e) {
          if constexpr (t.out < 0) v[e] = fma(to_arith(cp[ES * e]), g[e], v[e]);
          else o[t.out][e] = fma(to_arith(cp[ES * e]), g[e], o[t.out][e]);
        }
      }
    } else if constexpr (t.out < 0) {
#pragma unroll
      for (int e = 0; e < VX; ++e) v[e] = fma(w, x[e], v[e]);
    } else {
#pragma unroll
      for (int e = 0; e < VX; ++e) o[t.out][e] = fma(w, x[e], o[t.out][e]);
    }
  }

  template <typename T, int VX, int VY, int r, class WS, int... I>
  __device__ static __forceinline__ void eval_seq(const SweepParams &P, const WS &ws, const T *ring, int smod,
                                                  int cslot, int row0, int lane,
                                                  const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                                  typename Arith<T>::A (&v)[VX],
                                                  typename Arith<T>::A (&o)[kMaxOut][VX],
                                                  std::integer_sequence<int, I...>) {
    typename Arith<T>::A g[VX];
    (term<T, VX, VY, r, I>(P, ws, ring, smod, cslot, row0, lane, zq, v, o, g), ...);
  }

  template <typename T, int VX, int VY, int r, class WS>
  __device__ static __forceinline__ void eval_row(const SweepParams &P, const WS &ws, const T *ring, int smod,
                                                  int cslot, int row0, int lane,
                                                  const typename Arith<T>::A (&zq)[kQueue][VY][VX],
                                                  typename Arith<T>::A (&v)[VX],
                                                  typename Arith<T>::A (&o)[kMaxOut][VX]) {
    eval_seq<T, VX, VY, r>(P, ws, ring, smod, cslot, row0, lane, zq, v, o,
                           std::make_integer_sequence<int, Def::NT>{});
  }
};

// ---------------------------------------------------------------- vector lanes
// Loads G contiguous elements (16 bytes) from shared memory as arithmetic
// values; p is 16-byte aligned.  BF16 widens to FP32 by placing its bits in
// the upper half of the word (exact).
template <int G>
__device__ __forceinline__ void load_group(const float *p, float (&x)[G]) {
  static_assert(G % 4 == 0, "FP32 groups are whole float4s");
#pragma unroll
  for (int q = 0; q < G / 4; ++q) {
    const float4 v = reinterpret_cast<const float4 *>(p)[q];
    x[4 * q] = v.x;
    x[4 * q + 1] = v.y;
    x[4 * q + 2] = v.z;
    x[4 * q + 3] = v.w;
  }
}
template <int G>
__device__ __forceinline__ void load_group(const __nv_bfloat16 *p, float (&x)[G]) {
  static_assert(G % 8 == 0, "BF16 groups are whole 16-byte words");
#pragma unroll
  for (int q = 0; q < G / 8; ++q) {
    const uint4 v = reinterpret_cast<const uint4 *>(p)[q];
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      x[8 * q + 2 * k] = __uint_as_float(w[k] << 16);
      x[8 * q + 2 * k + 1] = __uint_as_float(w[k] & 0xffff0000u);
    }
  }
}

// Stores G contiguous results (16 bytes per float4 / 8 BF16) to global
// memory; p is 16-byte aligned.  BF16 rounds each pair with one conversion.
template <int G>
__device__ __forceinline__ void store_group(float *p, const float (&x)[G]) {
#pragma unroll
  for (int q = 0; q < G / 4; ++q)
    reinterpret_cast<float4 *>(p)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
}
template <int G>
__device__ __forceinline__ void store_group(__nv_bfloat16 *p, const float (&x)[G]) {
#pragma unroll
  for (int q = 0; q < G / 8; ++q) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(x[8 * q + 2 * k], x[8 * q + 2 * k + 1]);
      w[k] = *reinterpret_cast<const uint32_t *>(&h);
    }
    reinterpret_cast<uint4 *>(p)[q] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// acc[e] = fma(w, x[e], acc[e]) for every element of a group; FP32 pairs go
// through the packed two-lane FMA (each lane one fma.rn, so the bits are
// those of the scalar FMAs).
template <int G>
__device__ __forceinline__ void fma_group(float w, const float (&x)[G], float (&acc)[G]) {
#pragma unroll
  for (int e = 0; e + 1 < G; e += 2) {
    const float2 r = __ffma2_rn(make_float2(w, w), make_float2(x[e], x[e + 1]), make_float2(acc[e], acc[e + 1]));
    acc[e] = r.x;
    acc[e + 1] = r.y;
  }
  if constexpr (G % 2) acc[G - 1] = fmaf(w, x[G - 1], acc[G - 1]);
}
// acc[e] = fma(c[e], g[e], acc[e]): a coefficient run's product per element
template <int G>
__device__ __forceinline__ void fma_group(const float (&c)[G], const float (&g)[G], float (&acc)[G]) {
#pragma unroll
  for (int e = 0; e + 1 < G; e += 2) {
    const float2 r =
        __ffma2_rn(make_float2(c[e], c[e + 1]), make_float2(g[e], g[e + 1]), make_float2(acc[e], acc[e + 1]));
    acc[e] = r.x;
    acc[e + 1] = r.y;
  }
  if constexpr (G % 2) acc[G - 1] = fmaf(c[G - 1], g[G - 1], acc[G - 1]);
}

// Compile-time term table with vector lanes (FP32 / BF16 storage): a lane
// owns G = 16 / sizeof(T) contiguous columns of a tile row, so every read of
// a term's row is one 16-byte shared-memory load, the x neighbours come from
// the same registers (plus one scalar load at the group's edge), the FMAs
// run in FP32 pairs and the results leave as 16-byte stores.  A tile row of
// 128 columns takes 128 / G lanes: 32 for FP32, a half-warp for BF16 (the
// warp's two halves own the two halves of its rows, RPS = 2 row blocks per
// warp).  Each element is evaluated with the same operations in the same
// order as StaticOp<Def, 1>, so the two policies give bit-identical results.
template <class Def, int G>
struct StaticOpV {
  using Base = StaticOp<Def, 1>;
  static constexpr int kXStep = 1;
  static constexpr int kGroup = G;
  static constexpr int kLanesPerRow = 128 / G;
  static constexpr int kRowsPerSlot = 32 / kLanesPerRow;
  static constexpr int kTerms = Def::NT;
  static constexpr int kMaxOut = Base::kMaxOut;
  template <typename A, bool BATCH>
  using Weights = typename Base::template Weights<A, BATCH>;
  __device__ static constexpr int n_out(const SweepParams &P) { return Def::NOUT; }
  static constexpr int RZ = Base::RZ;
  static constexpr int ZQ = Base::ZQ;
  static constexpr int kQueue = Base::kQueue;

  __host__ __device__ static constexpr bool fits() {
    for (int i = 0; i < Def::NT; ++i) {
      const int dx = Def::table.t[i].dx;
      if (dx > G || -dx > G) return false;
    }
    return true;
  }

  // element (row, 0) of ring input IN's box in `slot` (its tile row `row`, first core column)
  template <int IN, typename T>
  __device__ static __forceinline__ const T *row_ptr(const SweepParams &P, const T *ring, int slot, int row) {
    constexpr int vec = 16 / (int)sizeof(T);
    constexpr int AX = (Base::radius(0, IN) + vec - 1) / vec * vec;
    constexpr int RY = Base::radius(1, IN);
    constexpr int BW = 128 + 2 * AX;
    return ring + P.in_base[IN] + slot * P.in_se[IN] + (row + RY) * BW + AX;
  }

  // BF16 storage keeps the queue's rows as the packed pairs they were loaded
  // as (G / 2 words in the first entries of each row, the rest unused) and
  // widens an element where a term reads it, exactly as load_group does:
  // half the queue's registers, the same values.
  template <typename T>
  __host__ __device__ static constexpr bool packed_queue() { return std::is_same<T, __nv_bfloat16>::value; }
  template <typename T, int VX>
  __device__ static __forceinline__ void queue_row(const T *p, float (&q)[VX]) {
    if constexpr (packed_queue<T>()) {
      static_assert(VX == 8, "BF16 vector lanes hold 8 columns (one 16-byte word)");
      const uint4 v = *reinterpret_cast<const uint4 *>(p);
      q[0] = __uint_as_float(v.x);
      q[1] = __uint_as_float(v.y);
      q[2] = __uint_as_float(v.z);
      q[3] = __uint_as_float(v.w);
    } else {
      load_group<G>(p, q);
    }
  }
  template <typename T, int VX>
  __device__ static __forceinline__ float queue_elem(const float (&q)[VX], int e) {
    if constexpr (packed_queue<T>()) {
      const uint32_t w = __float_as_uint(q[e >> 1]);
      return __uint_as_float((e & 1) ? (w & 0xffff0000u) : (w << 16));
    } else {
      return q[e];
    }
  }

  // Step start: queue rows of planes z - RZ .. z + RZ (col: this lane's first column).
  template <typename T, int VX, int VY>
  __device__ static __forceinline__ void advance_queue(const SweepParams &P, const T *ring, int smod, int row0,
                                                       int col, bool first, float (&zq)[kQueue][VY][VX]) {
    if constexpr (ZQ >= 0) {
      constexpr int used = packed_queue<T>() ? VX / 2 : VX;
      const int R = P.R;
      if (first) {
#pragma unroll
        for (int k = 0; k <= 2 * RZ; ++k) {
          int sl = smod + k - RZ;
          sl = sl >= R ? sl - R : (sl < 0 ? sl + R : sl);
#pragma unroll
          for (int r = 0; r < VY; ++r) queue_row<T, VX>(row_ptr<ZQ>(P, ring, sl, row0 + r) + col, zq[k][r]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 2 * RZ; ++k)
#pragma unroll
          for (int r = 0; r < VY; ++r)
#pragma unroll
            for (int e = 0; e < used; ++e) zq[k][r][e] = zq[k + 1][r][e];
        int sl = smod + RZ;
        sl = sl >= R ? sl - R : sl;
#pragma unroll
        for (int r = 0; r < VY; ++r) queue_row<T, VX>(row_ptr<ZQ>(P, ring, sl, row0 + r) + col, zq[2 * RZ][r]);
      }
    }
  }

  // Term I at tile row row0 + r; col = this lane's first column in the tile.
  template <typename T, int VX, int VY, int r, int I, class WS>
  __device__ static __forceinline__ void term(const SweepParams &P, const WS &ws, const T *ring, int smod, int cslot,
                                              int row0, int col, const float (&zq)[kQueue][VY][VX], float (&v)[VX],
                                              float (&o)[kMaxOut][VX], float (&g)[VX]) {
    static_assert(VX == G, "one group per lane and row");
    const int row = row0 + r;
    constexpr OpTerm t = Def::table.t[I];
    const int R = P.R;
    const float w = ws(P, I);
    float x[G];
    if constexpr (t.in < 0) {
#pragma unroll
      for (int e = 0; e < G; ++e) x[e] = v[e];
    } else if constexpr (Base::template in_centre_ring<T>(t.in)) {
      load_group<G>(ring + P.in_base[t.in] + cslot * P.in_se[t.in] + row * 128 + col, x);
    } else {
      int slot = smod + t.dz;
      if constexpr (t.dz > 0) slot = slot >= R ? slot - R : slot;
      if constexpr (t.dz < 0) slot = slot < 0 ? slot + R : slot;
      const T *rp = row_ptr<t.in>(P, ring, slot, row + t.dy) + col;
      float c[G];
      if constexpr (t.in == ZQ && r + t.dy >= 0 && r + t.dy < VY && t.dz >= -RZ && t.dz <= RZ) {
#pragma unroll
        for (int e = 0; e < G; ++e) c[e] = queue_elem<T, VX>(zq[t.dz + RZ][r + t.dy], e);
      } else {
        load_group<G>(rp, c);
      }
#pragma unroll
      for (int e = 0; e < G; ++e) {
        const int k = e + t.dx;  // compile-time after unrolling
        x[e] = (k >= 0 && k < G) ? c[k < 0 ? 0 : (k >= G ? G - 1 : k)] : to_arith(rp[k]);
      }
    }
    if constexpr (t.coef >= 0) {
      if constexpr (Base::run_first(I)) {
#pragma unroll
        for (int e = 0; e < G; ++e) g[e] = w * x[e];
      } else {
        fma_group<G>(w, x, g);
      }
      if constexpr (Base::run_last(I)) {
        float cf[G];
        if constexpr (Base::template in_centre_ring<T>(t.coef)) {
          load_group<G>(ring + P.in_base[t.coef] + cslot * P.in_se[t.coef] + row * 128 + col, cf);
        } else {
          load_group<G>(row_ptr<t.coef>(P, ring, smod, row) + col, cf);
        }
        if constexpr (t.out < 0) fma_group<G>(cf, g, v);
        else fma_group<G>(cf, g, o[t.out]);
      }
    } else if constexpr (t.out < 0) {
      fma_group<G>(w, x, v);
    } else {
      fma_group<G>(w, x, o[t.out]);
    }
  }

  template <typename T, int VX, int VY, int r, class WS, int... I>
  __device__ static __forceinline__ void eval_seq(const SweepParams &P, const WS &ws, const T *ring, int smod,
                                                  int cslot, int row0, int col, const float (&zq)[kQueue][VY][VX],
                                                  float (&v)[VX], float (&o)[kMaxOut][VX],
                                                  std::integer_sequence<int, I...>) {
    float g[VX];
    (term<T, VX, VY, r, I>(P, ws, ring, smod, cslot, row0, col, zq, v, o, g), ...);
  }

  template <typename T, int VX, int VY, int r, class WS>
  __device__ static __forceinline__ void eval_row(const SweepParams &P, const WS &ws, const T *ring, int smod,
                                                  int cslot, int row0, int col, const float (&zq)[kQueue][VY][VX],
                                                  float (&v)[VX], float (&o)[kMaxOut][VX]) {
    eval_seq<T, VX, VY, r>(P, ws, ring, smod, cslot, row0, col, zq, v, o, std::make_integer_sequence<int, Def::NT>{});
  }
};

// ---------------------------------------------------------------- reduction keys
// Exact FP32 -> FP64 widening from the IEEE 754 binary32 / binary64 layouts:
// for a normal float the sign and fraction bits carry over and the exponent
// bias changes from 127 to 1023 (+896), all on the integer pipe.  A group
// containing a zero, subnormal, infinity or NaN takes the hardware conversion.
template <int N>
__device__ __forceinline__ void widen_group(const float (&x)[N], double (&d)[N]) {
  bool normal = true;
#pragma unroll
  for (int i = 0; i < N; ++i) normal &= ((__float_as_uint(x[i]) >> 23) & 0xffu) - 1u < 254u;
  if (__all_sync(0xffffffffu, normal)) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const unsigned b = __float_as_uint(x[i]);
      const unsigned long long bits = ((unsigned long long)(b & 0x80000000u) << 32) |
                                      ((unsigned long long)(((b >> 23) & 0xffu) + 896u) << 52) |
                                      ((unsigned long long)(b & 0x7fffffu) << 29);
      d[i] = __longlong_as_double((long long)bits);
    }
  } else {
#pragma unroll
    for (int i = 0; i < N; ++i) d[i] = (double)x[i];
  }
}
template <int N>
__device__ __forceinline__ void widen_group(const double (&x)[N], double (&d)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) d[i] = x[i];
}
template <int N>
__device__ __forceinline__ void widen_group(const Df64 (&x)[N], double (&d)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) d[i] = combine_f64(x[i]);
}

// max |v| is tracked on the bits of |v| in the value's own format (for
// non-negative IEEE numbers the unsigned order of the bits is the numeric
// order, and NaN sorts above infinity), converted to double once at the end.
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}
__device__ __forceinline__ unsigned long long abs_key(float v) {
  return (unsigned long long)(__float_as_uint(v) & 0x7fffffffu);
}
__device__ __forceinline__ unsigned long long abs_key(Df64 v) { return abs_key(combine_f64(v)); }
__device__ __forceinline__ double key_value(unsigned long long k, double) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ double key_value(unsigned long long k, Df64) { return __longlong_as_double((long long)k); }
__device__ __forceinline__ double key_value(unsigned long long k, float) { return (double)__uint_as_float((unsigned)k); }

// ---------------------------------------------------------------- kernel
// Folds the CTA's per-thread (s, c) pairs (or max keys) in a fixed order;
// the result is valid in thread 0.  Uses s_red[2 * warps].
template <int RED>
__device__ __forceinline__ void block_fold(double &s, double &c, double *s_red, int NW) {
  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  for (int off = 16; off > 0; off >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, s, off);
    const double c2 = __shfl_down_sync(0xffffffffu, c, off);
    if (RED == RED_MAXABS) s = max_abs_bits(s, s2);
    else combine_pair(s, c, s2, c2);
  }
  __syncthreads();  // s_red may still be read from a previous fold
  if (lane == 0) {
    s_red[2 * wy] = s;
    s_red[2 * wy + 1] = c;
  }
  __syncthreads();
  if (tid == 0) {
    s = s_red[0];
    c = s_red[1];
    for (int w = 1; w < NW; ++w) {
      if (RED == RED_MAXABS) s = max_abs_bits(s, s_red[2 * w]);
      else combine_pair(s, c, s_red[2 * w], s_red[2 * w + 1]);
    }
  }
}

// The CTA's L2 partial for FP32 arithmetic, valid in thread 0 as (s, c) with
// value s - c: each warp folds its threads' square sums as FP32 pairs in a
// fixed shuffle tree, then thread 0 widens the warps' pairs to FP64 and
// combines them, in order, with the FP64 squares some threads took for
// out-of-range values (folded by block_fold only when there are any).
// (s, c) enter as the thread's FP64 part.
__device__ __forceinline__ void cta_fold_sq32(SquareSum32 q, double &s, double &c, double *s_red, int NW) {
  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  const bool any64 = __syncthreads_or(s != 0.0 || c != 0.0) != 0;
  q.fold_lanes();
  for (int off = 16; off > 0; off >>= 1) {
    const float h = __shfl_down_sync(0xffffffffu, q.hi.x, off);
    const float l = __shfl_down_sync(0xffffffffu, q.lo.x, off);
    q.add_sum(h, l);
  }
  if (any64) block_fold<RED_L2>(s, c, s_red, NW);
  __syncthreads();  // s_red may still be read by block_fold
  if (lane == 0) {
    s_red[2 * wy] = (double)q.hi.x;   // the warp's hi + lo as s - c
    s_red[2 * wy + 1] = -(double)q.lo.x;
  }
  __syncthreads();
  if (tid == 0) {
    double fs = any64 ? s : 0.0, fc = any64 ? c : 0.0;
    for (int w = 0; w < NW; ++w) combine_pair(fs, fc, s_red[2 * w], s_red[2 * w + 1]);
    s = fs;
    c = fc;
  }
}

// Warp wy owns the VY adjacent tile rows wy VY .. wy VY + VY - 1, so the
// y neighbour of one of its rows is the centre of the next (one shared-memory
// load serves both).
// BATCH: segments come from the device work-list and each segment's
// reduction goes to its own partial (per-instance results are folded by
// batch_finalize_kernel); otherwise the CTA derives its run of (tile, plane)
// pairs of the single grid and the last CTA folds all partials.
// Single-grid sweeps of small operators (up to 10 terms: the star / heat
// family) on FP32 grids are bound by memory and latency: they keep four
// 8-warp CTAs per SM (at most 64 registers per thread).  Reducing sweeps
// carry the square-sum pairs and spill under that bound, larger operators
// (the climate operator) are held to fewer CTAs by their shared memory, and
// BF16 vector lanes (two rows of 8 columns per thread; the z queue packed)
// fit three CTAs per SM at the compiler's own register target: those keep it.
template <typename T, bool BATCH, int RED, class Op>
constexpr int min_ctas_per_sm() {
  return (!BATCH && RED == RED_NONE && std::is_same<T, float>::value && Op::kTerms <= 10) ? 4 : 0;
}

template <typename T, int VX, int VY, int RED, class Op, bool BATCH>
__global__ void __launch_bounds__(256, min_ctas_per_sm<T, BATCH, RED, Op>())
    sweep_kernel(const __grid_constant__ SweepParams P) {
  using A = typename Arith<T>::A;
  constexpr int XS = Op::kXStep;
  constexpr int G = Op::kGroup;           // > 1: vector lanes (StaticOpV), G contiguous columns each
  constexpr int RPS = Op::kRowsPerSlot;   // row blocks per warp (2 when a tile row takes a half-warp)
  constexpr int TX = G > 1 ? 128 : 32 * XS * VX;
  constexpr int NO = Op::kMaxOut;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem);
  T *ring = reinterpret_cast<T *>(smem + kBarBytes);
  __shared__ int s_abort;
  __shared__ bool s_last;
  __shared__ double s_red[2 * 16];

  const int tid = threadIdx.x, lane = tid & 31, wy = tid >> 5;
  const int NW = blockDim.x >> 5;
  const int TY = NW * VY * RPS;
  const int R = P.R, rz = P.rz;
  // vector lanes: lane = rb * (128 / G) + cg owns columns G cg .. G cg + G - 1
  // of the rows of row block rb; the thread's first tile row
  const int cg = G > 1 ? lane % (128 / (G > 1 ? G : 1)) : 0;
  const int rb = G > 1 ? lane / (128 / (G > 1 ? G : 1)) : 0;
  const int wrow0 = (wy * RPS + rb) * VY;

  uint64_t *cbars = bars + kMaxRing;  // the centre ring's two slots
  const bool has_c = P.cmask != 0;
  if (tid == 0) {
    for (int r = 0; r < R; ++r) mbar_init(&bars[r], 1);
    if (has_c) {
      mbar_init(&cbars[0], 1);
      mbar_init(&cbars[1], 1);
    }
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  // Nothing above touches global memory: wait here for the previous sweep
  // (its outputs are this sweep's inputs).
  pdl_wait();

  typename Op::template Weights<A, BATCH> ws;  // the operator's weights (per instance in batches)
  Compensated acc;
  double sq = 0.0;          // L2: plain FP64 chain of squares within one segment
  // L2 of FP32 arithmetic (FP32 / BF16 storage): squares summed on the FP32 pipe
  constexpr bool kSq32 = RED == RED_L2 && std::is_same<A, float>::value;
  constexpr bool kSq64 = RED == RED_L2 && std::is_same<A, double>::value;  // IEEE FP64 (not pairs)
  SquareSum32 sq32;
  unsigned long long maxkey = 0;
  uint32_t seq = 0;         // planes issued by this CTA (identical in every thread)
  uint32_t issued_end = 0;  // thread 0: planes actually issued
  uint32_t waited_end = 0;  // planes this thread has waited for
  int wslot = 0;            // ring slot and phase parity of the next plane to wait for
  uint32_t wpar = 0;
  int islot = 0;            // thread 0: ring slot of the next plane to issue
  // centre ring: its planes are numbered over the CTA's whole run; plane g
  // uses slot g & 1 with phase parity (g >> 1) & 1
  uint32_t c_issued = 0;    // thread 0: centre planes issued
  uint32_t c_waited = 0;    // centre planes waited for (identical in every thread)
  bool ok = true;

  // Single grid: the (xy tile, z plane) pairs of the range, z fastest, split
  // into gridDim.x equal contiguous runs (one wave of CTAs); CTA b streams
  // through [W b / G, W (b+1) / G), one tile-column segment at a time.
  long long pos = 0, run_end = 0;
  int kseg = 0, kend = 0;
  if constexpr (BATCH) {
    kseg = P.cta_seg[blockIdx.x];
    kend = P.cta_seg[blockIdx.x + 1];
  } else {
    const long long nzr = P.inst.hi[2] - P.inst.lo[2];
    const long long W = (long long)P.inst.tiles_x * P.inst.tiles_y * nzr;
    pos = W * blockIdx.x / gridDim.x;
    run_end = W * (blockIdx.x + 1) / gridDim.x;
  }
  // With a grid that is a whole multiple of the tile columns (zalt), the
  // runs above are exactly k z ranges of each column (CTA c k + j: range j of
  // column c), so the CTAs j of all columns cover the same planes at the same
  // time and neighbouring tiles read their shared halo rows close together
  // (the second read is served by L2).
  auto adv = [&](int sl) { return sl + 1 == R ? 0 : sl + 1; };
  for (;;) {
    const InstDesc *I;
    long long col, zoff;
    int zlen;
    if constexpr (BATCH) {
      if (kseg >= kend) break;
      const Segment sg = P.segs[kseg];
      I = &P.insts[sg.inst];
      ws.load(P.inst_w + sg.inst);
      col = sg.col;
      zoff = sg.zoff;
      zlen = sg.zlen;
    } else {
      if (pos >= run_end) break;
      I = &P.inst;
      const long long nzr = I->hi[2] - I->lo[2];
      col = pos / nzr;
      zoff = pos - col * nzr;
      zlen = (int)min(nzr - zoff, run_end - pos);
      pos += zlen;
    }
    const int txi = (int)(col % I->tiles_x);
    const int tyi = (int)(col / I->tiles_x);
    const int64_t x0 = I->x_base + (int64_t)txi * TX;
    const int64_t y0 = I->y_base + (int64_t)tyi * TY;
    const int64_t zb = I->lo[2] + zoff;
    const int total = zlen + 2 * rz;
    const uint32_t g0 = seq;
    seq += total;

    // planes are issued and consumed in order, so slots and phases advance
    // by one per plane: plane q of this segment is z = zb - rz + q
    auto issue = [&](int q) {
      const int slot = islot;
      islot = adv(islot);
      uint64_t *bar = &bars[slot];
      mbar_arrive_expect_tx(bar, P.tx_bytes);
      const int zp = (int)(zb - rz + q);
      for (int a = 0; a < P.n_in; ++a)
        if (!((P.cmask >> a) & 1u))
          tma_load_3d(ring + P.in_base[a] + slot * P.in_se[a], &I->tmap[a], bar,
                      (int)(x0 - P.in_ax[a]) + I->cx_add[a], (int)(y0 - P.in_ry[a]) + I->cy_add[a],
                      zp + I->cz_add[a]);
      issued_end = g0 + q + 1;
    };
    auto wait_next = [&]() {
      if (!mbar_wait_bounded(&bars[wslot], wpar)) return false;
      ++waited_end;
      wslot = adv(wslot);
      if (wslot == 0) wpar ^= 1u;
      return true;
    };

    const uint32_t c0 = c_waited;  // centre plane of this segment's step 0
    // centre-ring inputs of step s (plane z of that step) into slot (c0 + s) & 1
    auto issue_c = [&](int st) {
      const uint32_t g = c0 + (uint32_t)st;
      uint64_t *bar = &cbars[g & 1u];
      mbar_arrive_expect_tx(bar, P.ctx_bytes);
      const int zp = (int)(zb + st);
      for (int a = 0; a < P.n_in; ++a)
        if ((P.cmask >> a) & 1u)
          tma_load_3d(ring + P.in_base[a] + (int)(g & 1u) * P.in_se[a], &I->tmap[a], bar,
                      (int)x0 + I->cx_add[a], (int)y0 + I->cy_add[a], zp + I->cz_add[a]);
      c_issued = g + 1;
    };

    if (tid == 0) {
      const int np = min(R, total);
      for (int q = 0; q < np; ++q) issue(q);
      if (has_c) {
        issue_c(0);
        if (zlen > 1) issue_c(1);
      }
    }

    int64_t y[VY];
    bool yok[VY];
#pragma unroll
    for (int r = 0; r < VY; ++r) {
      y[r] = y0 + wrow0 + r;
      yok[r] = (y[r] >= I->lo[1]) && (y[r] < I->hi[1]);
    }
    bool xok[VX];
#pragma unroll
    for (int e = 0; e < VX; ++e) {
      const int64_t x = G > 1 ? x0 + G * cg + e : x0 + lane + 32 * e;
      xok[e] = (x >= I->lo[0]) && (x < I->hi[0]);
    }
    int smod = wslot;  // slot of the centre plane of step 0
    for (int i = 0; i < rz; ++i) smod = adv(smod);
    A zq[Op::kQueue][VY][VX];  // z register queue (compile-time operators of the star family)

    for (int s = 0; s < zlen; ++s) {
      const int cslot = (int)((c0 + (uint32_t)s) & 1u);
      if (ok) {
        if (s == 0) {
          for (int d = 0; d <= 2 * rz && ok; ++d) ok = wait_next();
        } else {
          ok = wait_next();
        }
        if (ok && has_c) {
          ok = mbar_wait_bounded(&cbars[cslot], ((c0 + (uint32_t)s) >> 1) & 1u);
          if (ok) ++c_waited;
        }
        if (!ok) {
          s_abort = 1;
          atomicOr(P.err, 1);
        }
      }
      if (ok) {
        const int64_t z = zb + s;
        // colour-compacted sweeps: the warp's first row starts at column
        // 2 lane + p, p making (x + y + z) even for colour 0 (x0 and the
        // warp's first row y0 + wy VY differ from y0 by even amounts)
        const int carg = G > 1 ? G * cg : (XS == 1 ? lane : 2 * lane + (int)((P.color + y0 + z) & 1));
        Op::template advance_queue<T, VX, VY>(P, ring, smod, wrow0, carg, s == 0, zq);
        static_for<VY>([&](auto rc) {
          constexpr int r = decltype(rc)::value;
          A v[VX];
          A o[NO][VX];
#pragma unroll
          for (int e = 0; e < VX; ++e) {
            v[e] = A(0);
#pragma unroll
            for (int m = 0; m < NO; ++m) o[m][e] = A(0);
          }
          Op::template eval_row<T, VX, VY, r>(P, ws, ring, smod, cslot, wrow0, carg, zq, v, o);
          if constexpr (G > 1) {
            // vector lanes: one 16-byte store per output when the group is
            // whole and uncoloured; element by element at ragged edges and
            // in red-black sweeps (the group's columns alternate colours)
            if (yok[r]) {
#pragma unroll
              for (int m = 0; m < NO; ++m) {
                if (m < Op::n_out(P)) {
                  T *dst = reinterpret_cast<T *>(I->out[m].base) + z * I->out[m].plane + y[r] * I->out[m].pitch +
                           x0 + G * cg;
                  if (P.color < 0 && xok[0] && xok[G - 1]) {
                    store_group<G>(dst, o[m]);
                  } else {
#pragma unroll
                    for (int e = 0; e < VX; ++e)
                      if (xok[e] && (P.color < 0 || (int)((x0 + G * cg + e + y[r] + z) & 1) == P.color))
                        dst[e] = from_arith<T>(o[m][e]);
                  }
                }
              }
            }
          } else if constexpr (XS == 1) {
            // red-black colouring: a thread's columns x0 + lane + 32 e share one parity
            if (yok[r] && (P.color < 0 || (int)((x0 + lane + y[r] + z) & 1) == P.color)) {
#pragma unroll
              for (int m = 0; m < NO; ++m) {
                if (m < Op::n_out(P)) {
                  T *dst = reinterpret_cast<T *>(I->out[m].base) + z * I->out[m].plane + y[r] * I->out[m].pitch +
                           x0 + lane;
#pragma unroll
                  for (int e = 0; e < VX; ++e)
                    if (xok[e]) dst[32 * e] = from_arith<T>(o[m][e]);
                }
              }
            }
          } else if (yok[r]) {
            // colour-compacted: every element this thread computed is of the colour
            const int col = carg ^ (r & 1);
#pragma unroll
            for (int m = 0; m < NO; ++m) {
              if (m < Op::n_out(P)) {
                T *dst = reinterpret_cast<T *>(I->out[m].base) + z * I->out[m].plane + y[r] * I->out[m].pitch +
                         x0 + col;
#pragma unroll
                for (int e = 0; e < VX; ++e) {
                  const int64_t x = x0 + col + 64 * e;
                  if (x >= I->lo[0] && x < I->hi[0]) dst[64 * e] = from_arith<T>(o[m][e]);
                }
              }
            }
          }
          if constexpr (RED == RED_MAXABS) {
#pragma unroll
            for (int e = 0; e < VX; ++e)
              if (yok[r] && xok[e]) maxkey = max(maxkey, abs_key(v[e]));
          } else if constexpr (kSq32) {
            // the row's largest |v| in [2^-50, 2^50] (or every value 0): the
            // squares are exact in FP32 pairs; otherwise (an infinity, a
            // value out of that range) this row's squares go to the FP64
            // chain.  fmaxf passes over NaN, which then propagates through
            // the pair sums.  A whole group in range takes one max and one
            // test per row, without per-element masks.
            if (yok[r] && xok[0] && xok[VX - 1]) {
              float m = 0.0f;
#pragma unroll
              for (int e = 0; e < VX; ++e) m = fmaxf(m, fabsf(v[e]));
              if (m <= 0x1p50f && (m >= 0x1p-50f || m == 0.0f)) {
#pragma unroll
                for (int e = 0; e + 1 < VX; e += 2) sq32.add_squares(v[e], v[e + 1]);
              } else {
#pragma unroll
                for (int e = 0; e < VX; ++e) sq = fma((double)v[e], (double)v[e], sq);
              }
            } else if (yok[r]) {
              float w[VX];
              float m = 0.0f;
#pragma unroll
              for (int e = 0; e < VX; ++e) {
                w[e] = xok[e] ? v[e] : 0.0f;
                m = fmaxf(m, fabsf(w[e]));
              }
              if (m <= 0x1p50f && (m >= 0x1p-50f || m == 0.0f)) {
#pragma unroll
                for (int e = 0; e + 1 < VX; e += 2) sq32.add_squares(w[e], w[e + 1]);
              } else {
#pragma unroll
                for (int e = 0; e < VX; ++e) sq = fma((double)w[e], (double)w[e], sq);
              }
            }
          } else if constexpr (kSq64) {
            // squares on the FP32 pipe (split_double, add_split_squares) for
            // rows whose values are all in range; otherwise the FP64 chain
            bool in_range = true;
            double w[VX];
#pragma unroll
            for (int e = 0; e < VX; ++e) {
              w[e] = (yok[r] && xok[e]) ? v[e] : 0.0;
              in_range &= split_in_range(w[e]);
            }
            if (in_range) {
#pragma unroll
              for (int e = 0; e + 1 < VX; e += 2) {
                float ha, ea, hb, eb;
                split_double(w[e], ha, ea);
                split_double(w[e + 1], hb, eb);
                sq32.add_split_squares(ha, ea, hb, eb);
              }
            } else {
#pragma unroll
              for (int e = 0; e < VX; ++e) sq = fma(w[e], w[e], sq);
            }
          } else if constexpr (RED != RED_NONE) {
            double d[VX];
            widen_group<VX>(v, d);
            if (RED == RED_L2) {
#pragma unroll
              for (int e = 0; e < VX; ++e)
                if (yok[r] && xok[e]) sq = fma(d[e], d[e], sq);
            } else {
              double gsum = 0.0;
#pragma unroll
              for (int e = 0; e < VX; ++e)
                if (yok[r] && xok[e]) gsum += d[e];
              acc.add(gsum);
            }
          }
        });
        if constexpr (kSq32 || kSq64) sq32.renormalize();
      }
      smod = adv(smod);
      __syncthreads();
      if (s_abort) break;
      if (tid == 0 && s + R < total) issue(s + R);
      if (tid == 0 && has_c && s + 2 < zlen) issue_c(s + 2);
    }
    if (RED == RED_L2) {  // squares are non-negative: the chain's relative error is at most its length x eps
      acc.add(sq);
      sq = 0.0;
    }
    if (s_abort) break;
    if constexpr (BATCH && RED != RED_NONE) {
      // this segment's partial, in a fixed order; then start afresh
      double fs = RED == RED_MAXABS ? key_value(maxkey, A(0)) : acc.s;
      double fc = RED == RED_MAXABS ? 0.0 : acc.c;
      if constexpr (kSq32 || kSq64) cta_fold_sq32(sq32, fs, fc, s_red, NW);
      else block_fold<RED>(fs, fc, s_red, NW);
      if (tid == 0) {
        P.seg_partials[2 * kseg] = fs;
        P.seg_partials[2 * kseg + 1] = fc;
      }
      acc = Compensated();
      maxkey = 0;
      sq32 = SquareSum32();
    }
    if constexpr (BATCH) ++kseg;
  }

  // this CTA's sweep work is done: the next sweep may begin launching (it
  // still waits for this whole grid before reading anything)
  pdl_launch_dependents();

  if (s_abort) {
    // a wait gave up: let every copy this CTA issued land before exiting
    if (tid == 0)
      for (uint32_t g = waited_end; g < issued_end; ++g)
        mbar_wait_bounded(&bars[g % (uint32_t)R], (g / (uint32_t)R) & 1u);
    if (tid == 0)
      for (uint32_t g = c_waited; g < c_issued; ++g) mbar_wait_bounded(&cbars[g & 1u], (g >> 1) & 1u);
    __syncthreads();
    return;
  }

  if constexpr (RED == RED_NONE || BATCH) return;

  // ---- single grid: CTA partial, then the last CTA folds all partials
  double s = RED == RED_MAXABS ? key_value(maxkey, A(0)) : acc.s;  // widened: double bits from here on
  double c = RED == RED_MAXABS ? 0.0 : acc.c;
  if constexpr (kSq32 || kSq64) cta_fold_sq32(sq32, s, c, s_red, NW);
  else block_fold<RED>(s, c, s_red, NW);
  unsigned int *ticket = reinterpret_cast<unsigned int *>(P.workspace);
  double *partials = reinterpret_cast<double *>(P.workspace + 256);
  if (tid == 0) {
    partials[2 * blockIdx.x] = s;
    partials[2 * blockIdx.x + 1] = c;
    __threadfence();
    const unsigned int prev = atomicAdd(ticket, 1u);
    s_last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!s_last || wy != 0) return;
  __threadfence();
  // last CTA, one warp (FP64 work on B300's narrow FP64 pipe stays short):
  // lane i folds a fixed contiguous chunk of partials, then a fixed shuffle
  // tree combines the lanes in order.
  const int nctas = gridDim.x;
  const int chunk = (nctas + 31) / 32;
  s = 0.0;
  c = 0.0;
  for (int b = lane * chunk; b < min(nctas, (lane + 1) * chunk); ++b) {
    const double ps = __ldcg(&partials[2 * b]);
    const double pc = __ldcg(&partials[2 * b + 1]);
    if (RED == RED_MAXABS) s = max_abs_bits(s, ps);
    else combine_pair(s, c, ps, pc);
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, s, off);
    const double c2 = __shfl_down_sync(0xffffffffu, c, off);
    if (RED == RED_MAXABS) s = max_abs_bits(s, s2);
    else combine_pair(s, c, s2, c2);
  }
  if (tid == 0) {
    double r;
    if (RED == RED_MAXABS) r = P.within >= 0.0 ? (s <= P.within ? 1.0 : 0.0) : s;  // NaN fails the test
    else if (RED == RED_L2) r = sqrt(s - c);
    else r = s - c;
    *P.result = r;
    *ticket = 0u;  // ready for the next call
  }
}

// Per-instance results of a batched reduce: instance i's segments are the
// contiguous range [inst_seg[i], inst_seg[i + 1]) of the work-list.  One
// warp per instance: lane l folds the l-th of 32 equal contiguous chunks in
// order, then the lanes combine in a fixed shuffle tree (deterministic for a
// given work-list).  One thread per instance had made the fold a dependent
// chain of FP64 TwoSums as long as the instance's segment count, which on
// the FP64 pipe's latency took as long as the sweep for a large instance.
template <int RED>
__global__ void batch_finalize_kernel(const double *seg_partials, const int32_t *inst_seg, int n_inst,
                                      double *results) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n_inst) return;  // the whole warp
  const int k0 = inst_seg[i], n = inst_seg[i + 1] - k0;
  const int chunk = (n + 31) / 32;
  const int b = min(n, lane * chunk), e = min(n, b + chunk);
  double s = 0.0, c = 0.0;
  for (int k = k0 + b; k < k0 + e; ++k) {
    if (RED == RED_MAXABS) s = max_abs_bits(s, seg_partials[2 * k]);
    else combine_pair(s, c, seg_partials[2 * k], seg_partials[2 * k + 1]);
  }
  for (int off = 16; off > 0; off >>= 1) {
    const double s2 = __shfl_down_sync(0xffffffffu, s, off);
    const double c2 = __shfl_down_sync(0xffffffffu, c, off);
    if (RED == RED_MAXABS) s = max_abs_bits(s, s2);
    else combine_pair(s, c, s2, c2);
  }
  if (lane == 0) results[i] = RED == RED_MAXABS ? s : (RED == RED_L2 ? sqrt(s - c) : s - c);
}

// ---------------------------------------------------------------- launching
struct Plan {
  SweepParams P;
  int threads = 0;
  long long work = 0;         // (tile, z plane) pairs of a single-grid launch
  int max_ctas = 0x7fffffff;  // CTAs the reduction scratch can take partials from
  size_t smem = 0;
  int op = OP_GENERIC;        // StaticOpId of a matched compile-time operator
  bool batch = false;         // work-list launch of a batch
  int batch_ctas = 0;         // its grid (fixed when the work-list was built)
  bool narrow = false;        // batches of FP32 / BF16 grids: 64-column tiles, 4 rows per warp
  bool pair = false;          // FP64 grids in pair arithmetic (fixed when the plan is made)
  bool compact = false;       // colour-compacted red-black sweep (XS = 2 tiles)
  bool vec = false;           // vector lanes (StaticOpV): FP32 / BF16 compile-time operators
  bool eqw = false;           // IEEE FP64 group evaluation: StaticOp<Def, XS, true> (batches: some instance)
  bool eq_mixed = false;      // batches: only some instances allow it (a flag per instance)
  int tile_x = 0, tile_y = 0; // core elements per CTA tile
};

// Columns (TX = 32 VX) and rows (VY) per thread for each storage dtype: two
// rows give each thread independent FMA chains and halve the per-point share
// of the per-plane synchronisation.
template <typename T> struct VxOf { static constexpr int value = 4; };
template <> struct VxOf<double> { static constexpr int value = 2; };
template <> struct VxOf<f64pair> { static constexpr int value = 2; };
template <typename T> struct VyOf { static constexpr int value = 2; };
template <> struct VyOf<double> { static constexpr int value = 2; };

// Launches one wave: as many CTAs as the device holds at once (occupancy
// query per kernel and shape, cached), never more than there is work.  With
// occupancy_only set, reports resident CTAs per SM instead of launching.
template <typename T, int VX, int RED, class Op, bool BATCH, int VY = VyOf<T>::value>
gscl_status launch_t(const Plan &pl, cudaStream_t stream, int *occupancy_only) {
  auto kern = sweep_kernel<T, VX, VY, RED, Op, BATCH>;
  static std::mutex mu;
  // the shared-memory limit raised so far, per device (a function attribute
  // is set on the current device only)
  constexpr int kAttrDevices = 64;
  static size_t attr_set[kAttrDevices] = {};
  static int cached_threads = -1, cached_blocks = 0, cached_dev = -1;
  static size_t cached_smem = 0;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= kAttrDevices || pl.smem > attr_set[dev]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
      if (dev >= 0 && dev < kAttrDevices) attr_set[dev] = pl.smem;
    }
    if (cached_threads != pl.threads || cached_smem != pl.smem || cached_dev != dev) {
      int nb = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, pl.threads, pl.smem);
      if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
      cached_threads = pl.threads;
      cached_smem = pl.smem;
      cached_dev = dev;
      cached_blocks = nb > 0 ? nb : 1;
    }
    per_sm = cached_blocks;
  }
  if (occupancy_only) {
    *occupancy_only = per_sm;
    return GSCL_OK;
  }
  const long long slots = (long long)sm_count() * per_sm;
  long long ctas = BATCH ? (long long)pl.batch_ctas : std::min<long long>(pl.work, slots);
  if (!BATCH && pl.P.zalt) {
    // column-aligned wave: k z ranges per tile column (see sweep_kernel)
    const long long cols = (long long)pl.P.inst.tiles_x * pl.P.inst.tiles_y;
    const long long nz = pl.P.inst.hi[2] - pl.P.inst.lo[2];
    // only where it keeps at least 90% of the CTA slots busy
    if (cols > 0 && cols <= slots && nz > 0) {
      const long long aligned = cols * std::min(nz, slots / cols);
      if (10 * aligned >= 9 * std::min(pl.work, slots)) ctas = aligned;
    }
  }
  if (ctas > pl.max_ctas)
    return fail(GSCL_ERR_UNSUPPORTED,
                "this launch needs %lld partial sums but the reduction scratch holds %d", ctas, pl.max_ctas);
  if (ctas < 1) return GSCL_OK;
  // programmatic dependent launch: the kernel waits for its predecessor on
  // the stream itself, so the launch latency overlaps the previous sweep
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)ctas);
  cfg.blockDim = dim3((unsigned)pl.threads);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kern, pl.P);
  if (e != cudaSuccess) return cuda_fail(e, "sweep kernel launch");
  return GSCL_OK;
}

// Operator structures that batched launches are compiled for.
template <class Def> struct BatchCapable { static constexpr bool value = false; };
template <> struct BatchCapable<OpHeat7Rhs> { static constexpr bool value = true; };
template <> struct BatchCapable<OpStar7> { static constexpr bool value = true; };
template <> struct BatchCapable<OpJacobi7Rhs> { static constexpr bool value = true; };
template <> struct BatchCapable<OpHeat7RhsFused> { static constexpr bool value = true; };
template <> struct BatchCapable<OpHeat7Fused> { static constexpr bool value = true; };
template <> struct BatchCapable<OpResidual7Rhs> { static constexpr bool value = true; };
template <> struct BatchCapable<OpIdentity> { static constexpr bool value = true; };
template <> struct BatchCapable<OpJacobi5_2D> { static constexpr bool value = true; };

// Operator structures with a colour-compacted kernel (red-black Gauss-Seidel
// and SOR of the 7-point and 2D 5-point families, FP64 grids).
template <class Def> struct CompactCapable { static constexpr bool value = false; };
template <> struct CompactCapable<OpHeat7Rhs> { static constexpr bool value = true; };
template <> struct CompactCapable<OpStar7> { static constexpr bool value = true; };
template <> struct CompactCapable<OpJacobi7Rhs> { static constexpr bool value = true; };
template <> struct CompactCapable<OpJacobi5_2D> { static constexpr bool value = true; };

inline bool compact_capable(int op) {
  return op == OP_HEAT7_RHS || op == OP_STAR7 || op == OP_JACOBI7_RHS || op == OP_JACOBI5_2D;
}

inline bool batch_capable(int op) {
  return op == OP_HEAT7_RHS || op == OP_STAR7 || op == OP_JACOBI7_RHS || op == OP_HEAT7_RHS_FUSED ||
         op == OP_HEAT7_FUSED || op == OP_RESIDUAL7_RHS || op == OP_IDENTITY || op == OP_JACOBI5_2D;
}

// Launches the compile-time operator pl.op for storage type T (one
// translation unit per dtype instantiates these).
gscl_status launch_static_f64(const Plan &pl, int red, cudaStream_t stream, int *occupancy_only);
gscl_status launch_static_f32(const Plan &pl, int red, cudaStream_t stream, int *occupancy_only);
gscl_status launch_static_bf16(const Plan &pl, int red, cudaStream_t stream, int *occupancy_only);
gscl_status launch_static_f64pair(const Plan &pl, int red, cudaStream_t stream, int *occupancy_only);

template <typename T, int RED, class Def, bool BATCH>
gscl_status launch_op(const Plan &pl, cudaStream_t stream, int *occ) {
  if constexpr (RED != RED_NONE && !op_has_value<Def>()) {
    return fail(GSCL_ERR_INVALID, "reduction of an operator without a value");
  } else if constexpr (RED == RED_NONE && Def::NOUT == 0) {
    return fail(GSCL_ERR_INVALID, "sweep of an operator without outputs");
  } else if constexpr (BATCH && !BatchCapable<Def>::value) {
    return fail(GSCL_ERR_INVALID, "no batched kernel for this operator structure");
  } else {
    if constexpr (!IsFp64Storage<T>::value) {
      // narrow tiles (64 x 4 rows per warp, the same 8 points per thread) for
      // batches of FP32 / BF16 grids whose widths leave 128-column tiles idle
      if constexpr (BATCH) {
        if (pl.narrow) return launch_t<T, 2, RED, StaticOp<Def>, BATCH, 4>(pl, stream, occ);
      }
      // vector lanes: 16 bytes of a row per lane (every compile-time table fits)
      constexpr int G = 16 / (int)sizeof(T);
      static_assert(StaticOpV<Def, G>::fits(), "x reach beyond one group");
      if (!pl.vec) return fail(GSCL_ERR_INVALID, "FP32 / BF16 plan without vector lanes");
      return launch_t<T, G, RED, StaticOpV<Def, G>, BATCH>(pl, stream, occ);
    } else {
      // colour-compacted red-black sweeps of the star family on FP64 grids
      // (IEEE or pair arithmetic), single grids and coloured batches
      if constexpr (RED == RED_NONE && CompactCapable<Def>::value) {
        if (pl.compact) {
          if constexpr (std::is_same<T, double>::value && has_groups<Def>()) {
            if constexpr (BATCH) {
              if (pl.eqw && pl.eq_mixed)
                return launch_t<T, VxOf<T>::value, RED, StaticOp<Def, 2, true, true>, BATCH>(pl, stream, occ);
            }
            if (pl.eqw) return launch_t<T, VxOf<T>::value, RED, StaticOp<Def, 2, true>, BATCH>(pl, stream, occ);
          }
          return launch_t<T, VxOf<T>::value, RED, StaticOp<Def, 2>, BATCH>(pl, stream, occ);
        }
      }
      // equal axial weights: the neighbour sum partly on the integer pipe
      if constexpr (std::is_same<T, double>::value && has_groups<Def>()) {
        if constexpr (BATCH) {
          if (pl.eqw && pl.eq_mixed)
            return launch_t<T, VxOf<T>::value, RED, StaticOp<Def, 1, true, true>, BATCH>(pl, stream, occ);
        }
        if (pl.eqw) return launch_t<T, VxOf<T>::value, RED, StaticOp<Def, 1, true>, BATCH>(pl, stream, occ);
      }
      return launch_t<T, VxOf<T>::value, RED, StaticOp<Def>, BATCH>(pl, stream, occ);
    }
  }
}

template <typename T, int RED, bool BATCH>
gscl_status launch_static_red(const Plan &pl, cudaStream_t stream, int *occ) {
  switch (pl.op) {
    case OP_HEAT7_RHS: return launch_op<T, RED, OpHeat7Rhs, BATCH>(pl, stream, occ);
    case OP_STAR7: return launch_op<T, RED, OpStar7, BATCH>(pl, stream, occ);
    case OP_JACOBI7_RHS: return launch_op<T, RED, OpJacobi7Rhs, BATCH>(pl, stream, occ);
    case OP_JACOBI5_2D: return launch_op<T, RED, OpJacobi5_2D, BATCH>(pl, stream, occ);
    case OP_CLIMATE: return launch_op<T, RED, OpClimate, BATCH>(pl, stream, occ);
    case OP_HEAT7_RHS_FUSED: return launch_op<T, RED, OpHeat7RhsFused, BATCH>(pl, stream, occ);
    case OP_HEAT7_FUSED: return launch_op<T, RED, OpHeat7Fused, BATCH>(pl, stream, occ);
    case OP_RESIDUAL7_RHS: return launch_op<T, RED, OpResidual7Rhs, BATCH>(pl, stream, occ);
    case OP_DIFFERENCE: return launch_op<T, RED, OpDifference, BATCH>(pl, stream, occ);
    case OP_IDENTITY: return launch_op<T, RED, OpIdentity, BATCH>(pl, stream, occ);
  }
  return fail(GSCL_ERR_INVALID, "unknown compile-time operator %d", pl.op);
}

template <typename T, bool BATCH>
gscl_status launch_static_b(const Plan &pl, int red, cudaStream_t stream, int *occ) {
  switch (red) {
    case RED_NONE: return launch_static_red<T, RED_NONE, BATCH>(pl, stream, occ);
    case RED_SUM: return launch_static_red<T, RED_SUM, BATCH>(pl, stream, occ);
    case RED_MAXABS: return launch_static_red<T, RED_MAXABS, BATCH>(pl, stream, occ);
    case RED_L2: return launch_static_red<T, RED_L2, BATCH>(pl, stream, occ);
  }
  return fail(GSCL_ERR_INVALID, "unknown reduction");
}

template <typename T>
gscl_status launch_static_t(const Plan &pl, int red, cudaStream_t stream, int *occ) {
  return pl.batch ? launch_static_b<T, true>(pl, red, stream, occ) : launch_static_b<T, false>(pl, red, stream, occ);
}

}  // namespace gscl
