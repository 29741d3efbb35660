// FP64 grids evaluated in pairs of FP32 numbers ("pair" arithmetic).
//
// On B300 the FP64 pipe executes about 1.7 fused multiply-adds per clock per
// SM against 128 for FP32, so an FP64 sweep is bound by that pipe at a fifth
// of HBM bandwidth.  In pair mode a stored double x is split on the integer
// pipe into hi + lo (hi: x truncated to 24 significant bits, lo: the next 24
// bits of the remainder, so x - (hi + lo) is below 2^-47 |x|), each term
// w x is accumulated with an exact FP32 two-product and Knuth's two-sum on
// the high parts (the low parts summed in FP32), and the result is stored
// as the double nearest hi + lo (one FP64 add per stored element).  The
// arithmetic error of an operator is then a small multiple of 2^-47 times
// sum_t |w_t x_t| (the absolute stencil), against 2^-53 for IEEE FP64.
// A pair spans FP32's exponent range: magnitudes from about 2^-100 (below,
// the low part underflows) to below 2^128 (above, the high part overflows).
// Storage, TMA traffic and reductions (FP64 accumulation) are unchanged.
#pragma once

#include <stdint.h>

namespace gscl {

// Storage tag: an FP64 grid read and written by the pair arithmetic.
struct f64pair {
  double v;
};

struct Df64 {
  float hi, lo;
  Df64() = default;
  __device__ __forceinline__ Df64(int z) : hi((float)z), lo(0.f) {}
  __device__ __forceinline__ Df64(float h, float l) : hi(h), lo(l) {}
};

// x -> hi + lo: hi keeps the sign, exponent and top 23 fraction bits of x
// (integer pipe); lo is the 29-bit remainder converted to float (rounded to
// 24 bits) and scaled by 2^(E - 52) with an exponent add, which stays exact
// while the result is normal.  Normal doubles with 2^-74 <= |x| < 2^128 take
// this path; zero is a signed zero pair; anything else (tiny, huge, inf,
// NaN) takes the hardware conversions.
__device__ __forceinline__ Df64 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
  const unsigned sign = h32 & 0x80000000u;
  const int E = (int)((h32 >> 20) & 0x7ffu) - 1023;  // unbiased exponent
  if (E >= -74 && E <= 127) {
    const unsigned hb = sign | ((unsigned)(E + 127) << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    const unsigned rem = l32 & 0x1fffffffu;  // worth rem * 2^(E - 52)
    const unsigned r = __float_as_uint(__uint2float_rn(rem));
    const unsigned lb = rem ? (sign | (r + ((unsigned)(E - 52) << 23))) : sign;
    return Df64(__uint_as_float(hb), __uint_as_float(lb));
  }
  if ((b << 1) == 0) return Df64(__uint_as_float(sign), 0.f);
  const float h = __double2float_rn(x);
  return Df64(h, __double2float_rn(x - (double)h));
}

// Exact float -> double on the integer pipe for normal floats and zeros.
__device__ __forceinline__ double widen_f32(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex - 1u < 254u) {
    const unsigned long long bits = ((unsigned long long)(u & 0x80000000u) << 32) |
                                    ((unsigned long long)(ex + 896u) << 52) |
                                    ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
  }
  if ((u << 1) == 0) return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
  return (double)f;
}

// The double nearest hi + lo (one FP64 add).
__device__ __forceinline__ double combine_f64(Df64 a) { return widen_f32(a.hi) + widen_f32(a.lo); }

// a * b: exact product of the high parts (FMA) plus the cross terms.
__device__ __forceinline__ Df64 operator*(Df64 a, Df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return Df64(p, e);
}

}  // namespace gscl

// acc + w * x: the product as above, the high parts summed with two-sum
// (exact), the low parts and the two-sum error in FP32.  Declared beside the
// global fma overloads (float, double) so that unqualified calls in generic
// kernel code resolve among all three.
__device__ __forceinline__ gscl::Df64 fma(gscl::Df64 w, gscl::Df64 x, gscl::Df64 acc) {
  const float p = w.hi * x.hi;
  float e = fmaf(w.hi, x.hi, -p);
  e = fmaf(w.hi, x.lo, e);
  e = fmaf(w.lo, x.hi, e);
  const float s = acc.hi + p;
  const float bb = s - acc.hi;
  const float err = (acc.hi - (s - bb)) + (p - bb);
  return gscl::Df64(s, (acc.lo + e) + err);
}
