// IEEE 754 binary64 addition on the integer pipe.
//
// The IEEE FP64 sweeps are bound by the FP64 pipe while most of their
// instruction issue slots stay free.  An addition computed from the binary64
// definition with integer instructions gives the same bits as the FP64 adder
// and runs on the integer pipe, so moving a few of a sweep's additions there
// shortens the FP64 pipe's share of the work.
//
// The method is the textbook one for round-to-nearest-even addition: order
// the operands by magnitude, align the smaller significand with three extra
// bits (guard, round, and a sticky bit that ORs in everything shifted out),
// add or subtract the significands, normalise (a carry shifts right by one
// position, keeping the sticky bit; a cancellation shifts left by the
// leading-zero count, and is exact whenever it shifts by more than one),
// round on the three extra bits with ties to even, and repack.  One shift
// normalises in either direction, the rounding is an addition, and the
// exponent field absorbs a rounding carry (the packed value is
// (e - 1) * 2^52 + m with the hidden bit in m); only the rare special cases
// are a select at the end.
//
// It is exact for every input: subnormal operands align with exponent 1 and
// no hidden bit, a result below the normal range keeps exponent 1 (a sum
// that underflows is exact, so nothing is rounded there), a rounded
// exponent of 2047 is an infinity, and infinities and NaNs take the IEEE
// result (an infinity, or the default NaN for NaN operands and inf - inf).
#pragma once

namespace gscl {

// Leading zeros of a 64-bit value (64 for zero).
__host__ __device__ __forceinline__ int fp64_int_clz(unsigned long long m) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)m);
#else
  return m ? __builtin_clzll(m) : 64;
#endif
}

// Bits of a + b, IEEE 754 binary64 rounded to nearest even.
__host__ __device__ __forceinline__ unsigned long long fp64_add_int_bits(unsigned long long ua,
                                                                         unsigned long long ub) {
  constexpr unsigned long long kFrac = (1ull << 52) - 1ull, kHidden = 1ull << 52, kSign = 1ull << 63;
  constexpr unsigned long long kInf = 0x7ffull << 52, kNaN = 0x7fffffffffffffffull;
  // |a| >= |b|: magnitudes order as their bit patterns do
  if ((ub & ~kSign) > (ua & ~kSign)) {
    const unsigned long long t = ua;
    ua = ub;
    ub = t;
  }
  const unsigned ea = (unsigned)(ua >> 52) & 0x7ffu, eb = (unsigned)(ub >> 52) & 0x7ffu;
  const bool sub = ((ua ^ ub) & kSign) != 0ull;
  // significands with the hidden bit of a normal number, three extra bits;
  // subnormals (and zeros) count with exponent 1
  const unsigned long long ma = ((ua & kFrac) | (ea ? kHidden : 0ull)) << 3;
  const unsigned long long mb = ((ub & kFrac) | (eb ? kHidden : 0ull)) << 3;
  const int ea1 = ea ? (int)ea : 1, eb1 = eb ? (int)eb : 1;
  // alignment; a shift of 63 leaves only the sticky bit of a nonzero b
  // (mb < 2^56)
  unsigned d = (unsigned)(ea1 - eb1);
  d = d < 63u ? d : 63u;
  unsigned long long mbs = mb >> d;
  mbs |= (mbs << d) != mb ? 1ull : 0ull;
  const unsigned long long m = sub ? ma - mbs : ma + mbs;  // below 2^57
  // normalise the leading bit to position 55 (lz = -1 after a carry), but
  // not below exponent 1.  One shift serves both directions: after a carry
  // the bit shifted out is ORed back as the sticky bit; after a left shift
  // the OR is harmless (m's bit 0 is a sticky bit that can only be set when
  // lz <= 1, and there it leaves the rounding decision unchanged).
  int lz = fp64_int_clz(m) - 8;
  lz = lz < ea1 - 1 ? lz : ea1 - 1;
  const unsigned long long mn = ((m << (lz + 1)) >> 1) | (m & 1ull);
  const int e = ea1 - lz;
  // round to nearest, ties to even: adding 3 + lsb carries out of the three
  // extra bits exactly when they exceed one half, or equal it with an odd
  // lsb.  The exponent field takes a carry out of the significand (and a
  // subnormal's missing hidden bit leaves it at 0).
  const unsigned long long q = (mn + 3ull + ((mn >> 3) & 1ull)) >> 3;
  unsigned long long r = (ua & kSign) | (((unsigned long long)(e - 1) << 52) + q);
  // an exact zero: +0 for opposite signs, else the common sign
  r = m == 0ull ? (sub ? 0ull : (ua & kSign)) : r;
  // overflow (the normalised exponent reached 2047) and infinite or NaN
  // operands (a has the larger magnitude): an infinity of a's sign, or the
  // default NaN for a NaN operand and for inf - inf
  if (e >= 2047 || ea == 0x7ffu) {
    const bool nan = ea == 0x7ffu && ((ua & kFrac) != 0ull || (ua ^ ub) == kSign);
    r = nan ? kNaN : ((ua & kSign) | kInf);
  }
  return r;
}

#ifdef __CUDACC__
__device__ __forceinline__ double fp64_add_int(double a, double b) {
  return __longlong_as_double((long long)fp64_add_int_bits((unsigned long long)__double_as_longlong(a),
                                                           (unsigned long long)__double_as_longlong(b)));
}
#endif

}  // namespace gscl
