// Double-float arithmetic for the FP64 form's FFT line passes: a value is the
// unevaluated sum hi + lo of two floats, |lo| <= ulp(hi) / 2, about 48
// significant bits.  GB300 issues FP32 operations at about 77 times its FP64
// rate, so a transform carried in pairs of floats (roughly ten FP32
// operations per FP64 one) runs several times faster than in FP64, with
// relative errors of a few 2^-48 per operation -- far inside the FP64 form's
// 1e-12 per-call tolerance.  Building blocks (Dekker 1971; Knuth, TAOCP 2,
// 4.2.2; Joldes, Muller and Popescu, ACM TOMS 44 (2017)):
//   TwoSum(a, b)      s = fl(a + b) and the exact error e, a + b = s + e;
//   FastTwoSum(a, b)  the same for |a| >= |b|, three operations;
//   sum               TwoSum of the high parts, the low parts added to the
//                     error, renormalised by FastTwoSum ("sloppy" pair sum:
//                     error a few u^2 of |x| + |y|, u = 2^-24, the normwise
//                     bound an FFT needs);
//   product           FMA gives the exact error of the high product; the
//                     cross terms are added to it, renormalised by FastTwoSum.
// Every operation whose rounding the construction relies on is written with
// the _rn intrinsics, which the compiler never contracts into FMAs.
#pragma once

#include "sky_internal.cuh"

namespace sky {

struct dd {
  float hi, lo;
  __host__ __device__ constexpr dd() : hi(0.0f), lo(0.0f) {}
  __host__ __device__ constexpr dd(float h, float l) : hi(h), lo(l) {}
  // The nearest pair to x (compile-time constants and host tables).
  __host__ __device__ constexpr explicit dd(double x)
      : hi((float)x), lo((float)(x - (double)(float)x)) {}
};
struct ddc {
  dd x, y;
};
template <> struct CxT<dd> { using type = ddc; };

__device__ __forceinline__ dd two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dd(s, e);
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dd(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dd operator+(dd a, dd b) {
  const dd s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dd operator-(dd a) { return dd(-a.hi, -a.lo); }
__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }
__device__ __forceinline__ dd operator*(dd a, dd b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

__device__ __forceinline__ ddc operator+(ddc a, ddc b) { return ddc{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ ddc operator-(ddc a, ddc b) { return ddc{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ ddc operator-(ddc a) { return ddc{-a.x, -a.y}; }
__device__ __forceinline__ ddc operator*(dd s, ddc a) { return ddc{s * a.x, s * a.y}; }
__device__ __forceinline__ ddc mul_i(ddc a) { return ddc{-a.y, a.x}; }
__device__ __forceinline__ ddc mul_mi(ddc a) { return ddc{a.y, -a.x}; }
__device__ __forceinline__ ddc half(ddc a) {   // exact (barring underflow)
  return ddc{dd(a.x.hi * 0.5f, a.x.lo * 0.5f), dd(a.y.hi * 0.5f, a.y.lo * 0.5f)};
}

// a / b: the quotient of the high parts (hardware reciprocal) corrected
// once by the exact residual a - q1 b; relative error a few 2^-46.
__device__ __forceinline__ dd ddiv(dd a, dd b) {
  const float y = __fdividef(1.0f, b.hi);
  const float q1 = __fmul_rn(a.hi, y);
  const dd r = a - dd(q1, 0.0f) * b;
  const float q2 = __fmul_rn(r.hi, y);
  return fast_two_sum(q1, q2);
}

// double <-> pair.  GB300's FP64 unit issues about one seventieth of the FP32
// rate, and conversions between double and float run on it, so both
// directions work on the bit patterns with integer operations where the
// values allow (normal floats on both sides), keeping the FP64 unit for one
// addition per stored value.
//
// double -> pair: the pattern P of |x| rounded at bit 29 (half up; a carry
// into the exponent is the correct rounding) is hi widened to double; the
// pattern difference P - Ph counts units of 2^(e - 1075) (e the biased
// exponent of x) exactly, also across a binade boundary, since the ulp of
// the lower binade is the unit on both sides; |P - Ph| <= 2^28, so the
// integer-to-float conversion rounds once and lo = that float times
// 2^(e - 1075), an exponent add.  Valid for 949 <= e <= 1149 (hi and lo
// normal floats: 2^-74 <= |x| < 2^127); zeros, smaller or larger magnitudes,
// infinities and NaNs take the FP64 route.
__device__ __forceinline__ dd dd_of_fp64(double x) {
  const float h = __double2float_rn(x);
  return dd(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ dd dd_of(double x) {
  const long long P = __double_as_longlong(x);
  const int e = (int)((P >> 52) & 0x7ff);
  if ((unsigned)(e - 949) > (unsigned)(1149 - 949)) return dd_of_fp64(x);
  const long long Ph = (P + (1LL << 28)) & ~((1LL << 29) - 1);
  const unsigned sgn = (unsigned)(P >> 32) & 0x80000000u;
  const unsigned hb = sgn | ((unsigned)((Ph & 0x7fffffffffffffffLL) >> 29) - (896u << 23));
  const int dl = (int)(P - Ph);
  const float fl = __int2float_rn(dl);
  const unsigned lb = dl == 0 ? 0u : (((unsigned)__float_as_int(fl) + ((unsigned)(e - 1075) << 23)) ^ sgn);
  return dd(__int_as_float((int)hb), __int_as_float((int)lb));
}
// float -> double by its pattern: exponent rebased 127 -> 1023, mantissa
// moved up 29 bits (exact); zeros by select; subnormals, infinities and NaNs
// by the FP64 conversion.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned m = u & 0x7fffffffu;
  const unsigned ef = m >> 23;
  if (ef - 1u >= 254u && m != 0u) return (double)f;
  const long long mag = m == 0u ? 0LL : ((long long)m << 29) + (896LL << 52);
  return __longlong_as_double(mag | ((long long)(u & 0x80000000u) << 32));
}
// hi + lo rounded to a double by integer operations: hi widened exactly; lo
// counted in units of the last place of hi's double, an integer shift of
// lo's significand (rounded half up when the unit is coarser), added to or
// subtracted from hi's pattern.  For a normalised pair (|lo| <= ulp(hi) / 2,
// what every operation here returns) the count stays below 2^28, so the sum
// never leaves hi's binade, except downwards from a power of two, where the
// unit of the binade below (half as large) is used.  Zeros, subnormals,
// infinities, NaNs and pairs with |lo| > 2^-24 |hi| take one FP64 addition.
__device__ __forceinline__ double dbl_of(dd a) {
  const unsigned uh = __float_as_uint(a.hi), ul = __float_as_uint(a.lo);
  const unsigned mh = uh & 0x7fffffffu, ml = ul & 0x7fffffffu;
  const int eh = (int)(mh >> 23), el = (int)(ml >> 23);
  const long long sgn = (long long)(uh & 0x80000000u) << 32;
  if (ml == 0u && (unsigned)(eh - 1) < 254u)   // exact float: widen
    return __longlong_as_double((((long long)mh << 29) + (896LL << 52)) | sgn);
  if ((unsigned)(eh - 1) >= 254u || (unsigned)(el - 1) >= 254u || eh - el < 24)
    return __dadd_rn(widen(a.hi), widen(a.lo));
  long long hd = ((long long)mh << 29) + (896LL << 52);     // |hi| as a double pattern
  const long long sig = (long long)((ul & 0x7fffffu) | 0x800000u);
  const bool same = ((uh ^ ul) & 0x80000000u) == 0u;
  const bool down = !same && (mh & 0x7fffffu) == 0u;       // |hi| a power of two, decreasing
  const int sh = 29 - (eh - el) + (down ? 1 : 0);           // |lo| / unit = sig 2^sh
  long long K;
  if (sh >= 0) {
    K = sig << sh;
  } else {
    const int r = -sh;
    K = r > 25 ? 0 : ((sig >> (r - 1)) + 1) >> 1;
  }
  hd = same ? hd + K : hd - K;
  return __longlong_as_double(hd | sgn);
}
__device__ __forceinline__ ddc ddc_of(double2 v) { return ddc{dd_of(v.x), dd_of(v.y)}; }

// A sum of products of floats in a float pair (the FP32 forms' reductions):
// a b = p + e exactly (e from an FMA); p joins the high part by TwoSum and
// both errors collect in the low part, so each term costs a few FP32
// operations instead of FP64 ones, about 2^-48 of the running sum per term.
struct AccF {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(err, e));
  }
  // sign * Re(conj(a) d) and sign * Im(conj(a) d) (sign +-1: exact)
  __device__ __forceinline__ void re_cj(float sg, float2 a, float2 d) {
    add_prod(a.x, sg * d.x);
    add_prod(a.y, sg * d.y);
  }
  __device__ __forceinline__ void im_cj(float sg, float2 a, float2 d) {
    add_prod(a.x, sg * d.y);
    add_prod(a.y, -sg * d.x);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ double2 dbl2_of(ddc v) { return make_double2(dbl_of(v.x), dbl_of(v.y)); }

}  // namespace sky
