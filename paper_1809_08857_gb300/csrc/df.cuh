// Double-float arithmetic and FP32 <-> FP64 conversions on the integer pipe.
//
// On GB300 the FP64 pipe issues about 1/57 of the FP32 rate, so kernels that
// need FP64 accuracy on FP64 data (the refinement residual, the electric
// field) carry values as double-floats: unevaluated sums hi + lo of two FP32
// numbers with |lo| <= ulp(hi), 48 significant bits.  Products and sums are
// made exact with the error-free transformations of Dekker (product via FMA)
// and Knuth (two-sum); the _rn intrinsics keep the compiler from contracting
// or reassociating them.
#ifndef MG_DF_CUH
#define MG_DF_CUH

namespace mg {
namespace df {

// IEEE-754 binary32 -> binary64 by re-biasing the exponent (1023 - 127 = 896)
// and widening the fraction, on the integer pipe.  Zeros and binary32
// subnormals (< 1.2e-38, never reached by a correction of a physical field)
// map to a signed zero; infinities and NaNs keep their class.
__device__ __forceinline__ double widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned long long sgn = (unsigned long long)(b >> 31) << 63;
  const unsigned ex = (b >> 23) & 0xffu;
  const unsigned long long man = (unsigned long long)(b & 0x7fffffu) << 29;
  const unsigned long long e64 = ex == 0xffu ? 0x7ffull : (unsigned long long)ex + 896ull;
  const unsigned long long bits = ex == 0u ? sgn : (sgn | (e64 << 52) | man);
  return __longlong_as_double((long long)bits);
}

// binary64 -> binary32 by truncation (round toward zero: at most one FP32
// ulp, harmless for the right-hand side of the FP32 inner cycle), integer
// pipe.  Values below the binary32 normal range flush to zero, values above
// it become infinity, NaN stays NaN.
__device__ __forceinline__ float narrow(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 63) << 31;
  const int ex = (int)((b >> 52) & 0x7ffull);
  const unsigned man = (unsigned)((b >> 29) & 0x7fffffull);
  const int e32 = ex - 896;
  unsigned bits;
  if (ex == 0x7ff) bits = sgn | 0x7f800000u | (man ? 0x400000u : 0u);
  else if (e32 >= 255) bits = sgn | 0x7f800000u;
  else if (e32 <= 0) bits = sgn;
  else bits = sgn | ((unsigned)e32 << 23) | man;
  return __uint_as_float(bits);
}

// binary64 -> double-float without an FP64 instruction: hi = x truncated to
// 24 significant bits (integer pipe), lo = the remaining 29 bits rounded to
// FP32 (one integer -> float conversion and a power-of-two scale).  For
// |x| < 2^-74 lo is dropped; below the FP32 normal range x flushes to 0.
__device__ __forceinline__ float2 split_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const float hi = narrow(x);
  const int se = (int)((b >> 52) & 0x7ffull) - 948;  // FP32 exponent field of 2^(ex - 1075)
  const float scale = (se >= 1 && se <= 254) ? __uint_as_float((unsigned)se << 23) : 0.0f;
  const float lo = __fmul_rn(__uint2float_rn((unsigned)(b & 0x1fffffffull)), scale);
  return make_float2(hi, (b >> 63) ? -lo : lo);
}

// Running sum s + e of double-float products.  add(c, u): s + e += c * u.
// The product's rounding error (FMA) and its cross terms, and the two-sum
// error of s, go into e; e itself is a plain FP32 sum of terms 2^-24 below
// the leading ones, so the total error stays near 2^-48 of the largest term.
struct DfAcc {
  float s, e;
  __device__ __forceinline__ void add(float2 c, float2 u) {
    const float p = __fmul_rn(c.x, u.x);
    float q = fmaf(c.x, u.x, -p);
    q = fmaf(c.x, u.y, q);
    q = fmaf(c.y, u.x, q);
    const float t = __fadd_rn(s, p);
    const float v = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(p, v));
    s = t;
    e = __fadd_rn(e, __fadd_rn(err, q));
  }
  __device__ __forceinline__ float value() const { return __fadd_rn(s, e); }
};

// a + b (double-float plus FP32) renormalised: two-sum of the leading parts,
// then the fast two-sum of the result with the low parts.
__device__ __forceinline__ float2 df_add(float2 a, float b) {
  const float s = __fadd_rn(a.x, b);
  const float v = __fsub_rn(s, a.x);
  const float t = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b, v));
  const float lo = __fadd_rn(t, a.y);
  const float hi = __fadd_rn(s, lo);
  return make_float2(hi, __fsub_rn(lo, __fsub_rn(hi, s)));
}

// ---- paired forms: two cells at once ----------------------------------------
//
// The same error-free steps lane by lane on float2 values (lane x: cell A,
// lane y: cell B) with the FP32x2 instructions of sm_100 and later (one
// FADD2 / FMUL2 / FFMA2 does two correctly rounded FP32 operations), so two
// cells cost the instructions of one.  a - b is formed as fma(b, -1, a): the
// product is exact, so the single rounding gives the correctly rounded
// difference.

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// A pair of double-floats: hi = (A.hi, B.hi), lo = (A.lo, B.lo).
struct Df2 {
  float2 hi, lo;
};

// Running sums s + e of the pair (DfAcc lane by lane).
struct DfAcc2 {
  float2 s, e;
  // s + e += c * u, c and u pairs of double-floats
  __device__ __forceinline__ void add(const Df2& c, const Df2& u) {
    const float2 p = mul2(c.hi, u.hi);
    float2 q = fma2(c.hi, u.hi, make_float2(-p.x, -p.y));
    q = fma2(c.hi, u.lo, q);
    q = fma2(c.lo, u.hi, q);
    const float2 t = add2(s, p);
    const float2 v = sub2(t, s);
    const float2 err = add2(sub2(s, sub2(t, v)), sub2(p, v));
    s = t;
    e = add2(e, add2(err, q));
  }
  __device__ __forceinline__ float2 value() const { return add2(s, e); }
};

// Running double-float sums s + e of pairs of double-floats: two-sum of the
// leading parts (exact), the low parts and the two-sum errors summed in FP32
// into e.  The neighbour sum of a constant-coefficient stencil, formed before
// its one product by 1/h^2 (8 operations per term against 12 for a product
// and sum).  s + e need not be renormalised before the product: e stays a few
// ulp of s.
struct DfSum2 {
  float2 s, e;
  __device__ __forceinline__ void add(const Df2& v) {
    const float2 t = add2(s, v.hi);
    const float2 bv = sub2(t, s);
    const float2 err = add2(sub2(s, sub2(t, bv)), sub2(v.hi, bv));
    s = t;
    e = add2(e, add2(err, v.lo));
  }
};

// a + b (pair of double-floats plus a pair of FP32), renormalised (df_add
// lane by lane).
__device__ __forceinline__ Df2 df_add2(const Df2& a, float2 b) {
  const float2 s = add2(a.hi, b);
  const float2 v = sub2(s, a.hi);
  const float2 t = add2(sub2(a.hi, sub2(s, v)), sub2(b, v));
  const float2 lo = add2(t, a.lo);
  const float2 hi = add2(s, lo);
  return Df2{hi, sub2(lo, sub2(hi, s))};
}

// a + b for a pair of double-floats plus one double-float b (the same b for
// both cells), renormalised: two-sum of the leading parts, the low parts and
// the two-sum error summed, then a fast two-sum.
__device__ __forceinline__ Df2 df_add_df2(const Df2& a, float2 b) {
  const float2 bh = make_float2(b.x, b.x), bl = make_float2(b.y, b.y);
  const float2 s = add2(a.hi, bh);
  const float2 v = sub2(s, a.hi);
  const float2 t = add2(add2(sub2(a.hi, sub2(s, v)), sub2(bh, v)), add2(a.lo, bl));
  const float2 hi = add2(s, t);
  return Df2{hi, sub2(t, sub2(hi, s))};
}

}  // namespace df
}  // namespace mg

#endif
