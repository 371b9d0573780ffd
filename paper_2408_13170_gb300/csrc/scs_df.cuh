// scs_df.cuh -- double-float arithmetic: a value is the unevaluated sum
// hi + lo of two FP32 numbers (|lo| <= ulp(hi)/2), about 48 significant
// bits.  GB300 issues FP32 instructions at many times its FP64 rate, so
// work that needs near-FP64 precision but only a moderate exponent range
// (angles, unit vectors, the response's complex sums) runs faster this way.
//
// The error-free transformations are Knuth's two-sum, Dekker's fast
// two-sum (|a| >= |b|) and the FMA two-product; the rounded operations are
// written with the _rn intrinsics so that the compiler cannot contract a
// product and a sum into an FMA and break them.  Addition is the cheap
// variant (one two-sum on the high parts): its error is bounded by a few
// units of 2^-48 relative to |a| + |b|, which is the bound the users of
// this header need (sums of bounded terms, not cancellation-sensitive
// differences of large ones).
#pragma once
#include <cuda_runtime.h>

namespace scs {

struct dfl {
  float hi, lo;
};

// split of a double constant (evaluated at compile time for constants)
__host__ __device__ constexpr dfl df_const(double x) {
  return dfl{(float)x, (float)(x - (double)(float)x)};
}
__device__ __forceinline__ dfl df_from(double x) {
  const float h = __double2float_rn(x);
  return dfl{h, __double2float_rn(x - (double)h)};
}

// The split (df_split) and the join back to a double (df_join) with integer
// operations on the bit patterns instead of FP64 conversion instructions
// (which GB300 issues at its FP64 rate).  Valid for 0 and for magnitudes
// whose parts are normal floats (about 1e-30 .. 1e38).  df_split: hi = x
// rounded to 24 significant bits (ties away from zero), lo = x - hi rounded
// to FP32.
__device__ __forceinline__ dfl df_split(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned long long m = b & 0x7fffffffffffffffULL;
  if (m == 0ULL) return dfl{0.f, 0.f};
  if (m < (964ULL << 52) || m >= (1150ULL << 52)) return df_from(x);   // outside 2^-59 .. 2^127
  const unsigned long long mr = (m + (1ULL << 28)) & ~((1ULL << 29) - 1ULL);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int eh = (int)(mr >> 52) - 1023;   // exponent of hi
  const unsigned hb = sign | ((unsigned)(eh + 127) << 23) | (unsigned)((mr >> 29) & 0x7fffffULL);
  // lo = (m - mr) units of 2^(ex - 52), ex the exponent of x
  const int ex = (int)(m >> 52) - 1023;
  const int r = (int)((long long)m - (long long)mr);
  const float scale = __int_as_float((ex - 52 + 127) << 23);
  const float lo = (float)r * scale;
  return dfl{__int_as_float((int)hb), sign ? -lo : lo};
}
// exact FP32 -> FP64 of a normal float (or 0) by its bits
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = (unsigned)__float_as_int(f);
  const unsigned mag = u & 0x7fffffffu;
  if (mag == 0u) return 0.0;
  if (mag < 0x00800000u || mag >= 0x7f800000u) return (double)f;   // subnormal, inf, nan
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned long long e = (unsigned long long)((mag >> 23) + 896u) << 52;
  const unsigned long long mant = (unsigned long long)(mag & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(sign | e | mant));
}
__device__ __forceinline__ double df_join(dfl a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }
__device__ __forceinline__ dfl df_f(float x) { return dfl{x, 0.f}; }

__device__ __forceinline__ dfl df_fast(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dfl{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return dfl{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl{-a.hi, -a.lo}; }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast(p, e);
}
__device__ __forceinline__ dfl operator*(dfl a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_fast(p, e);
}
// exact scaling by a power of two
__device__ __forceinline__ dfl df_scale2(dfl a, float p2) { return dfl{a.hi * p2, a.lo * p2}; }

// a / b: FP32 quotient refined by one correction from the double-float
// residual a - b q1 (relative error ~1e-14)
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, rb);
  const dfl r = a - b * q1;
  return df_fast(q1, __fmul_rn(r.hi, rb));
}

struct cdfl {
  dfl re, im;
};
__device__ __forceinline__ cdfl operator+(cdfl a, cdfl b) { return cdfl{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cdfl operator-(cdfl a, cdfl b) { return cdfl{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cdfl operator*(cdfl a, cdfl b) {
  return cdfl{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
__device__ __forceinline__ cdfl cdf_conj(cdfl a) { return cdfl{a.re, -a.im}; }
__device__ __forceinline__ dfl cdf_norm2(cdfl a) { return a.re * a.re + a.im * a.im; }

// sin and cos of |r| <= pi/4 + a little (Taylor series, 1/n! coefficients).
// The terms from r^11 (sin) and r^10 (cos) on are below 3e-8 of the result
// and are summed in FP32, the rest in double-float; truncation after r^17
// and r^16 is below 1e-17.
__device__ __forceinline__ void df_sincos_small(dfl r, dfl* s, dfl* c) {
  const dfl r2 = r * r;
  const float y = r2.hi;
  float ts = 2.81145725434552076e-15f;          //  1/17!
  ts = fmaf(ts, y, -7.64716373181981648e-13f);  // -1/15!
  ts = fmaf(ts, y, 1.60590438368216146e-10f);   //  1/13!
  ts = fmaf(ts, y, -2.50521083854417188e-08f);  // -1/11!
  float tc = 4.77947733238738530e-14f;          //  1/16!
  tc = fmaf(tc, y, -1.14707455977297247e-11f);  // -1/14!
  tc = fmaf(tc, y, 2.08767569878680990e-09f);   //  1/12!
  tc = fmaf(tc, y, -2.75573192239858907e-07f);  // -1/10!
  constexpr dfl i9 = df_const(1.0 / 362880.0), i7 = df_const(-1.0 / 5040.0),
                i5 = df_const(1.0 / 120.0), i3 = df_const(-1.0 / 6.0);
  constexpr dfl i8 = df_const(1.0 / 40320.0), i6 = df_const(-1.0 / 720.0),
                i4 = df_const(1.0 / 24.0);
  dfl ps = df_f(ts) * r2 + i9;
  ps = ps * r2 + i7;
  ps = ps * r2 + i5;
  ps = ps * r2 + i3;
  *s = (ps * r2) * r + r;
  dfl pc = df_f(tc) * r2 + i8;
  pc = pc * r2 + i6;
  pc = pc * r2 + i4;
  pc = pc * r2 + df_f(-0.5f);
  *c = pc * r2 + df_f(1.0f);
}

// sin and cos of |x| <= pi (+ a little): reduction by multiples of pi/2 with
// pi/2 in three FP32 parts (k pi/2 exact in double-float for |k| <= 2).
__device__ __forceinline__ void df_sincos(dfl x, dfl* s, dfl* c) {
  const float k = rintf(x.hi * 0.636619772367581343f);
  constexpr float p1 = 1.5707963705062866f;        // pi/2 to FP32
  constexpr float p2 = -4.371138828673793e-08f;     // pi/2 - p1 to FP32
  constexpr float p3 = -1.7151245100058819e-15f;    // pi/2 - p1 - p2 (rest ~1e-23)
  dfl r = x - dfl{k * p1, 0.f};   // k * p1 is exact (|k| <= 2)
  r = r - df_f(k) * dfl{p2, p3};
  dfl sr, cr;
  df_sincos_small(r, &sr, &cr);
  const int q = (int)k & 3;
  *s = q == 0 ? sr : (q == 1 ? cr : (q == 2 ? -sr : -cr));
  *c = q == 0 ? cr : (q == 1 ? -sr : (q == 2 ? -cr : sr));
}

// sin(x)/x for |x| <= 0.3: 1 - x^2/3! + x^4/5! - x^6/7! in double-float,
// the terms from x^8/9! on (below 2e-10) in FP32; truncation after x^14/15!
// is below 1e-19.
__device__ __forceinline__ dfl df_sinc_small(dfl x) {
  const dfl x2 = x * x;
  const float y = x2.hi;
  float t = -7.64716373181981648e-13f;          // -1/15!
  t = fmaf(t, y, 1.60590438368216146e-10f);     //  1/13!
  t = fmaf(t, y, -2.50521083854417188e-08f);    // -1/11!
  t = fmaf(t, y, 2.75573192239858907e-06f);     //  1/9!
  constexpr dfl i7 = df_const(-1.0 / 5040.0), i5 = df_const(1.0 / 120.0),
                i3 = df_const(-1.0 / 6.0);
  dfl p = df_f(t * y) + i7;
  p = p * x2 + i5;
  p = p * x2 + i3;
  return p * x2 + df_f(1.0f);
}

}  // namespace scs
