// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// FP32 numbers with |lo| <= ulp(hi) / 2 (Dekker 1971), about 48 significant
// bits; the error-free transformations TwoSum (Knuth) and TwoProduct (with
// FMA) give additions and products whose rounding error is about 2^-47 of
// the operands' magnitude.  On GB300 FP32 runs at 64 times the FP64 rate,
// where an FP64 warp instruction holds an SMSP's FP64 pipe for 64 cycles, so
// FP64-class accuracy costs far less in FP32 pairs than in FP64.  Operands
// must lie within FP32's exponent range; callers scale by powers of two.
#pragma once
#include <cuda_runtime.h>

namespace scs {

struct __align__(8) dfl {
  float hi, lo;
};

__device__ __forceinline__ dfl df_make(float h, float l) {
  dfl r;
  r.hi = h;
  r.lo = l;
  return r;
}
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return df_make(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  const dfl s = df_two_sum(x.hi, y.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ dfl df_neg(dfl x) { return df_make(-x.hi, -x.lo); }
// x y + z
__device__ __forceinline__ dfl df_fma(dfl x, dfl y, dfl z) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
  const dfl s = df_two_sum(p, z.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, z.lo)));
}
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfl df_zero() { return df_make(0.0f, 0.0f); }
// x + y u + z w with one renormalisation (TwoProduct of each hi part, TwoSum
// of the three leading terms, the error terms summed in FP32).
__device__ __forceinline__ dfl df_add2prod(dfl x, dfl y, dfl u, dfl z, dfl w) {
  const float p1 = __fmul_rn(y.hi, u.hi);
  float e1 = __fmaf_rn(y.hi, u.hi, -p1);
  e1 = __fmaf_rn(y.hi, u.lo, __fmaf_rn(y.lo, u.hi, e1));
  const float p2 = __fmul_rn(z.hi, w.hi);
  float e2 = __fmaf_rn(z.hi, w.hi, -p2);
  e2 = __fmaf_rn(z.hi, w.lo, __fmaf_rn(z.lo, w.hi, e2));
  const dfl s1 = df_two_sum(x.hi, p1);
  const dfl s2 = df_two_sum(s1.hi, p2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(x.lo, e1), __fadd_rn(e2, s1.lo)), s2.lo);
  return df_fast_two_sum(s2.hi, lo);
}
// x + y1 u1 + y2 u2 + y3 u3 + y4 u4 with one renormalisation (the real or
// imaginary part of a complex update a + v w + p q).
__device__ __forceinline__ dfl df_add4prod(dfl x, dfl y1, dfl u1, dfl y2, dfl u2, dfl y3, dfl u3, dfl y4, dfl u4) {
  const float p1 = __fmul_rn(y1.hi, u1.hi);
  float e = __fmaf_rn(y1.hi, u1.hi, -p1);
  e = __fmaf_rn(y1.hi, u1.lo, __fmaf_rn(y1.lo, u1.hi, e));
  const float p2 = __fmul_rn(y2.hi, u2.hi);
  e = __fadd_rn(e, __fmaf_rn(y2.hi, u2.hi, -p2));
  e = __fmaf_rn(y2.hi, u2.lo, __fmaf_rn(y2.lo, u2.hi, e));
  const float p3 = __fmul_rn(y3.hi, u3.hi);
  e = __fadd_rn(e, __fmaf_rn(y3.hi, u3.hi, -p3));
  e = __fmaf_rn(y3.hi, u3.lo, __fmaf_rn(y3.lo, u3.hi, e));
  const float p4 = __fmul_rn(y4.hi, u4.hi);
  e = __fadd_rn(e, __fmaf_rn(y4.hi, u4.hi, -p4));
  e = __fmaf_rn(y4.hi, u4.lo, __fmaf_rn(y4.lo, u4.hi, e));
  dfl s = df_two_sum(x.hi, p1);
  float lo = __fadd_rn(x.lo, s.lo);
  s = df_two_sum(s.hi, p2);
  lo = __fadd_rn(lo, s.lo);
  s = df_two_sum(s.hi, p3);
  lo = __fadd_rn(lo, s.lo);
  s = df_two_sum(s.hi, p4);
  lo = __fadd_rn(__fadd_rn(lo, s.lo), e);
  return df_fast_two_sum(s.hi, lo);
}
// Compensated dot product of double-float vectors (the scheme of Ogita, Rump
// and Oishi's Dot2): the products' hi parts are summed with TwoSum into s,
// every error term into the FP32 compensation c; df_dot_value renormalises.
struct df_dot {
  float s, c;
};
__device__ __forceinline__ df_dot df_dot_zero() {
  df_dot d;
  d.s = 0.0f;
  d.c = 0.0f;
  return d;
}
__device__ __forceinline__ df_dot df_dot_add(df_dot d, dfl a, dfl x) {
  const float p = __fmul_rn(a.hi, x.hi);
  float e = __fmaf_rn(a.hi, x.hi, -p);
  e = __fmaf_rn(a.hi, x.lo, __fmaf_rn(a.lo, x.hi, e));
  const dfl t = df_two_sum(d.s, p);
  d.s = t.hi;
  d.c = __fadd_rn(d.c, __fadd_rn(t.lo, e));
  return d;
}
__device__ __forceinline__ dfl df_dot_value(df_dot d) { return df_two_sum(d.s, d.c); }
// FP64 <-> double-float (FP64 pipe: used at the boundaries only)
__device__ __forceinline__ dfl df_from_d(double x) {
  const float h = __double2float_rn(x);
  return df_make(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double df_to_d(dfl x) { return (double)x.hi + (double)x.lo; }
// The same split by integer operations (no FP64-pipe instruction): hi is x
// rounded to FP32 (to nearest, ties to even) from its 53-bit significand,
// lo the remaining 29 bits rounded to FP32.  For operands bounded in
// magnitude: |x| below 2^-126 gives 0, and lo is dropped below 2^-74
// (its weight is under 2^-98 there); |x| beyond FP32's range gives +-inf.
// df_from_d_scaled(x, s) converts x 2^-s the same way (s a whole number, the
// power of two applied to the exponent field).
__device__ __forceinline__ dfl df_from_d_scaled(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const int eraw = (int)((b >> 52) & 0x7FF);
  if (eraw == 0) return df_zero();
  const int e = eraw == 0x7FF ? eraw : eraw - s;
  if (e < 1023 - 126) return df_zero();
  if (e > 1023 + 127) return df_make(__int_as_float(sgn | 0x7F800000u | (e == 0x7FF && (b << 12) ? 0x400000u : 0u)), 0.0f);
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  unsigned mh = (unsigned)(m >> 29);     // top 24 bits, in [2^23, 2^24)
  int rem = (int)(m & 0x1FFFFFFFull);   // the 29 bits below them
  if (rem > 0x10000000 || (rem == 0x10000000 && (mh & 1u))) {
    ++mh;
    rem -= 0x20000000;
  }
  int fe = e - 1023 + 127;
  if (mh == 0x1000000u) {
    mh = 0x800000u;
    ++fe;
  }
  if (fe > 254) return df_make(__int_as_float(sgn | 0x7F800000u), 0.0f);
  const float hi = __int_as_float(sgn | ((unsigned)fe << 23) | (mh & 0x7FFFFFu));
  float lo = 0.0f;
  const int le = e - 1075 + 127;  // biased exponent of the weight of rem's unit
  if (rem != 0 && le >= 1) {
    lo = __fmul_rn(__int2float_rn(rem), __int_as_float((unsigned)le << 23));
    if (sgn) lo = -lo;
  }
  return df_make(hi, lo);
}
__device__ __forceinline__ dfl df_from_d_int(double x) { return df_from_d_scaled(x, 0); }
__device__ __forceinline__ dfl df_shfl_xor(dfl v, int o) {
  return df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// Square root and quotient in double-float: a correctly rounded FP32
// estimate and one Newton correction from the exact residual (about 2^-46
// relative); the correction, about 2^-24 of the estimate, takes an
// approximate FP32 quotient.
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (a.hi <= 0.0f) return df_zero();
  const float y = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(y, y);
  const float pe = __fmaf_rn(y, y, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), pe), a.lo);
  // the correction is about 2^-24 of y: an approximate quotient (2 ulp) suffices
  return df_fast_two_sum(y, __fdividef(r, __fmul_rn(2.0f, y)));
}
__device__ __forceinline__ dfl df_div(dfl x, dfl y) {
  const float q1 = __fdiv_rn(x.hi, y.hi);
  const dfl r = df_fma(df_make(-q1, 0.0f), y, x);
  return df_fast_two_sum(q1, __fdividef(r.hi, y.hi));
}


// Kernels written once for FP64 and double-float elements (the generic
// arithmetic below): FP64 where the operands span FP64's range, double-float
// where they are bounded in magnitude (eigenvector blocks, reflectors of a
// scaled matrix), where every product is FP32 pipe work and only the
// conversions at the boundary use the FP64 pipe.
__device__ __forceinline__ void g_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void g_zero(dfl& a) { a = df_zero(); }
__device__ __forceinline__ void g_cvt(double& d, double v) { d = v; }
__device__ __forceinline__ void g_cvt(dfl& d, double v) { d = df_from_d_int(v); }
__device__ __forceinline__ double g_mad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ dfl g_mad(dfl a, dfl b, dfl c) { return df_fma(a, b, c); }
__device__ __forceinline__ double g_val(double a) { return a; }
__device__ __forceinline__ double g_val(dfl a) { return df_to_d(a); }
__device__ __forceinline__ double g_add(double a, double b) { return a + b; }
__device__ __forceinline__ dfl g_add(dfl a, dfl b) { return df_add(a, b); }
__device__ __forceinline__ double g_neg(double a) { return -a; }
__device__ __forceinline__ dfl g_neg(dfl a) { return df_neg(a); }
__device__ __forceinline__ bool g_is_zero(double a) { return a == 0.0; }
__device__ __forceinline__ bool g_is_zero(dfl a) { return a.hi == 0.0f && a.lo == 0.0f; }
__device__ __forceinline__ double g_shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfl g_shfl_xor(dfl v, int o) { return df_shfl_xor(v, o); }
// read-only (non-coherent) loads
__device__ __forceinline__ double g_ldg(const double* p) { return __ldg(p); }
__device__ __forceinline__ dfl g_ldg(const dfl* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df_make(v.x, v.y);
}

// Complex double-float: re and im parts as double-float values (16 bytes).
struct __align__(16) cdf {
  dfl re, im;
};
__device__ __forceinline__ cdf c_make(dfl r, dfl i) {
  cdf c;
  c.re = r;
  c.im = i;
  return c;
}
__device__ __forceinline__ cdf c_zero() { return c_make(df_zero(), df_zero()); }
__device__ __forceinline__ cdf c_one() { return c_make(df_make(1.0f, 0.0f), df_zero()); }
__device__ __forceinline__ cdf c_conj(cdf a) { return c_make(a.re, df_neg(a.im)); }
__device__ __forceinline__ cdf c_neg(cdf a) { return c_make(df_neg(a.re), df_neg(a.im)); }
__device__ __forceinline__ cdf c_add(cdf a, cdf b) { return c_make(df_add(a.re, b.re), df_add(a.im, b.im)); }
// a b + c
__device__ __forceinline__ cdf c_fma(cdf a, cdf b, cdf c) {
  return c_make(df_fma(a.re, b.re, df_fma(df_neg(a.im), b.im, c.re)), df_fma(a.re, b.im, df_fma(a.im, b.re, c.im)));
}
// conj(a) b + c
__device__ __forceinline__ cdf c_cfma(cdf a, cdf b, cdf c) {
  return c_make(df_fma(a.re, b.re, df_fma(a.im, b.im, c.re)), df_fma(a.re, b.im, df_fma(df_neg(a.im), b.re, c.im)));
}
__device__ __forceinline__ cdf c_mul(cdf a, cdf b) { return c_fma(a, b, c_zero()); }
// a + v w + p q with one renormalisation per part
__device__ __forceinline__ cdf c_add2prod(cdf a, cdf v, cdf w, cdf p, cdf q) {
  return c_make(df_add4prod(a.re, v.re, w.re, df_neg(v.im), w.im, p.re, q.re, df_neg(p.im), q.im),
                df_add4prod(a.im, v.re, w.im, v.im, w.re, p.re, q.im, p.im, q.re));
}
// compensated accumulation of conj(a) x
struct c_dot {
  df_dot re, im;
};
__device__ __forceinline__ c_dot c_dot_zero() {
  c_dot d;
  d.re = df_dot_zero();
  d.im = df_dot_zero();
  return d;
}
__device__ __forceinline__ c_dot c_dot_add(c_dot d, cdf a, cdf x) {
  d.re = df_dot_add(df_dot_add(d.re, a.re, x.re), a.im, x.im);
  d.im = df_dot_add(df_dot_add(d.im, a.re, x.im), df_neg(a.im), x.re);
  return d;
}
__device__ __forceinline__ cdf c_dot_value(c_dot d) { return c_make(df_dot_value(d.re), df_dot_value(d.im)); }
// compensated accumulation of a x (no conjugate)
__device__ __forceinline__ c_dot c_dotn_add(c_dot d, cdf a, cdf x) {
  d.re = df_dot_add(df_dot_add(d.re, a.re, x.re), df_neg(a.im), x.im);
  d.im = df_dot_add(df_dot_add(d.im, a.re, x.im), a.im, x.re);
  return d;
}
__device__ __forceinline__ cdf c_shfl_xor(cdf v, int o) { return c_make(df_shfl_xor(v.re, o), df_shfl_xor(v.im, o)); }
__device__ __forceinline__ cdf c_from_d(double re, double im) { return c_make(df_from_d(re), df_from_d(im)); }

}  // namespace scs
