// Complex numbers as pairs of FP32 (hi + lo, about 46 significant bits) for the FMA pipe,
// which on this GPU issues ~70x more operations per second than the FP64 pipe: a complex
// value is a float4 (hi re, hi im, lo re, lo im).  Built from Dekker's and Knuth's
// error-free transformations (TwoProduct by FMA, TwoSum, FastTwoSum); the reciprocal by one
// Newton step on an FP32 seed.
#pragma once

#include <cuda_runtime.h>

namespace gbsbin {

// The intrinsics keep the compiler from contracting or reassociating these sequences.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {   // Knuth: a + b = s + e
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // Dekker, |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ float4 df_from(double2 v) {
  const float hr = __double2float_rn(v.x), hi = __double2float_rn(v.y);
  return make_float4(hr, hi, __double2float_rn(v.x - (double)hr), __double2float_rn(v.y - (double)hi));
}
__device__ __forceinline__ double2 df_to(float4 v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}
// a b of normalised pairs: the hi x hi products exactly (TwoProduct by FMA), the cross
// terms in FP32, one renormalisation per component
__device__ __forceinline__ float4 df_mul(float4 a, float4 b) {
  const float p1 = __fmul_rn(a.x, b.x), e1 = fmaf(a.x, b.x, -p1);
  const float p2 = __fmul_rn(a.y, b.y), e2 = fmaf(a.y, b.y, -p2);
  float sr, er;
  two_sum(p1, -p2, sr, er);
  er = __fadd_rn(er, __fsub_rn(e1, e2));
  er = fmaf(a.x, b.z, er);
  er = fmaf(a.z, b.x, er);
  er = fmaf(-a.y, b.w, er);
  er = fmaf(-a.w, b.y, er);
  const float p3 = __fmul_rn(a.x, b.y), e3 = fmaf(a.x, b.y, -p3);
  const float p4 = __fmul_rn(a.y, b.x), e4 = fmaf(a.y, b.x, -p4);
  float si, ei;
  two_sum(p3, p4, si, ei);
  ei = __fadd_rn(ei, __fadd_rn(e3, e4));
  ei = fmaf(a.x, b.w, ei);
  ei = fmaf(a.z, b.y, ei);
  ei = fmaf(a.y, b.z, ei);
  ei = fmaf(a.w, b.x, ei);
  float4 r;
  fast_two_sum(sr, er, r.x, r.z);
  fast_two_sum(si, ei, r.y, r.w);
  return r;
}
__device__ __forceinline__ float4 df_add(float4 a, float4 b) {
  float sr, er, si, ei;
  two_sum(a.x, b.x, sr, er);
  two_sum(a.y, b.y, si, ei);
  er = __fadd_rn(er, __fadd_rn(a.z, b.z));
  ei = __fadd_rn(ei, __fadd_rn(a.w, b.w));
  float4 r;
  fast_two_sum(sr, er, r.x, r.z);
  fast_two_sum(si, ei, r.y, r.w);
  return r;
}
__device__ __forceinline__ float4 df_conj(float4 a) { return make_float4(a.x, -a.y, a.z, -a.w); }
__device__ __forceinline__ float4 df_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }
// c + a b
__device__ __forceinline__ float4 df_fma(float4 a, float4 b, float4 c) { return df_add(c, df_mul(a, b)); }
// c - a b, fused: per component the two hi x hi products exactly (TwoProduct by FMA), each
// subtracted from c's hi part by a TwoSum, the rounding errors, c's lo part and the cross
// terms gathered in FP32, one renormalisation (the product is never renormalised on its own)
__device__ __forceinline__ float4 df_fms(float4 c, float4 a, float4 b) {
  // real: c - (a.re b.re - a.im b.im)
  const float p1 = __fmul_rn(a.x, b.x), e1 = fmaf(a.x, b.x, -p1);
  const float p2 = __fmul_rn(a.y, b.y), e2 = fmaf(a.y, b.y, -p2);
  float s, t1, s2, t2;
  two_sum(c.x, -p1, s, t1);
  two_sum(s, p2, s2, t2);
  float er = __fadd_rn(__fadd_rn(t1, t2), c.z);
  er = __fadd_rn(__fsub_rn(er, e1), e2);
  er = fmaf(-a.x, b.z, er);
  er = fmaf(-a.z, b.x, er);
  er = fmaf(a.y, b.w, er);
  er = fmaf(a.w, b.y, er);
  // imaginary: c - (a.re b.im + a.im b.re)
  const float p3 = __fmul_rn(a.x, b.y), e3 = fmaf(a.x, b.y, -p3);
  const float p4 = __fmul_rn(a.y, b.x), e4 = fmaf(a.y, b.x, -p4);
  float u, t3, u2, t4;
  two_sum(c.y, -p3, u, t3);
  two_sum(u, -p4, u2, t4);
  float ei = __fadd_rn(__fadd_rn(t3, t4), c.w);
  ei = __fsub_rn(__fsub_rn(ei, e3), e4);
  ei = fmaf(-a.x, b.w, ei);
  ei = fmaf(-a.w, b.x, ei);
  ei = fmaf(-a.y, b.z, ei);
  ei = fmaf(-a.z, b.y, ei);
  float4 r;
  fast_two_sum(s2, er, r.x, r.z);
  fast_two_sum(u2, ei, r.y, r.w);
  return r;
}

// 1 / a for a nonzero pair a: d = |a|^2 as a real pair, s = 1/d from the FP32 seed s0 =
// 1/hi(d) by one Newton step s = s0 + s0 (1 - d s0) (the residual 1 - d s0 formed with an
// FMA, so the step doubles the seed's ~24 bits), then conj(a) s.
__device__ __forceinline__ float4 df_recip(float4 a) {
  // d = a.re^2 + a.im^2 (hi parts exactly by FMA, cross terms in FP32)
  const float p1 = __fmul_rn(a.x, a.x), e1 = fmaf(a.x, a.x, -p1);
  const float p2 = __fmul_rn(a.y, a.y), e2 = fmaf(a.y, a.y, -p2);
  float dh, dl;
  two_sum(p1, p2, dh, dl);
  dl = __fadd_rn(dl, __fadd_rn(e1, e2));
  dl = fmaf(2.0f * a.x, a.z, dl);
  dl = fmaf(2.0f * a.y, a.w, dl);
  float t;
  fast_two_sum(dh, dl, dh, t);
  dl = t;
  const float s0 = __frcp_rn(dh);
  const float r = __fsub_rn(fmaf(-dh, s0, 1.0f), __fmul_rn(dl, s0));   // 1 - d s0
  float sh, sl;
  fast_two_sum(s0, __fmul_rn(s0, r), sh, sl);
  return df_mul(df_conj(a), make_float4(sh, 0.f, sl, 0.f));
}

// Real pairs (hi, lo) in the x and z components of a float4 (y = w = 0).
// 1 / a by one Newton step on the FP32 seed (as in df_recip).
__device__ __forceinline__ float4 df_rrecip(float4 a) {
  const float s0 = __frcp_rn(a.x);
  const float r = __fsub_rn(fmaf(-a.x, s0, 1.0f), __fmul_rn(a.z, s0));   // 1 - a s0
  float sh, sl;
  fast_two_sum(s0, __fmul_rn(s0, r), sh, sl);
  return make_float4(sh, 0.f, sl, 0.f);
}
// sqrt(a), a >= 0, by one Newton (Heron) step on the FP32 seed t = sqrt(hi):
// sqrt(a) = t + (a - t^2) / (2 t), the residual a - t^2 formed with an FMA.
__device__ __forceinline__ float4 df_rsqrt_root(float4 a) {
  if (!(a.x > 0.f)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float t = __fsqrt_rn(a.x);
  const float res = __fadd_rn(fmaf(-t, t, a.x), a.z);                      // a - t^2
  const float corr = __fdiv_rn(res, __fmul_rn(2.0f, t));
  float h, l;
  fast_two_sum(t, corr, h, l);
  return make_float4(h, 0.f, l, 0.f);
}
// Principal square root of a complex pair z = x + i y: r = |z|, s = sqrt((r + |x|) / 2),
// then (s, y / (2 s)) for x >= 0 and (|y| / (2 s), sign(y) s) otherwise.
__device__ __forceinline__ float4 df_csqrt(float4 z) {
  const float4 x = make_float4(z.x, 0.f, z.z, 0.f), y = make_float4(z.y, 0.f, z.w, 0.f);
  const float4 r = df_rsqrt_root(df_add(df_mul(x, x), df_mul(y, y)));
  const bool neg = z.x < 0.f;
  const float4 ax = neg ? df_neg(x) : x;
  const float4 half = make_float4(0.5f, 0.f, 0.f, 0.f);
  const float4 s = df_rsqrt_root(df_mul(df_add(r, ax), half));
  if (!(s.x > 0.f)) return make_float4(0.f, 0.f, 0.f, 0.f);
  const float4 q = df_mul(y, df_rrecip(df_mul(s, make_float4(2.f, 0.f, 0.f, 0.f))));   // y / (2 s)
  if (!neg) return make_float4(s.x, q.x, s.z, q.z);
  const float sg = z.y < 0.f ? -1.f : 1.f;
  return make_float4(fabsf(q.x), sg * s.x, q.x < 0.f ? -q.z : q.z, sg * s.z);
}

// Full-warp shuffles of 16-byte elements (pairs of FP32 or FP64 complex values).
__device__ __forceinline__ float4 shfl(float4 v, int src) {
  return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                     __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
__device__ __forceinline__ double2 shfl(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float4 shfl_xor(float4 v, int mask) {
  return make_float4(__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask),
                     __shfl_xor_sync(0xffffffffu, v.z, mask), __shfl_xor_sync(0xffffffffu, v.w, mask));
}
__device__ __forceinline__ double2 shfl_xor(double2 v, int mask) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, mask), __shfl_xor_sync(0xffffffffu, v.y, mask));
}

// ----------------------------------------------------- the tree's two arithmetics
// Element type E (16 bytes either way), the operations the tree kernels use, and a complex
// scaling by a power of two that returns the exponent taken out.
struct ArDF {                                        // pairs of FP32 on the FMA pipe
  using E = float4;
  static __device__ __forceinline__ E from(double2 v) { return df_from(v); }
  static __device__ __forceinline__ double2 to(E v) { return df_to(v); }
  static __device__ __forceinline__ E one() { return make_float4(1.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ E zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ E mul(E a, E b) { return df_mul(a, b); }
  static __device__ __forceinline__ E add(E a, E b) { return df_add(a, b); }
  static __device__ __forceinline__ E neg(E a) { return df_neg(a); }
  static __device__ __forceinline__ E fma(E a, E b, E c) { return df_fma(a, b, c); }
  static __device__ __forceinline__ E fms(E c, E a, E b) { return df_fms(c, a, b); }
  static __device__ __forceinline__ E recip(E a) { return df_recip(a); }
  static __device__ __forceinline__ E csqrt(E a) { return df_csqrt(a); }
  static __device__ __forceinline__ E conj(E a) { return df_conj(a); }
  // |a|^2 as a real pair; sqrt and reciprocal of a real pair (imaginary parts zero)
  static __device__ __forceinline__ E norm2(E a) {
    const float4 x = make_float4(a.x, 0.f, a.z, 0.f), y = make_float4(a.y, 0.f, a.w, 0.f);
    return df_add(df_mul(x, x), df_mul(y, y));
  }
  static __device__ __forceinline__ E rsqrt_real(E a) { return df_rsqrt_root(a); }
  static __device__ __forceinline__ E rrecip(E a) { return df_rrecip(a); }
  static __device__ __forceinline__ float re(E a) { return a.x; }
  static __device__ __forceinline__ float im(E a) { return a.y; }
  // mx = 2^(ex - 1) f, f in [1, 2): ex from the exponent bits, the scaling by 2^-ex an exact
  // multiply (ex in [-99, 100] here); subnormal magnitudes take frexpf/ldexpf
  static __device__ __forceinline__ int normalise(E& a) {
    const float mx = fmaxf(fabsf(a.x), fabsf(a.y));
    if (!(mx > 0.f && mx < 1.0e30f)) return 0;
    if (mx < 1.0e-30f) {
      int ex;
      frexpf(mx, &ex);
      a = make_float4(ldexpf(a.x, -ex), ldexpf(a.y, -ex), ldexpf(a.z, -ex), ldexpf(a.w, -ex));
      return ex;
    }
    const int ex = (int)((__float_as_uint(mx) >> 23) & 0xffu) - 126;
    const float sc = __uint_as_float((unsigned)(127 - ex) << 23);
    a = make_float4(a.x * sc, a.y * sc, a.z * sc, a.w * sc);
    return ex;
  }
};

struct ArF64 {                                       // FP64 throughout
  using E = double2;
  static __device__ __forceinline__ E from(double2 v) { return v; }
  static __device__ __forceinline__ double2 to(E v) { return v; }
  static __device__ __forceinline__ E one() { return make_double2(1.0, 0.0); }
  static __device__ __forceinline__ E zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ E mul(E a, E b) {
    return make_double2(::fma(a.x, b.x, -a.y * b.y), ::fma(a.x, b.y, a.y * b.x));
  }
  static __device__ __forceinline__ E add(E a, E b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ E neg(E a) { return make_double2(-a.x, -a.y); }
  static __device__ __forceinline__ E fma(E a, E b, E c) {   // c + a b
    return make_double2(::fma(a.x, b.x, ::fma(-a.y, b.y, c.x)), ::fma(a.x, b.y, ::fma(a.y, b.x, c.y)));
  }
  static __device__ __forceinline__ E fms(E c, E a, E b) {   // c - a b
    return make_double2(::fma(-a.x, b.x, ::fma(a.y, b.y, c.x)), ::fma(-a.x, b.y, ::fma(-a.y, b.x, c.y)));
  }
  // 1 / a = conj(a) / |a|^2, the real reciprocal by two Newton steps s <- s (2 - d s) on the
  // FP32 seed (each doubles the ~24 correct bits): FP64 division is a long sequence on
  // this GPU's FP64 pipe
  static __device__ __forceinline__ E recip(E a) {
    const double d = ::fma(a.x, a.x, a.y * a.y);
    double s = (double)__frcp_rn((float)d);
    s = ::fma(s, ::fma(-d, s, 1.0), s);
    s = ::fma(s, ::fma(-d, s, 1.0), s);
    return make_double2(a.x * s, -a.y * s);
  }
  // principal square root: r = |a|, t = sqrt((r + |x|) / 2), (t, y / (2 t)) for x >= 0,
  // (|y| / (2 t), sign(y) t) otherwise
  static __device__ __forceinline__ E csqrt(E a) {
    const double r = ::sqrt(::fma(a.x, a.x, a.y * a.y));
    const double t = ::sqrt(0.5 * (r + ::fabs(a.x)));
    if (!(t > 0.0)) return make_double2(0.0, 0.0);
    const double q = a.y / (2.0 * t);
    if (a.x >= 0.0) return make_double2(t, q);
    return make_double2(::fabs(q), a.y < 0.0 ? -t : t);
  }
  static __device__ __forceinline__ E conj(E a) { return make_double2(a.x, -a.y); }
  static __device__ __forceinline__ E norm2(E a) { return make_double2(::fma(a.x, a.x, a.y * a.y), 0.0); }
  static __device__ __forceinline__ E rsqrt_real(E a) { return make_double2(a.x > 0.0 ? ::sqrt(a.x) : 0.0, 0.0); }
  static __device__ __forceinline__ E rrecip(E a) { return make_double2(1.0 / a.x, 0.0); }
  static __device__ __forceinline__ float re(E a) { return (float)a.x; }
  static __device__ __forceinline__ float im(E a) { return (float)a.y; }
  // as ArDF::normalise, from the FP64 exponent bits (ex in [-996, 997] here)
  static __device__ __forceinline__ int normalise(E& a) {
    const double mx = ::fmax(::fabs(a.x), ::fabs(a.y));
    if (!(mx > 0.0 && mx < 1.0e300)) return 0;
    if (mx < 1.0e-300) {
      int ex;
      ::frexp(mx, &ex);
      a = make_double2(::ldexp(a.x, -ex), ::ldexp(a.y, -ex));
      return ex;
    }
    const int ex = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1022;
    const double sc = __longlong_as_double((long long)(1023 - ex) << 52);
    a = make_double2(a.x * sc, a.y * sc);
    return ex;
  }
};

}  // namespace gbsbin
