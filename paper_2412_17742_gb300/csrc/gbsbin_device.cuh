// Device helpers shared by the point kernels: complex arithmetic, roots of unity, grid
// digits, warp reductions, the exact-branch log det of a chunk of pivots and the Dot2
// error-free accumulator.
#pragma once

#include <cuda_runtime.h>

#include "gbsbin_internal.h"

namespace gbsbin {

// ------------------------------------------------------------------ complex helpers
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cfnma(double2 a, double2 b, double2 c) {  // a - b c
  return make_double2(fma(-b.x, c.x, fma(b.y, c.y, a.x)), fma(-b.x, c.y, fma(-b.y, c.x, a.y)));
}
__device__ __forceinline__ double2 crecip(double2 a) {
  double s = 1.0 / fma(a.x, a.x, a.y * a.y);
  return make_double2(a.x * s, -a.y * s);
}
__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfnmaf(float2 a, float2 b, float2 c) {
  return make_float2(fmaf(-b.x, c.x, fmaf(b.y, c.y, a.x)), fmaf(-b.x, c.y, fmaf(-b.y, c.x, a.y)));
}
__device__ __forceinline__ float2 crecipf(float2 a) {
  float s = __frcp_rn(fmaf(a.x, a.x, a.y * a.y));   // correctly rounded, as 1.0f / x
  return make_float2(a.x * s, -a.y * s);
}

// Half-grid index of a plan's evaluated point e: a shard evaluates point 0 first, then its
// slice [e_lo, e_hi).
__device__ __forceinline__ long long global_point(long long e, const GridDesc& g) {
  return g.e_lo > 0 ? (e == 0 ? 0 : e - 1 + g.e_lo) : e;
}

// Digit l of evaluated point e: last axis in [0, half), the others full radix.  32-bit
// arithmetic (grids hold at most GBSBIN_MAX_POINTS = 2^26 points): 64-bit division would
// expand to a long instruction sequence.
__device__ __forceinline__ int point_digit(long long e64, const GridDesc& g, int l) {
  const int e = (int)global_point(e64, g);
  const int last = e % g.half;
  if (l == g.L - 1) return last;
  int rest = e / g.half;
  for (int m = g.L - 2; m > l; --m) rest /= g.radix[m];
  return rest % g.radix[l];
}

// w_l = exp(2 pi i k / R_l) for digit k of axis l, from the plan's twiddle table tw (the
// exact-index values exp(-2 pi i m / R_l), m < R_l, axis after axis): a load instead of an
// FP64 sincospi per point.
__device__ __forceinline__ double2 grid_root(const double2* tw, const GridDesc& g, int l, int k) {
  int off = 0;
  for (int m = 0; m < l; ++m) off += g.radix[m];
  const double2 t = tw[off + k];
  return make_double2(t.x, -t.y);
}

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_min_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum over i of Log(d_i u'_ii) for one point, by one warp.  diag(i) returns u'_ii as
// double2.  Returns (ld, min_i Re(d_i u'_ii)) in lane 0 (all lanes hold the sums).
template <typename DiagFn>
__device__ __forceinline__ void warp_logdet(int n, const double2* w, const int* lab, DiagFn diag, double2* ld,
                                            double* minre) {
  const int lane = threadIdx.x & 31;
  const int chunk = (n + 31) >> 5;
  const int i0 = lane * chunk, i1 = min(n, i0 + chunk);
  double2 p = make_double2(1.0, 0.0);
  int e2 = 0;
  float argsum = 0.0f;
  double mn = 1.0e300;
  for (int i = i0; i < i1; ++i) {
    double2 z = cmul(w[lab[i]], diag(i));
    mn = fmin(mn, z.x);
    if (!(z.x == z.x) || !(z.y == z.y)) mn = -1.0e300;
    argsum += atan2f((float)z.y, (float)z.x);
    p = cmul(p, z);
    int ex;
    double m = fmax(fabs(p.x), fabs(p.y));
    if (m > 0.0 && m < 1.0e300) {
      frexp(m, &ex);
      p.x = ldexp(p.x, -ex);
      p.y = ldexp(p.y, -ex);
      e2 += ex;
    }
  }
  const double LN2 = 0.693147180559945309417232121458;
  const double TWO_PI = 6.283185307179586476925286766559;
  double re = 0.0, im = 0.0;
  if (i1 > i0) {
    double a = atan2(p.y, p.x);
    double wind = rint(((double)argsum - a) / TWO_PI);
    re = 0.5 * log(fma(p.x, p.x, p.y * p.y)) + (double)e2 * LN2;
    im = a + TWO_PI * wind;
  }
  re = warp_sum_d(re);
  im = warp_sum_d(im);
  mn = warp_min_d(mn);
  *ld = make_double2(re, im);
  *minre = mn;
}

// ---------------------------------------------------- error-free FP32 transformations
// Dot2 accumulator: s is the rounded running sum, c collects the exact rounding errors.
struct Acc2 {
  float s, c;
};
__device__ __forceinline__ void acc2_add_prod(Acc2& a, float x, float y) {
  float p = x * y;
  float pe = fmaf(x, y, -p);          // x*y = p + pe exactly
  float t = a.s + p;                  // TwoSum(a.s, p) (Knuth)
  float bb = t - a.s;
  float te = (a.s - (t - bb)) + (p - bb);
  a.s = t;
  a.c += te + pe;
}
__device__ __forceinline__ void acc2_add(Acc2& a, float v) {
  float t = a.s + v;
  float bb = t - a.s;
  float te = (a.s - (t - bb)) + (v - bb);
  a.s = t;
  a.c += te;
}
__device__ __forceinline__ float acc2_value(const Acc2& a) { return a.s + a.c; }

// ------------------------------------------------- fixed-point digits of the FP32 factors
// 2^s as FP32 for -126 <= s <= 127.
__device__ __forceinline__ float pow2f(int s) { return __int_as_float((127 + s) << 23); }

// Smallest e with m < 2^e for finite m > 0 (-126 for m = 0 or subnormal, 129 for inf/NaN).
__device__ __forceinline__ int exponent_bound(float m) { return ((__float_as_int(m) >> 23) & 0xff) - 126; }

// int64 -> FP32, rounded to nearest: the 32-bit conversion (a full-rate instruction) when
// the value fits, the 64-bit one (on the FP64 pipe) otherwise.
__device__ __forceinline__ float ll2f(long long v) {
  const int lo = (int)v;
  return (long long)lo == v ? __int2float_rn(lo) : __ll2float_rn(v);
}

// conj(d) on the diagonal of M in the fixed-point scale 2^GBSBIN_FIX_BITS of -XA.
__device__ __forceinline__ longlong2 conj_fix(double2 d) {
  const double s = 4611686018427387904.0;   // 2^62
  return make_longlong2(__double2ll_rn(d.x * s), -__double2ll_rn(d.y * s));
}

}  // namespace gbsbin
