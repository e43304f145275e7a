// Double-float arithmetic shared by the transform and wall-normal kernels.
#pragma once
#include <cuda_runtime.h>

// Double-float real: value = h + l with |l| <= ulp(h)/2 (Dekker 1971).  The
// error-free sum is Knuth's two-sum, the product uses the FMA to recover the
// low part of h_a h_b; every operation is an explicit round-to-nearest
// intrinsic so that the compiler neither contracts nor reassociates it.
// Relative precision about 2^-47 at FP32 throughput.
struct dfr {
  float h, l;
};
struct dfc {
  dfr x, y;
};
__device__ __forceinline__ dfr operator+(dfr a, dfr b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  const float t = __fadd_rn(s, e);
  return dfr{t, __fsub_rn(e, __fsub_rn(t, s))};
}
__device__ __forceinline__ dfr operator-(dfr a) { return dfr{-a.h, -a.l}; }
__device__ __forceinline__ dfr operator-(dfr a, dfr b) { return a + (-b); }
__device__ __forceinline__ dfr operator*(dfr a, dfr b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const float t = __fadd_rn(p, e);
  return dfr{t, __fsub_rn(e, __fsub_rn(t, p))};
}

// Sum left unnormalised: Knuth's two-sum of the high parts (exact) plus both low parts,
// without the final fast two-sum.  For sums that feed another addition or product
// straight away; the value is the one a + b represents before its renormalisation.
__device__ __forceinline__ dfr add_u(dfr a, dfr b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fsub_rn(s, a.h);
  float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  return dfr{s, e};
}

// Product left unnormalised, (p, e) with p = fl(a.h b.h) and e its FMA residual plus the
// cross terms: the same value as a * b without the final fast two-sum, for products that
// feed an addition straight away (the addition's two-sum takes the whole low part).
__device__ __forceinline__ dfr mul_u(dfr a, dfr b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dfr{p, e};
}

// Split a double into the nearest float and the float nearest to the rest
// (one FP64 subtraction; the conversions do not use the FP64 pipe).
__device__ __forceinline__ dfr df_split(double x) {
  const float h = __double2float_rn(x);
  return dfr{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_merge(dfr a) { return (double)a.h + (double)a.l; }

// Stored Fourier values.  In the double-float mode a complex field holds, in the
// 16 bytes of each complex double, the pairs (re.h, re.l, im.h, im.l) as floats.
// These read a stored value back as FP64 (pair: the exact sum of its floats,
// rounded once).
__device__ __forceinline__ double2 load_c(const double2* p, size_t o, int pair) {
  if (!pair) return p[o];
  const float4 q = reinterpret_cast<const float4*>(p)[o];
  return make_double2((double)q.x + (double)q.y, (double)q.z + (double)q.w);
}
__device__ __forceinline__ double load_re(const double2* p, size_t o, int pair) {
  if (!pair) return p[o].x;
  const float2 q = reinterpret_cast<const float2*>(p)[2 * o];
  return (double)q.x + (double)q.y;
}

// FP32 <-> FP64 conversions on the integer pipe (the hardware conversions issue on the
// FP64 pipe, the bottleneck of the mixed mode's sweeps).  f2d_int is exact for zero,
// normal floats, infinities and NaNs, and flushes float subnormals to zero.  d2f_int
// rounds the 52-bit mantissa to 23 bits, ties away from zero, for |x| in the float
// normal range; smaller magnitudes flush to zero, larger ones (and NaN) give infinity.
__device__ __forceinline__ double f2d_int(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u, ex = (u >> 23) & 0xffu, mant = u & 0x7fffffu;
  unsigned hi = sign, lo = 0u;
  if (ex != 0u) {
    const unsigned e = ex == 255u ? 2047u : ex + 896u;
    hi = sign | (e << 20) | (mant >> 3);
    lo = mant << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32);
  const int ex = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  const unsigned m = (unsigned)((b >> 29) & 0x7fffffu), rb = (unsigned)(b >> 28) & 1u;
  unsigned r = ((unsigned)ex << 23) + m + rb;   // a carry out of the mantissa bumps the exponent
  r = ex <= 0 ? 0u : (ex >= 255 ? 0x7f800000u : r);
  return __uint_as_float((hi & 0x80000000u) | r);
}
