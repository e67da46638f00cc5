// Double-float arithmetic: a value is an unevaluated sum hi + lo of two
// float32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.  On this
// GPU the float32 pipe issues 64 times the float64 rate, so the bulk of the
// low-rank recompression (Householder QR and applying Q) runs in double-float.
// Products use the FMA-based exact product (TwoProduct); sums use Knuth's
// TwoSum; dot products follow Ogita, Rump and Oishi, "Accurate sum and dot
// product" (SIAM J. Sci. Comput. 26, 2005), algorithm Dot2, with the error
// terms accumulated separately.
#pragma once
#include <cuda_runtime.h>

typedef float2 dfloat;  // x = hi, y = lo

__device__ __forceinline__ dfloat df_from(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ double df_to(dfloat a) { return (double)a.x + (double)a.y; }

// b - d * a
__device__ __forceinline__ dfloat df_sub_prod(dfloat b, dfloat d, dfloat a) {
  const float p = d.x * a.x;
  float pe = fmaf(d.x, a.x, -p);
  pe = fmaf(d.x, a.y, pe);
  pe = fmaf(d.y, a.x, pe);
  const float s = b.x - p;
  const float z = s - b.x;
  float e = (b.x - (s - z)) - (p + z);
  e += b.y - pe;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// a * d
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat d) {
  const float p = a.x * d.x;
  float pe = fmaf(a.x, d.x, -p);
  pe = fmaf(a.x, d.y, pe);
  pe = fmaf(a.y, d.x, pe);
  const float hi = p + pe;
  return make_float2(hi, pe - (hi - p));
}

// Dot2 accumulation step: (s, c) += a * b
__device__ __forceinline__ void df_dot_add(float& s, float& c, dfloat a, dfloat b) {
  const float p = a.x * b.x;
  float pe = fmaf(a.x, b.x, -p);
  pe = fmaf(a.x, b.y, pe);
  pe = fmaf(a.y, b.x, pe);
  const float t = s + p;
  const float z = t - s;
  const float e = (s - (t - z)) + (p - z);
  s = t;
  c += e + pe;
}

// --- conversions by bit manipulation (integer pipe; no float64 instruction) ---
// 2^e as a float, -126 <= e <= 127
__device__ __forceinline__ float df_pow2f(int e) { return __int_as_float((e + 127) << 23); }

// v * 2^sh as double-float: hi = v's significand truncated to 24 bits, lo = the
// remaining 29 bits rounded to 24.  Magnitudes below 2^-126 after scaling are
// flushed to zero (negligible next to the O(1) column maxima they sit in);
// non-finite or overflowing inputs give NaN, which the callers detect.
__device__ __forceinline__ dfloat df_from_scaled(double v, int sh) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7ff);
  if (ex == 0) return make_float2(0.f, 0.f);
  const int e = ex - 1023 + sh;
  if (ex == 0x7ff || e > 127) return make_float2(__int_as_float(0x7fc00000), 0.f);
  if (e < -126) return make_float2(0.f, 0.f);
  const unsigned int sign = (unsigned int)(b >> 63) << 31;
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const float hi = __int_as_float(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)(mant >> 29));
  const unsigned int rem = (unsigned int)(mant & 0x1FFFFFFFu);
  float lo = ((float)rem * 2.220446049250313e-16f) * df_pow2f(e);  // rem * 2^-52 * 2^e
  return make_float2(hi, sign ? -lo : lo);
}

__device__ __forceinline__ double df_f2d(float f, int sh) {  // exact float -> double with a power-of-two scale
  const unsigned int b = (unsigned int)__float_as_int(f);
  const int ex = (int)((b >> 23) & 0xff);
  if (ex == 0 || ex == 0xff) return ex == 0 ? 0.0 : __longlong_as_double(0x7ff8000000000000ll);
  const unsigned long long sign = (unsigned long long)(b >> 31) << 63;
  const unsigned long long e = (unsigned long long)(ex - 127 + sh + 1023);
  return __longlong_as_double((long long)(sign | (e << 52) | ((unsigned long long)(b & 0x7fffff) << 29)));
}

// double-float * 2^sh to double (one float64 addition)
__device__ __forceinline__ double df_to_scaled(dfloat a, int sh) { return df_f2d(a.x, sh) + df_f2d(a.y, sh); }

// a + b
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
  const float s = a.x + b.x;
  const float z = s - a.x;
  float e = (a.x - (s - z)) + (b.x - z);
  e += a.y + b.y;
  const float hi = s + e;
  return make_float2(hi, e - (hi - s));
}

// Dot2 accumulator (s, c) as a normalised double-float
__device__ __forceinline__ dfloat df_norm(float s, float c) {
  const float hi = s + c;
  return make_float2(hi, c - (hi - s));
}

__device__ __forceinline__ dfloat df_warp_sum(dfloat v) {
  for (int o = 16; o > 0; o >>= 1) {
    dfloat w;
    w.x = __shfl_xor_sync(0xffffffffu, v.x, o);
    w.y = __shfl_xor_sync(0xffffffffu, v.y, o);
    v = df_add(v, w);
  }
  return v;
}
