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
