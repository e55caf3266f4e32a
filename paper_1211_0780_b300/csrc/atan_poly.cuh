// Generated by atan_poly.py (do not edit): atan(r) ~ r P(r^2) on [0, 1],
// P of degree 8 in r^2, minimax under the weight r (Lawson's iteration,
// FP64); approximation error 5.76e-09 before rounding the coefficients to FP32.
#pragma once
#include <cmath>

namespace xy {

// P(s) by Horner's rule with fused multiply-adds.
__host__ __device__ __forceinline__ float atan_poly(float s) {
  float p = 0x1.4201f40000000p-9f;  // s^8: 0.00245672325
  p = fmaf(p, s, -0x1.d7e7520000000p-7f);  // s^7: -0.0144013548
  p = fmaf(p, s, 0x1.45e3460000000p-5f);  // s^6: 0.039781224
  p = fmaf(p, s, -0x1.2856fc0000000p-4f);  // s^5: -0.0723485798
  p = fmaf(p, s, 0x1.ae09700000000p-4f);  // s^4: 0.104989469
  p = fmaf(p, s, -0x1.2205a00000000p-3f);  // s^3: -0.141612291
  p = fmaf(p, s, 0x1.994fb60000000p-3f);  // s^2: 0.199859068
  p = fmaf(p, s, -0x1.5553680000000p-2f);  // s^1: -0.333325982
  p = fmaf(p, s, 0x1.fffffc0000000p-1f);  // s^0: 0.999999881
  return p;
}

#ifdef __CUDACC__
// P of two values at once (__ffma2_rn: each lane rounds as fmaf does).
__device__ __forceinline__ float2 atan_poly2(float2 s) {
  float2 p = make_float2(0x1.4201f40000000p-9f, 0x1.4201f40000000p-9f);
  p = __ffma2_rn(p, s, make_float2(-0x1.d7e7520000000p-7f, -0x1.d7e7520000000p-7f));
  p = __ffma2_rn(p, s, make_float2(0x1.45e3460000000p-5f, 0x1.45e3460000000p-5f));
  p = __ffma2_rn(p, s, make_float2(-0x1.2856fc0000000p-4f, -0x1.2856fc0000000p-4f));
  p = __ffma2_rn(p, s, make_float2(0x1.ae09700000000p-4f, 0x1.ae09700000000p-4f));
  p = __ffma2_rn(p, s, make_float2(-0x1.2205a00000000p-3f, -0x1.2205a00000000p-3f));
  p = __ffma2_rn(p, s, make_float2(0x1.994fb60000000p-3f, 0x1.994fb60000000p-3f));
  p = __ffma2_rn(p, s, make_float2(-0x1.5553680000000p-2f, -0x1.5553680000000p-2f));
  p = __ffma2_rn(p, s, make_float2(0x1.fffffc0000000p-1f, 0x1.fffffc0000000p-1f));
  return p;
}
#endif

}  // namespace xy
