// Double-float (df64) error-free transformations shared by the kernels that carry values as
// unevaluated sums of two FP32 numbers (hi + lo, about 48 significant bits): the Arnoldi
// kernels of the outer FGMRES and the leaf's Gauss-Jordan inverse.  A complex df64 value is
// a float4 (re_hi, im_hi, re_lo, im_lo).
//
// Every rounding step uses the _rn intrinsics, which the compiler never contracts into fused
// multiply-adds (a contracted s + a*b would break TwoSum).
#pragma once

#include <cuda_runtime.h>

namespace hps {
namespace dfops {

// t + err = a + b exactly (TwoSum, Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& t, float& err) {
  t = __fadd_rn(a, b);
  const float v = __fsub_rn(t, a);
  err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, v)), __fsub_rn(b, v));
}

// (s, c) += a * b for real df64 a = (ah, al), b = (bh, bl): TwoProduct of the leading
// parts (FMA) with the cross terms folded into its error, TwoSum into s, errors into c.
__device__ __forceinline__ void dot2(float& s, float& c, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// (s, c) += a * b for df64 a = (ah, al) and FP32 b
__device__ __forceinline__ void dot2f(float& s, float& c, float ah, float al, float b) {
  const float p = __fmul_rn(ah, b);
  float e = __fmaf_rn(ah, b, -p);
  e = __fmaf_rn(al, b, e);
  float t, err;
  two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// normalise (s, c) into (hi, lo)
__device__ __forceinline__ void fast2(float s, float c, float& hi, float& lo) { two_sum(s, c, hi, lo); }

// complex df64 v - f r
__device__ __forceinline__ float4 cfms(float4 v, float4 f, float4 r) {
  float sr = v.x, cr = v.z, si = v.y, ci = v.w;
  dot2(sr, cr, -f.x, -f.z, r.x, r.z);  // - Re f Re r
  dot2(sr, cr, f.y, f.w, r.y, r.w);    // + Im f Im r
  dot2(si, ci, -f.x, -f.z, r.y, r.w);  // - Re f Im r
  dot2(si, ci, -f.y, -f.w, r.x, r.z);  // - Im f Re r
  float4 o;
  fast2(sr, cr, o.x, o.z);
  fast2(si, ci, o.y, o.w);
  return o;
}

// complex df64 a b
__device__ __forceinline__ float4 cmul(float4 a, float4 b) {
  float sr = 0.f, cr = 0.f, si = 0.f, ci = 0.f;
  dot2(sr, cr, a.x, a.z, b.x, b.z);
  dot2(sr, cr, -a.y, -a.w, b.y, b.w);
  dot2(si, ci, a.x, a.z, b.y, b.w);
  dot2(si, ci, a.y, a.w, b.x, b.z);
  float4 o;
  fast2(sr, cr, o.x, o.z);
  fast2(si, ci, o.y, o.w);
  return o;
}

// complex df64 1 / a = conj(a) / |a|^2: |a|^2 in df64, its reciprocal from an approximate FP32
// one by a Newton step in df64 (r = r0 + r0 (1 - d r0)), then conj(a) r
__device__ __forceinline__ float4 cinv(float4 a) {
  float ds = 0.f, dc = 0.f;
  dot2(ds, dc, a.x, a.z, a.x, a.z);
  dot2(ds, dc, a.y, a.w, a.y, a.w);
  float dh, dl;
  fast2(ds, dc, dh, dl);
  float r0;  // approximate reciprocal: the Newton step below supplies the remaining bits
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0) : "f"(dh));
  float es = 1.f, ec = 0.f;
  dot2(es, ec, -dh, -dl, r0, 0.f);  // 1 - d r0, about 2^-24
  const float e = __fadd_rn(es, ec);
  float rh, rl;
  two_sum(r0, __fmul_rn(r0, e), rh, rl);
  float4 o;
  float s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f;
  dot2(s1, c1, a.x, a.z, rh, rl);
  dot2(s2, c2, -a.y, -a.w, rh, rl);
  fast2(s1, c1, o.x, o.z);
  fast2(s2, c2, o.y, o.w);
  return o;
}

__device__ __forceinline__ float4 from_d2(double2 v) {
  const float rh = (float)v.x, ih = (float)v.y;
  return make_float4(rh, ih, (float)(v.x - (double)rh), (float)(v.y - (double)ih));
}
__device__ __forceinline__ double2 to_d2(float4 v) {
  return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
}

}  // namespace dfops
}  // namespace hps
