// Float-float ("double-single") arithmetic on the FP32 pipe: a real number is
// the unevaluated sum hi + lo of two floats, a complex number a float4
// (re_hi, re_lo, im_hi, im_lo). Used by the float-float Dslash kernels (the
// reliable-update passes of the mixed solvers), where the GB300's FP64 rate,
// 1/64 of FP32, would otherwise bound the work.
//   TwoProduct(a, b) = (p, e): p = fl(a b), e = fma(a, b, -p)   exact (Dekker 1971, with an FMA)
//   TwoSum(s, p) = (s', t): s' = fl(s + p), b' = s' - s,
//                  t = (s - (s' - b')) + (p - b')              exact (Knuth, TAOCP vol. 2, 4.2.2)
#pragma once

#include <cuda_runtime.h>

// s += a * b for float-float a = (ah, al), b = (bh, bl); s = (sh, sl) with sl carrying the low part,
// not renormalised between steps. The _rn intrinsics keep the compiler from fusing these steps into
// FMAs, which would break the exactness of TwoSum.
__device__ __forceinline__ void ff_acc(float& sh, float& sl, float ah, float al, float bh, float bl) {
  const float p = __fmul_rn(ah, bh);
  float e = fmaf(ah, bh, -p);
  e = fmaf(ah, bl, e);
  e = fmaf(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float bv = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bv)), __fsub_rn(p, bv));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

__device__ __forceinline__ void ff_norm(float& h, float& l) {
  const float s = __fadd_rn(h, l);
  l = __fsub_rn(l, __fsub_rn(s, h));
  h = s;
}

// acc (re_h, re_l, im_h, im_l per colour) += U v
__device__ __forceinline__ void ff_mv(float4 (&acc)[3], const float4 (&U)[9], const float4 (&v)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 u = U[a * 3 + b], w = v[b];
      ff_acc(acc[a].x, acc[a].y, u.x, u.y, w.x, w.y);    // + ur vr
      ff_acc(acc[a].x, acc[a].y, -u.z, -u.w, w.z, w.w);  // - ui vi
      ff_acc(acc[a].z, acc[a].w, u.x, u.y, w.z, w.w);    // + ur vi
      ff_acc(acc[a].z, acc[a].w, u.z, u.w, w.x, w.y);    // + ui vr
    }
}

// acc -= U^dagger v
__device__ __forceinline__ void ff_mdv_sub(float4 (&acc)[3], const float4 (&U)[9], const float4 (&v)[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float4 u = U[b * 3 + a], w = v[b];  // conj(U[b][a]) v[b], subtracted
      ff_acc(acc[a].x, acc[a].y, -u.x, -u.y, w.x, w.y);  // - ur vr
      ff_acc(acc[a].x, acc[a].y, -u.z, -u.w, w.z, w.w);  // - ui vi
      ff_acc(acc[a].z, acc[a].w, -u.x, -u.y, w.z, w.w);  // - ur vi
      ff_acc(acc[a].z, acc[a].w, u.z, u.w, w.x, w.y);    // + ui vr
    }
}

// FP64 -> float-float: hi = fl32(d), lo = fl32(d - hi)
__device__ __forceinline__ float4 split_ff(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

// float-float -> FP64
__device__ __forceinline__ double2 join_ff(float4 v) {
  return make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}
