// Double-float ("double-word") arithmetic on the FP32 pipe: a value is h + l
// with |l| at most about half an ulp of h once normalised.  Built from the
// error-free transforms TwoSum (Knuth), FastTwoSum (Dekker) and TwoProd by
// FMA; products drop l*l and sums add the low parts without compensation, so
// an operation's relative error is a small multiple of u^2 (u = 2^-24),
// about 2^-46, against 2^-53 in FP64, at FP32-pipe throughput (GB300's FP64
// pipe runs at about 1/64 of the FP32 rate).
//
// Every operation is an explicitly rounded intrinsic (__fadd_rn, __fmul_rn,
// fmaf), so the compiler cannot contract a product into a later sum and break
// the error-free transforms.
#pragma once
#include <cuda_runtime.h>

namespace sps_dw {

struct dw {
  float h, l;
  dw() = default;
  __device__ __forceinline__ dw(float a, float b) : h(a), l(b) {}
  __device__ __forceinline__ dw(int a) : h((float)a), l(0.f) {}   // exact for |a| < 2^24
};
__device__ __forceinline__ dw two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return dw(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}
__device__ __forceinline__ dw fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return dw(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dw operator+(dw a, dw b) {
  const dw s = two_sum(a.h, b.h);
  return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dw operator-(dw a) { return dw(-a.h, -a.l); }
__device__ __forceinline__ dw operator-(dw a, dw b) { return a + (-b); }
__device__ __forceinline__ dw& operator+=(dw& a, dw b) { return a = a + b; }
__device__ __forceinline__ dw operator*(dw a, dw b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
  return fast_two_sum(p, e);
}
__device__ __forceinline__ dw operator*(int a, dw b) { return dw(a) * b; }
// 1 / a: one Newton step from the FP32 reciprocal, its residual by FMAs
__device__ __forceinline__ dw recip(dw a) {
  const float y = __frcp_rn(a.h);
  const float r = fmaf(-a.l, y, fmaf(-a.h, y, 1.0f));
  return fast_two_sum(y, __fmul_rn(y, r));
}
__device__ __forceinline__ dw operator/(dw a, dw b) { return a * recip(b); }
// acc += a b without renormalising acc (the low part collects the errors)
__device__ __forceinline__ void dw_mac(dw& acc, dw a, dw b) {
  const float p = __fmul_rn(a.h, b.h);
  const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
  const dw s = two_sum(acc.h, p);
  acc.h = s.h;
  acc.l = __fadd_rn(acc.l, __fadd_rn(s.l, e));
}
__device__ __forceinline__ dw dw_of(double d) {
  const float h = __double2float_rn(d);
  return dw(h, __double2float_rn(d - (double)h));
}
__device__ __forceinline__ double dw_val(dw a) { return (double)a.h + (double)a.l; }

// Unnormalised forms for long dependent chains (renormalise with dw_norm
// before a value's low part could grow past a few ulps of its high part):
// sum with TwoSum on the high parts, product by TwoProd without the l*l term.
__device__ __forceinline__ dw dw_add_u(dw a, dw b) {
  const dw s = two_sum(a.h, b.h);
  return dw(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dw dw_mul_u(dw a, dw b) {
  const float p = __fmul_rn(a.h, b.h);
  return dw(p, fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p))));
}
__device__ __forceinline__ dw dw_sqr_u(dw a) {
  const float p = __fmul_rn(a.h, a.h);
  return dw(p, fmaf(a.h, a.l, fmaf(a.h, a.l, fmaf(a.h, a.h, -p))));
}
__device__ __forceinline__ dw dw_norm(dw a) { return fast_two_sum(a.h, a.l); }

// 1 / sqrt(a), a > 0: the SFU estimate refined once in FP32, then one Newton
// step with the residual 1 - a y^2 formed by FMAs (y^2 = t + te exactly)
__device__ __forceinline__ dw dw_rsqrt(dw a) {
  float y = rsqrtf(a.h);
  y = __fmul_rn(y, fmaf(__fmul_rn(-0.5f, a.h), __fmul_rn(y, y), 1.5f));
  const float t = __fmul_rn(y, y), te = fmaf(y, y, -t);
  const float r = fmaf(-a.l, t, fmaf(-a.h, te, fmaf(-a.h, t, 1.0f)));
  return fast_two_sum(y, __fmul_rn(__fmul_rn(0.5f, y), r));
}

}  // namespace sps_dw
