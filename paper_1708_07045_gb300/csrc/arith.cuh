// Scalar arithmetic for the correlation path, in two forms that share every
// kernel through templates:
//
//   float : plain IEEE single precision.
//   ff    : a compensated pair of floats (hi + lo, |lo| <= ulp(hi)/2 after
//           normalisation) carrying ~44-48 significant bits, built only from
//           FP32 instructions (error-free TwoSum / TwoProd with FMA).
//
// Why the pair form exists: an FFT correlation's rounding error scales with
// the GLOBAL magnitude of the grids (roughly eps * sqrt(log2 N^3) * rms(G_R) *
// ||G_L||_2), not with the energy of a given pose.  Receptor LJ-repulsive grids
// clipped at 1e4 and ligand factors sqrt(eps) R^12 ~ 1e3 put that error near
// 1 kcal/mol in FP32, three orders above the 1e-3 kcal/mol target; the pair
// form brings it to ~1e-6.
//
// Every operation uses the explicit round-to-nearest intrinsics so that the
// compiler cannot contract or reassociate the error-free transformations.
// Adds and multiplies return lazily normalised pairs; values are renormalised
// once per butterfly output and before every store.
#pragma once
#include <cuda_runtime.h>

namespace bpmf {

struct ff {
  float hi, lo;
};

// ---- float ---------------------------------------------------------------
__device__ __forceinline__ float s_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float s_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float s_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float s_neg(float a) { return -a; }
__device__ __forceinline__ float s_hi(float a) { return a; }
__device__ __forceinline__ float s_lo(float) { return 0.f; }
__device__ __forceinline__ float s_norm(float a) { return a; }

// ---- ff ------------------------------------------------------------------
__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return ff{s, e};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff{s, e};
}
// Lazy float-pair add: the error-free sum of the high parts plus both low
// parts, NOT renormalised (|lo| may reach a few ulp(hi)); every operation
// below accepts such operands, and s_norm renormalises where a canonical pair
// is needed (shared / global stores, comparisons).
__device__ __forceinline__ ff s_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  return ff{s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo))};
}
__device__ __forceinline__ ff s_norm(ff a) { return fast_two_sum(a.hi, a.lo); }
__device__ __forceinline__ ff s_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff s_sub(ff a, ff b) { return s_add(a, s_neg(b)); }
__device__ __forceinline__ ff s_mul(ff a, ff b) {  // lazy, like s_add
  float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return ff{p, e};
}
__device__ __forceinline__ float s_hi(ff a) { return a.hi; }
__device__ __forceinline__ float s_lo(ff a) { return a.lo; }

// ---- construction from (hi, lo) and zero, selected by the result type -----
template <class T> __device__ __forceinline__ T s_mk(float hi, float lo);
template <> __device__ __forceinline__ float s_mk<float>(float hi, float) { return hi; }
template <> __device__ __forceinline__ ff s_mk<ff>(float hi, float lo) { return ff{hi, lo}; }
template <class T> __device__ __forceinline__ T s_zero() { return s_mk<T>(0.f, 0.f); }
template <class T> __device__ __forceinline__ T s_from(float a) { return s_mk<T>(a, 0.f); }

// ---- complex -------------------------------------------------------------
template <class T>
struct cx {
  T re, im;
};

template <class T>
__device__ __forceinline__ cx<T> c_add(cx<T> a, cx<T> b) {
  return cx<T>{s_add(a.re, b.re), s_add(a.im, b.im)};
}
template <class T>
__device__ __forceinline__ cx<T> c_sub(cx<T> a, cx<T> b) {
  return cx<T>{s_sub(a.re, b.re), s_sub(a.im, b.im)};
}
// a*b + c*d for float pairs with one TwoSum: both products' error terms and
// the cross terms are gathered by FMA before a single renormalisation.
__device__ __forceinline__ ff ff_dot2(ff a, ff b, ff c, ff d) {
  const float p1 = __fmul_rn(a.hi, b.hi);
  float e1 = __fmaf_rn(a.hi, b.hi, -p1);
  e1 = __fmaf_rn(a.hi, b.lo, e1);
  e1 = __fmaf_rn(a.lo, b.hi, e1);
  const float p2 = __fmul_rn(c.hi, d.hi);
  float e2 = __fmaf_rn(c.hi, d.hi, -p2);
  e2 = __fmaf_rn(c.hi, d.lo, e2);
  e2 = __fmaf_rn(c.lo, d.hi, e2);
  const ff s = two_sum(p1, p2);
  return ff{s.hi, __fadd_rn(s.lo, __fadd_rn(e1, e2))};  // lazy
}
__device__ __forceinline__ float ff_dot2(float a, float b, float c, float d) {
  return __fmaf_rn(a, b, __fmul_rn(c, d));
}

template <class T>
__device__ __forceinline__ cx<T> c_mul(cx<T> a, cx<T> b) {
  return cx<T>{ff_dot2(a.re, b.re, s_neg(a.im), b.im), ff_dot2(a.re, b.im, a.im, b.re)};
}
// a * conj(b)
template <class T>
__device__ __forceinline__ cx<T> c_mulconj(cx<T> a, cx<T> b) {
  return cx<T>{ff_dot2(a.re, b.re, a.im, b.im), ff_dot2(a.im, b.re, s_neg(a.re), b.im)};
}
template <class T>
__device__ __forceinline__ cx<T> c_conj(cx<T> a) {
  return cx<T>{a.re, s_neg(a.im)};
}
// multiply by -i (forward) or +i (inverse)
template <class T>
__device__ __forceinline__ cx<T> c_rot(cx<T> a, bool inverse) {
  return inverse ? cx<T>{s_neg(a.im), a.re} : cx<T>{a.im, s_neg(a.re)};
}
template <class T>
__device__ __forceinline__ cx<T> c_scale(cx<T> a, T s) {
  return cx<T>{s_mul(a.re, s), s_mul(a.im, s)};
}
template <class T>
__device__ __forceinline__ cx<T> c_norm(cx<T> a) {
  return cx<T>{s_norm(a.re), s_norm(a.im)};
}
template <class T>
__device__ __forceinline__ cx<T> c_zero() {
  return cx<T>{s_zero<T>(), s_zero<T>()};
}

// Twiddle tables hold exp(-2 pi i k / P) for k in [0, P) as
// float4 {re_hi, im_hi, re_lo, im_lo}, rounded from a long-double evaluation.
template <class T>
__device__ __forceinline__ cx<T> tw_load(const float4 &w, bool inverse) {
  T re = s_mk<T>(w.x, w.z), im = s_mk<T>(w.y, w.w);
  return cx<T>{re, inverse ? s_neg(im) : im};
}

// ---- placement ("FFT-based BPMF Estimation": the lowest coordinate of each
// axis two grid spacings above plane 0) ---------------------------------------
// Grid-unit position g = (x - lo) / h + 2 as a float pair: x - lo exactly
// (TwoSum), then a two-step quotient by the float-pair spacing.
__device__ __forceinline__ ff place_ff(float x, float lo, ff h) {
  const ff dx = two_sum(x, -lo);
  const float q1 = __fdiv_rn(dx.hi, h.hi);
  const float p = __fmul_rn(q1, h.hi);
  const float pe = __fmaf_rn(q1, h.hi, -p);
  float r = __fsub_rn(__fsub_rn(dx.hi, p), pe);
  r = __fadd_rn(r, __fsub_rn(dx.lo, __fmul_rn(q1, h.lo)));
  const float q2 = __fdiv_rn(r, h.hi);
  return s_norm(s_add(fast_two_sum(q1, q2), ff{2.f, 0.f}));
}

// Trilinear cell and fraction of a float-pair coordinate: c = floor(g) (the
// cell below an exact node position), f = g - c exactly, clamped to [0, 1].
__device__ __forceinline__ void cell_ff(ff g, int &c, ff &f) {
  float cf = floorf(g.hi);
  if (g.hi == cf && g.lo < 0.f) cf -= 1.f;
  f = two_sum(__fsub_rn(g.hi, cf), g.lo);  // g.hi - cf is exact
  if (f.hi < 0.f) f = ff{0.f, 0.f};
  if (f.hi > 1.f || (f.hi == 1.f && f.lo > 0.f)) f = ff{1.f, 0.f};
  c = (int)cf;
}

}  // namespace bpmf
