// CTA-wide mixed-radix Stockham FFT over a tile of lines held in shared
// memory (Eq. fft_correlation_func needs forward and inverse 3D DFTs; each is
// three passes of these 1D line transforms).
//
// Element n of line l lives at buf[n * es + l * ls].  Strided passes (lines
// along y or x, consecutive lines = consecutive innermost indices) use
// es = number of lines, ls = 1; contiguous passes (lines along z) use es = 1,
// ls = P + 1 (odd, so a warp touching consecutive lines hits distinct banks).
//
// Stage with radix R after Ns points have been combined (Ns = product of the
// earlier radices): butterfly i in [0, P/R) reads x[i + r P/R], multiplies by
// w_P^(r (i mod Ns) P/(Ns R)), takes an R-point DFT and writes to
// (i / Ns) Ns R + (i mod Ns) + r Ns.  Radices 8, 4, 2, 3 and 5 are hand-written;
// 7 uses the R-point DFT matrix read from the same twiddle table.
#pragma once
#include <type_traits>

#include "arith.cuh"
#include "tc05.cuh"
#include "tc_dft.cuh"

namespace bpmf {

struct FftPlan {
  int n;       // transform length P
  int nst;     // number of stages
  int r[12];   // radix of each stage, product = n; 32 = tensor-core stage
  const uint4 *tca;  // fragment table of the tensor-core radix-32 stage (split-bf16), or null
  // tcgen05 form of that stage (when set): the DFT-32 matrix parts in the
  // tensor cores' shared-memory layout, the byte offset of kTc05Smem bytes of
  // scratch in the kernel's dynamic shared memory, and an error flag
  const __nv_bfloat16 *tc05_f;
  int tc05_off;
  int *err;
};

// exp(-2 pi i m / R) for the radices of dft_small (R <= 16, 0 <= m < R): the
// float nearest to the real and the imaginary part, the same values as the
// hi parts of the shared-memory twiddle table, as compile-time constants so
// that the float path of dft_small reads no table for its internal twiddles.
__host__ __device__ constexpr float unit_root_re(int R, int m) {
  switch (R * 16 + m) {
    case 3 * 16 + 1: return -0.5f;
    case 3 * 16 + 2: return -0.5f;
    case 5 * 16 + 1: return 0.309017f;
    case 5 * 16 + 2: return -0.809017f;
    case 5 * 16 + 3: return -0.809017f;
    case 5 * 16 + 4: return 0.309017f;
    case 7 * 16 + 1: return 0.6234898f;
    case 7 * 16 + 2: return -0.22252093f;
    case 7 * 16 + 3: return -0.90096885f;
    case 7 * 16 + 4: return -0.90096885f;
    case 7 * 16 + 5: return -0.22252093f;
    case 7 * 16 + 6: return 0.6234898f;
    case 8 * 16 + 1: return 0.70710677f;
    case 8 * 16 + 2: return -0.0f;
    case 8 * 16 + 3: return -0.70710677f;
    case 8 * 16 + 4: return -1.0f;
    case 8 * 16 + 5: return -0.70710677f;
    case 8 * 16 + 6: return 0.0f;
    case 8 * 16 + 7: return 0.70710677f;
    case 9 * 16 + 1: return 0.76604444f;
    case 9 * 16 + 2: return 0.17364818f;
    case 9 * 16 + 3: return -0.5f;
    case 9 * 16 + 4: return -0.9396926f;
    case 9 * 16 + 5: return -0.9396926f;
    case 9 * 16 + 6: return -0.5f;
    case 9 * 16 + 7: return 0.17364818f;
    case 9 * 16 + 8: return 0.76604444f;
    case 10 * 16 + 1: return 0.809017f;
    case 10 * 16 + 2: return 0.309017f;
    case 10 * 16 + 3: return -0.309017f;
    case 10 * 16 + 4: return -0.809017f;
    case 10 * 16 + 5: return -1.0f;
    case 10 * 16 + 6: return -0.809017f;
    case 10 * 16 + 7: return -0.309017f;
    case 10 * 16 + 8: return 0.309017f;
    case 10 * 16 + 9: return 0.809017f;
    case 12 * 16 + 1: return 0.8660254f;
    case 12 * 16 + 2: return 0.5f;
    case 12 * 16 + 3: return -0.0f;
    case 12 * 16 + 4: return -0.5f;
    case 12 * 16 + 5: return -0.8660254f;
    case 12 * 16 + 6: return -1.0f;
    case 12 * 16 + 7: return -0.8660254f;
    case 12 * 16 + 8: return -0.5f;
    case 12 * 16 + 9: return 0.0f;
    case 12 * 16 + 10: return 0.5f;
    case 12 * 16 + 11: return 0.8660254f;
    case 14 * 16 + 1: return 0.90096885f;
    case 14 * 16 + 2: return 0.6234898f;
    case 14 * 16 + 3: return 0.22252093f;
    case 14 * 16 + 4: return -0.22252093f;
    case 14 * 16 + 5: return -0.6234898f;
    case 14 * 16 + 6: return -0.90096885f;
    case 14 * 16 + 7: return -1.0f;
    case 14 * 16 + 8: return -0.90096885f;
    case 14 * 16 + 9: return -0.6234898f;
    case 14 * 16 + 10: return -0.22252093f;
    case 14 * 16 + 11: return 0.22252093f;
    case 14 * 16 + 12: return 0.6234898f;
    case 14 * 16 + 13: return 0.90096885f;
    case 15 * 16 + 1: return 0.9135454f;
    case 15 * 16 + 2: return 0.6691306f;
    case 15 * 16 + 3: return 0.309017f;
    case 15 * 16 + 4: return -0.104528464f;
    case 15 * 16 + 5: return -0.5f;
    case 15 * 16 + 6: return -0.809017f;
    case 15 * 16 + 7: return -0.9781476f;
    case 15 * 16 + 8: return -0.9781476f;
    case 15 * 16 + 9: return -0.809017f;
    case 15 * 16 + 10: return -0.5f;
    case 15 * 16 + 11: return -0.104528464f;
    case 15 * 16 + 12: return 0.309017f;
    case 15 * 16 + 13: return 0.6691306f;
    case 15 * 16 + 14: return 0.9135454f;
    case 16 * 16 + 1: return 0.9238795f;
    case 16 * 16 + 2: return 0.70710677f;
    case 16 * 16 + 3: return 0.38268343f;
    case 16 * 16 + 4: return -0.0f;
    case 16 * 16 + 5: return -0.38268343f;
    case 16 * 16 + 6: return -0.70710677f;
    case 16 * 16 + 7: return -0.9238795f;
    case 16 * 16 + 8: return -1.0f;
    case 16 * 16 + 9: return -0.9238795f;
    case 16 * 16 + 10: return -0.70710677f;
    case 16 * 16 + 11: return -0.38268343f;
    case 16 * 16 + 12: return 0.0f;
    case 16 * 16 + 13: return 0.38268343f;
    case 16 * 16 + 14: return 0.70710677f;
    case 16 * 16 + 15: return 0.9238795f;
    default: return 1.f;  // m = 0
  }
}
__host__ __device__ constexpr float unit_root_im(int R, int m) {
  switch (R * 16 + m) {
    case 3 * 16 + 1: return -0.8660254f;
    case 3 * 16 + 2: return 0.8660254f;
    case 5 * 16 + 1: return -0.95105654f;
    case 5 * 16 + 2: return -0.58778524f;
    case 5 * 16 + 3: return 0.58778524f;
    case 5 * 16 + 4: return 0.95105654f;
    case 7 * 16 + 1: return -0.7818315f;
    case 7 * 16 + 2: return -0.9749279f;
    case 7 * 16 + 3: return -0.43388373f;
    case 7 * 16 + 4: return 0.43388373f;
    case 7 * 16 + 5: return 0.9749279f;
    case 7 * 16 + 6: return 0.7818315f;
    case 8 * 16 + 1: return -0.70710677f;
    case 8 * 16 + 2: return -1.0f;
    case 8 * 16 + 3: return -0.70710677f;
    case 8 * 16 + 4: return 0.0f;
    case 8 * 16 + 5: return 0.70710677f;
    case 8 * 16 + 6: return 1.0f;
    case 8 * 16 + 7: return 0.70710677f;
    case 9 * 16 + 1: return -0.64278764f;
    case 9 * 16 + 2: return -0.9848077f;
    case 9 * 16 + 3: return -0.8660254f;
    case 9 * 16 + 4: return -0.34202015f;
    case 9 * 16 + 5: return 0.34202015f;
    case 9 * 16 + 6: return 0.8660254f;
    case 9 * 16 + 7: return 0.9848077f;
    case 9 * 16 + 8: return 0.64278764f;
    case 10 * 16 + 1: return -0.58778524f;
    case 10 * 16 + 2: return -0.95105654f;
    case 10 * 16 + 3: return -0.95105654f;
    case 10 * 16 + 4: return -0.58778524f;
    case 10 * 16 + 5: return 0.0f;
    case 10 * 16 + 6: return 0.58778524f;
    case 10 * 16 + 7: return 0.95105654f;
    case 10 * 16 + 8: return 0.95105654f;
    case 10 * 16 + 9: return 0.58778524f;
    case 12 * 16 + 1: return -0.5f;
    case 12 * 16 + 2: return -0.8660254f;
    case 12 * 16 + 3: return -1.0f;
    case 12 * 16 + 4: return -0.8660254f;
    case 12 * 16 + 5: return -0.5f;
    case 12 * 16 + 6: return 0.0f;
    case 12 * 16 + 7: return 0.5f;
    case 12 * 16 + 8: return 0.8660254f;
    case 12 * 16 + 9: return 1.0f;
    case 12 * 16 + 10: return 0.8660254f;
    case 12 * 16 + 11: return 0.5f;
    case 14 * 16 + 1: return -0.43388373f;
    case 14 * 16 + 2: return -0.7818315f;
    case 14 * 16 + 3: return -0.9749279f;
    case 14 * 16 + 4: return -0.9749279f;
    case 14 * 16 + 5: return -0.7818315f;
    case 14 * 16 + 6: return -0.43388373f;
    case 14 * 16 + 7: return 0.0f;
    case 14 * 16 + 8: return 0.43388373f;
    case 14 * 16 + 9: return 0.7818315f;
    case 14 * 16 + 10: return 0.9749279f;
    case 14 * 16 + 11: return 0.9749279f;
    case 14 * 16 + 12: return 0.7818315f;
    case 14 * 16 + 13: return 0.43388373f;
    case 15 * 16 + 1: return -0.40673664f;
    case 15 * 16 + 2: return -0.7431448f;
    case 15 * 16 + 3: return -0.95105654f;
    case 15 * 16 + 4: return -0.9945219f;
    case 15 * 16 + 5: return -0.8660254f;
    case 15 * 16 + 6: return -0.58778524f;
    case 15 * 16 + 7: return -0.20791169f;
    case 15 * 16 + 8: return 0.20791169f;
    case 15 * 16 + 9: return 0.58778524f;
    case 15 * 16 + 10: return 0.8660254f;
    case 15 * 16 + 11: return 0.9945219f;
    case 15 * 16 + 12: return 0.95105654f;
    case 15 * 16 + 13: return 0.7431448f;
    case 15 * 16 + 14: return 0.40673664f;
    case 16 * 16 + 1: return -0.38268343f;
    case 16 * 16 + 2: return -0.70710677f;
    case 16 * 16 + 3: return -0.9238795f;
    case 16 * 16 + 4: return -1.0f;
    case 16 * 16 + 5: return -0.9238795f;
    case 16 * 16 + 6: return -0.70710677f;
    case 16 * 16 + 7: return -0.38268343f;
    case 16 * 16 + 8: return 0.0f;
    case 16 * 16 + 9: return 0.38268343f;
    case 16 * 16 + 10: return 0.70710677f;
    case 16 * 16 + 11: return 0.9238795f;
    case 16 * 16 + 12: return 1.0f;
    case 16 * 16 + 13: return 0.9238795f;
    case 16 * 16 + 14: return 0.70710677f;
    case 16 * 16 + 15: return 0.38268343f;
    default: return 0.f;  // m = 0
  }
}

// v times w_R^m = exp(-2 pi i m / R) (conjugated for the inverse), for the
// twiddles inside dft_small: the float path takes the constants above (-i, +i
// and -1 as a rotation and a negation), the float-pair path the table, whose
// entries for R lie P / R apart.
template <class T, int R>
__device__ __forceinline__ cx<T> tw_small_mul(cx<T> v, int m, bool inv, const float4 *tw, int P) {
  if constexpr (std::is_same<T, float>::value) {
    if (4 * m == R) return c_rot(v, inv);
    if (4 * m == 3 * R) return c_rot(v, !inv);
    if (2 * m == R) return cx<float>{-v.re, -v.im};
    const float im = unit_root_im(R, m);
    return c_mul(v, cx<float>{unit_root_re(R, m), inv ? -im : im});
  } else {
    return c_mul(v, tw_load<T>(tw[m * (P / R)], inv));
  }
}
// w_R^m as a table entry {re hi, im hi, re lo, im lo} (the float path: the
// constants, lo parts zero)
template <class T, int R>
__device__ __forceinline__ float4 root_q(int m, const float4 *tw, int P) {
  if constexpr (std::is_same<T, float>::value) {
    return make_float4(unit_root_re(R, m), unit_root_im(R, m), 0.f, 0.f);
  } else {
    return tw[m * (P / R)];
  }
}

template <class T, int R>
__device__ __forceinline__ void dft_small(cx<T> *v, bool inv, const float4 *tw, int P) {
  if constexpr (R == 2) {
    cx<T> a = v[0], b = v[1];
    v[0] = c_add(a, b);
    v[1] = c_sub(a, b);
  } else if constexpr (R == 4) {
    cx<T> a = c_add(v[0], v[2]), b = c_sub(v[0], v[2]);
    cx<T> c = c_add(v[1], v[3]), d = c_rot(c_sub(v[1], v[3]), inv);
    v[0] = c_add(a, c);
    v[2] = c_sub(a, c);
    v[1] = c_add(b, d);
    v[3] = c_sub(b, d);
  } else if constexpr (R == 8) {
    cx<T> a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      a[k] = c_add(v[k], v[k + 4]);
      b[k] = c_sub(v[k], v[k + 4]);
    }
    // b1 *= w8, b2 *= w8^2 = -i (fwd), b3 *= w8^3; conjugated for inverse
    const float4 q = root_q<T, 8>(1, tw, P);    // exp(-i pi/4): (c, -c)
    const T c = s_mk<T>(q.x, q.z);                 // cos(pi/4) as hi/lo
    {
      T x = b[1].re, y = b[1].im;
      b[1] = inv ? cx<T>{s_mul(s_sub(x, y), c), s_mul(s_add(x, y), c)}
                 : cx<T>{s_mul(s_add(x, y), c), s_mul(s_sub(y, x), c)};
    }
    b[2] = c_rot(b[2], inv);
    {
      T x = b[3].re, y = b[3].im;
      b[3] = inv ? cx<T>{s_neg(s_mul(s_add(x, y), c)), s_mul(s_sub(x, y), c)}
                 : cx<T>{s_mul(s_sub(y, x), c), s_neg(s_mul(s_add(x, y), c))};
    }
    dft_small<T, 4>(a, inv, tw, P);
    dft_small<T, 4>(b, inv, tw, P);
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      v[2 * m] = a[m];
      v[2 * m + 1] = b[m];
    }
  } else if constexpr (R == 3) {
    // X0 = a + (b + c);  X1,2 = a - (b + c)/2 -/+ i (sqrt(3)/2)(b - c)  (forward)
    const float4 q = root_q<T, 3>(1, tw, P);     // exp(-2 pi i / 3) = (-1/2, -sqrt(3)/2)
    const T s3 = s_neg(s_mk<T>(q.y, q.w));       // sqrt(3)/2 as hi/lo
    const T half = s_mk<T>(0.5f, 0.f);
    const cx<T> sp = c_add(v[1], v[2]), sm = c_sub(v[1], v[2]);
    const cx<T> t1 = c_sub(v[0], cx<T>{s_mul(sp.re, half), s_mul(sp.im, half)});
    const cx<T> t2 = c_rot(cx<T>{s_mul(sm.re, s3), s_mul(sm.im, s3)}, inv);  // -i t (fwd), +i t (inv)
    v[0] = c_add(v[0], sp);
    v[1] = c_add(t1, t2);
    v[2] = c_sub(t1, t2);
  } else if constexpr (R == 5) {
    // with w = exp(-2 pi i / 5) = c1 - i sa, w^2 = c2 - i sb and w^(5-m) the
    // conjugate of w^m, the pairs (1, 4) and (2, 3) combine as
    //   X1,4 = v0 + c1 (v1 + v4) + c2 (v2 + v3) -/+ i (sa (v1 - v4) + sb (v2 - v3))
    //   X2,3 = v0 + c2 (v1 + v4) + c1 (v2 + v3) -/+ i (sb (v1 - v4) - sa (v2 - v3))
    // (forward; the inverse flips the sign of i)
    const float4 q1 = root_q<T, 5>(1, tw, P), q2 = root_q<T, 5>(2, tw, P);
    const T c1 = s_mk<T>(q1.x, q1.z), sa = s_neg(s_mk<T>(q1.y, q1.w));
    const T c2 = s_mk<T>(q2.x, q2.z), sb = s_neg(s_mk<T>(q2.y, q2.w));
    const cx<T> s1 = c_add(v[1], v[4]), d1 = c_sub(v[1], v[4]);
    const cx<T> s2 = c_add(v[2], v[3]), d2 = c_sub(v[2], v[3]);
    const cx<T> t1 = c_add(v[0], cx<T>{s_add(s_mul(s1.re, c1), s_mul(s2.re, c2)), s_add(s_mul(s1.im, c1), s_mul(s2.im, c2))});
    const cx<T> t2 = c_add(v[0], cx<T>{s_add(s_mul(s1.re, c2), s_mul(s2.re, c1)), s_add(s_mul(s1.im, c2), s_mul(s2.im, c1))});
    const cx<T> u1 = c_rot(cx<T>{s_add(s_mul(d1.re, sa), s_mul(d2.re, sb)), s_add(s_mul(d1.im, sa), s_mul(d2.im, sb))}, inv);
    const cx<T> u2 = c_rot(cx<T>{s_sub(s_mul(d1.re, sb), s_mul(d2.re, sa)), s_sub(s_mul(d1.im, sb), s_mul(d2.im, sa))}, inv);
    v[0] = c_add(v[0], c_add(s1, s2));
    v[1] = c_add(t1, u1);
    v[4] = c_sub(t1, u1);
    v[2] = c_add(t2, u2);
    v[3] = c_sub(t2, u2);
  } else if constexpr (R == 9 || R == 10 || R == 12 || R == 14 || R == 15 || R == 16) {
    // composite radix R = R1 R2 in registers (Cooley-Tukey, decimation in
    // time): R2 DFTs of length R1 over the strided inputs v[R2 n1 + n2],
    // internal twiddles w_R^(n2 k1), then R1 DFTs of length R2; output
    // k1 + R1 k2
    constexpr int R1 = (R == 9 || R == 15) ? 3 : ((R == 10 || R == 14) ? 2 : 4);
    constexpr int R2 = R / R1;
    cx<T> a[R2][R1];
#pragma unroll
    for (int n2 = 0; n2 < R2; ++n2) {
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) a[n2][n1] = v[R2 * n1 + n2];
      dft_small<T, R1>(a[n2], inv, tw, P);
#pragma unroll
      for (int k1 = 1; k1 < R1; ++k1)
        if (n2 > 0) a[n2][k1] = tw_small_mul<T, R>(a[n2][k1], n2 * k1, inv, tw, P);
    }
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) {
      cx<T> b[R2];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) b[n2] = a[n2][k1];
      dft_small<T, R2>(b, inv, tw, P);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k1 + R1 * k2] = b[k2];
    }
  } else {
    // radix 7: X[a] = sum_b v[b] w_R^(a b)
    cx<T> out[R];
#pragma unroll
    for (int a = 0; a < R; ++a) {
      cx<T> acc = v[0];
#pragma unroll
      for (int b = 1; b < R; ++b) acc = c_add(acc, tw_small_mul<T, R>(v[b], (a * b) % R, inv, tw, P));
      out[a] = acc;
    }
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = out[a];
  }
}

template <class T, int R, int NL>
__device__ __forceinline__ void fft_stage(const cx<T> *src, cx<T> *dst, int es, int ls, int nlines_rt, int P, int Ns,
                                          const float4 *tw, bool inv) {
  const int nlines = NL > 0 ? NL : nlines_rt;  // compile-time line count when given
  const int nb = P / R;
  const int items = nb * nlines;
  const int tstride = P / (Ns * R);
  for (int it = threadIdx.x; it < items; it += blockDim.x) {
    const int l = it % nlines, i = it / nlines;
    const int j = i % Ns;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(i + r * nb) * es + l * ls];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw_load<T>(tw[r * j * tstride], inv));
    }
    dft_small<T, R>(v, inv, tw, P);
    const int o = (i / Ns) * Ns * R + j;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(o + r * Ns) * es + l * ls] = v[r];  // lazy pairs; stores renormalise
  }
}

// Transforms nlines lines in place-by-ping-pong.  Data must be in b0 and
// visible to the CTA (caller syncs before).  Returns the buffer holding the
// result; the CTA is synchronised on return.  NL > 0 fixes the line count at
// compile time (it must equal nlines).
// TC: compile the tensor-core radix-32 stages (split-bf16 kernels only).
template <class T, int NL = 0, bool TC = false>
__device__ cx<T> *cta_fft(cx<T> *b0, cx<T> *b1, int es, int ls, int nlines, const FftPlan &pl, const float4 *tw,
                          bool inv) {
  int Ns = 1;
  cx<T> *src = b0, *dst = b1;
  for (int s = 0; s < pl.nst; ++s) {
    const int R = pl.r[s];
    switch (R) {
      case 32:
        if constexpr (TC && std::is_same<T, float>::value) {
          if (pl.tc05_f) {
            extern __shared__ unsigned char tc05_dyn[];
            tc05_dft32_stage(src, dst, es, ls, nlines, pl.n, Ns, tw, inv, pl.tc05_f, tc05_dyn + pl.tc05_off, pl.err);
          } else {
            tc_dft32_stage(src, dst, es, ls, nlines, pl.n, Ns, tw, inv, pl.tca);
          }
        }
        break;
      case 8: fft_stage<T, 8, NL>(src, dst, es, ls, nlines, pl.n, Ns, tw, inv); break;
      case 4: fft_stage<T, 4, NL>(src, dst, es, ls, nlines, pl.n, Ns, tw, inv); break;
      case 2: fft_stage<T, 2, NL>(src, dst, es, ls, nlines, pl.n, Ns, tw, inv); break;
      case 3: fft_stage<T, 3, NL>(src, dst, es, ls, nlines, pl.n, Ns, tw, inv); break;
      case 5: fft_stage<T, 5, NL>(src, dst, es, ls, nlines, pl.n, Ns, tw, inv); break;
      default: fft_stage<T, 7, NL>(src, dst, es, ls, nlines, pl.n, Ns, tw, inv); break;
    }
    __syncthreads();
    cx<T> *t = src;
    src = dst;
    dst = t;
    Ns *= R;
  }
  return src;
}

// ---------------------------------------------------------------------------
// Compile-time plans for common transform lengths: radices, stage strides and
// the line count are constants, so the per-butterfly index arithmetic folds
// away.  CtPlan<P, false> has the stages of the generic engine (the same
// rounding); CtPlan<P, true> ("few") combines them into two stages with a
// composite last radix (9, 10 or 12 in registers): one shared-memory pass and
// one barrier fewer, for callers with enough lines per stage and registers.
template <int P, bool FEW>
struct CtPlan {
  static constexpr int nst = 0;
  __host__ __device__ static constexpr int r(int) { return 1; }
};
template <bool FEW>
struct CtPlan<32, FEW> {
  static constexpr int nst = 2;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : 4; }
};
template <bool FEW>
struct CtPlan<64, FEW> {
  static constexpr int nst = 2;
  __host__ __device__ static constexpr int r(int) { return 8; }
};
template <>
struct CtPlan<96, false> {
  static constexpr int nst = 3;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : (s == 1 ? 4 : 3); }
};
template <>
struct CtPlan<96, true> {
  static constexpr int nst = 2;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : 12; }
};
template <>
struct CtPlan<80, false> {
  static constexpr int nst = 3;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : (s == 1 ? 2 : 5); }
};
template <>
struct CtPlan<80, true> {
  static constexpr int nst = 2;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : 10; }
};
template <>
struct CtPlan<72, false> {
  static constexpr int nst = 3;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : 3; }
};
template <>
struct CtPlan<72, true> {
  static constexpr int nst = 2;
  __host__ __device__ static constexpr int r(int s) { return s == 0 ? 8 : 9; }
};
template <bool FEW>
struct CtPlan<128, FEW> {
  static constexpr int nst = 3;
  __host__ __device__ static constexpr int r(int s) { return s < 2 ? 8 : 2; }
};
template <int P, bool FEW, int S>
__host__ __device__ constexpr int ct_ns() {  // product of the radices before stage S
  int n = 1;
  for (int i = 0; i < S; ++i) n *= CtPlan<P, FEW>::r(i);
  return n;
}

template <class T, int P, bool FEW, int S, int NL, int ES, int LS, int NT>
__device__ __forceinline__ void fft_stage_ct(const cx<T> *src, cx<T> *dst, const float4 *tw, bool inv) {
  constexpr int R = CtPlan<P, FEW>::r(S);
  constexpr int Ns = ct_ns<P, FEW, S>();
  constexpr int nb = P / R;
  constexpr int items = nb * NL;
  constexpr int tstride = P / (Ns * R);
#pragma unroll 1
  for (int it = threadIdx.x; it < items; it += NT) {
    const int l = it % NL, i = it / NL;
    const int j = i % Ns;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(i + r * nb) * ES + l * LS];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = c_mul(v[r], tw_load<T>(tw[r * j * tstride], inv));
    }
    dft_small<T, R>(v, inv, tw, P);
    const int o = (i / Ns) * Ns * R + j;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(o + r * Ns) * ES + l * LS] = v[r];
  }
}

template <class T, int P, bool FEW, int S, int NL, int ES, int LS, int NT>
__device__ __forceinline__ cx<T> *cta_fft_ct_from(cx<T> *src, cx<T> *dst, const float4 *tw, bool inv) {
  if constexpr (S == CtPlan<P, FEW>::nst) {
    return src;
  } else {
    fft_stage_ct<T, P, FEW, S, NL, ES, LS, NT>(src, dst, tw, inv);
    __syncthreads();
    return cta_fft_ct_from<T, P, FEW, S + 1, NL, ES, LS, NT>(dst, src, tw, inv);
  }
}

// Compile-time counterpart of cta_fft for P in {32, 64, 72, 80, 96, 128}; NT
// must equal blockDim.x.
template <class T, int P, bool FEW, int NL, int ES, int LS, int NT>
__device__ __forceinline__ cx<T> *cta_fft_ct(cx<T> *b0, cx<T> *b1, const float4 *tw, bool inv) {
  return cta_fft_ct_from<T, P, FEW, 0, NL, ES, LS, NT>(b0, b1, tw, inv);
}

// Transform with the compile-time engine when the plan and line count match a
// specialisation (lines contiguous: CONTIG, element stride 1, line stride
// P + 1; otherwise element stride NL, line stride 1), else the generic engine.
template <class T, int NL, int NT, bool CONTIG, bool FEW = false, bool TC = false>
__device__ __forceinline__ cx<T> *cta_fft_auto(cx<T> *b0, cx<T> *b1, int es, int ls, int nlines, const FftPlan &pl,
                                               const float4 *tw, bool inv) {
  if (nlines == NL && pl.tca == nullptr) {
    switch (pl.n) {
#define BPMF_CT_CASE(PP)                                                                    \
  case PP:                                                                                 \
    return CONTIG ? cta_fft_ct<T, PP, FEW, NL, 1, PP + 1, NT>(b0, b1, tw, inv)             \
                  : cta_fft_ct<T, PP, FEW, NL, NL, 1, NT>(b0, b1, tw, inv);
      BPMF_CT_CASE(96)
      BPMF_CT_CASE(80)
      BPMF_CT_CASE(72)
      BPMF_CT_CASE(64)
      BPMF_CT_CASE(32)
#undef BPMF_CT_CASE
      default:
        break;
    }
  }
  return cta_fft<T, 0, TC>(b0, b1, es, ls, nlines, pl, tw, inv);
}

}  // namespace bpmf
