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
    const float4 q = tw[P / 8];                 // exp(-i pi/4): (c, -c)
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
    const float4 q = tw[P / 3];                  // exp(-2 pi i / 3) = (-1/2, -sqrt(3)/2)
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
    const float4 q1 = tw[P / 5], q2 = tw[2 * (P / 5)];
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
        if (n2 > 0) a[n2][k1] = c_mul(a[n2][k1], tw_load<T>(tw[(n2 * k1) * (P / R)], inv));
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
    // radix 7: X[a] = sum_b v[b] w_R^(a b), w_R^m = tw[m P / R]
    cx<T> out[R];
    const int st = P / R;
#pragma unroll
    for (int a = 0; a < R; ++a) {
      cx<T> acc = v[0];
#pragma unroll
      for (int b = 1; b < R; ++b) acc = c_add(acc, c_mul(v[b], tw_load<T>(tw[((a * b) % R) * st], inv)));
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
