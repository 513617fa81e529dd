// The y and z inverse transforms of the FP32 forms on compile-time edges
// P = A R (64, 72, 80, 96 = 8 R; 70 = 7 x 10, 84 = 7 x 12, 90 = 9 x 10,
// 100 = 10 x 10, 108 = 9 x 12), fused with the
// site mask and the plane's reduction: the work of k_zinv<float, NY> (Eq.
// fft_correlation_func's inverse transform, pruned to the site window, Eq.
// sample_mean_BPMF's sum), organised like k_xpass: each inverse DFT is two
// stages of a four-step factorisation (f = k2 + R k1, n = n1 + A n2, P = A R),
// each stage unit a half-warp whose 16 lanes are 16 lines (a quarter warp of
// 8 lines in the z stages, whose row pairs are few), so index arithmetic is
// per unit and the lanes of a unit access consecutive values.
//
// One CTA per (configuration, receptor, site plane s0), 256 threads:
//   y, unit (k2, g): rows k2 + R1 k1 (k1 < A1) of the x-pass plane [P1][F2],
//      columns 16 g .. 16 g + 15, read from global memory into registers;
//      inverse A1-point DFT over k1, times conj(w_P1^(n1 k2)) -> Y rows A1 k2 + n1;
//   y, unit (n1, g): inverse R1-point DFT over k2 -> y rows n1 + A1 n2; the rows
//      of the site window go to Zs[z frequency][s1];
//   z, unit (k2, g), a quarter warp: lines l = 8 g .. 8 g + 7 are the row pairs (2 l,
//      2 l + 1) packed as A + i B over the Hermitian-extended frequencies
//      k2 + R2 k1; inverse A2-point DFT, twiddle -> W rows A2 k2 + n1;
//   z, unit (n1, g): inverse R2-point DFT -> z index n1 + A2 n2, real part row
//      2 l, imaginary part row 2 l + 1: scaled, masked, into the plane's
//      energies (refined form) or -E/kT values (FP32 form);
// then the plane's reduction: the refined form's running minimum and
// candidate appends, or the FP32 form's max-shifted log-sum-exp partial.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "kernels.cuh"
#include "tma.cuh"

namespace bpmf {

namespace {

constexpr int kYzNT = 256;

__device__ __forceinline__ int imod_yz(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}

// row stride of Zs (complex values): even (16-byte pair loads) and 2 mod 4
// (the y stage's column-wise stores spread over the banks), >= 2 L
__host__ __device__ __forceinline__ int yz_zst(int S1) {
  const int two_l = 2 * ((S1 + 1) / 2);
  return (two_l & 2) ? two_l : two_l + 2;
}

// Shared memory of the edges (P1, P2) at a 40^2 site (the protein-scale one)
constexpr int yz_smem_40(int P1, int P2) {
  return 16 * (P1 + P2) + 8 * ((P1 * (P2 / 2 + 1) > P2 * 24 ? P1 * (P2 / 2 + 1) : P2 * 24) + (P2 / 2 + 1) * 42) + 6400;
}
// CTAs per SM the registers are budgeted for: 4 where that shared memory
// fits four CTAs (56 KB each with the static part), else 3
template <int A1, int R1, int A2, int R2>
__global__ void __launch_bounds__(kYzNT, yz_smem_40(A1 * R1, A2 * R2) <= 57296 ? 4 : 3) k_yzinv(ZinvArgs a) {
  constexpr int P1 = A1 * R1, P2 = A2 * R2;
  static_assert(P1 % 2 == 0, "a plane is a 16-byte multiple (bulk prefetch)");
  constexpr int F2 = P2 / 2 + 1;
  constexpr int NG1 = (F2 + 15) / 16;  // line groups of the y transform (columns)
  const int S1 = a.S1, S2 = a.S2;
  const int L = (S1 + 1) / 2;          // row pairs: lines of the z transform
  const int NGz = (L + 7) / 8;         // the z stages' units are 8 lanes (a quarter warp): few lines
  const int WS = 8 * NGz;              // row stride of W
  const int YW = P1 * F2 > P2 * WS ? P1 * F2 : P2 * WS;  // Y [P1][F2], then W [P2][WS]
  const int ZST = yz_zst(S1);
  extern __shared__ float4 smem[];
  float4 *tw1 = smem;                                     // [P1] exp(-2 pi i k / P1)
  float4 *tw2 = tw1 + P1;                                 // [P2]
  cx<float> *Y = reinterpret_cast<cx<float> *>(tw2 + P2); // [P1][F2], then W [P2][WS]
  cx<float> *W = Y;
  cx<float> *Zs = Y + YW;                                 // [F2][ZST]
  float *es = reinterpret_cast<float *>(Zs + F2 * ZST);   // [S1][S2]
  __shared__ float s_red[8];
  __shared__ float s_thr;
  const int tid = threadIdx.x, hw = tid >> 4, hl = tid & 15, qw = tid >> 3, ql = tid & 7;
  const int s0 = blockIdx.x % a.S0;
  const int jk = blockIdx.x / a.S0;  // j * K + k
  const PairInfo inf = a.info[jk];
  const bool refine = a.rs.cand != nullptr;
  if (!(s0 >= inf.sa[0] && s0 <= inf.sb[0])) {  // no valid translation in this plane
    if (tid == 0) a.part[blockIdx.x] = make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
    return;
  }
  const cx<float> *plane = reinterpret_cast<const cx<float> *>(a.x2) + (long long)blockIdx.x * a.Qx;
  // the whole plane is prefetched into the L2 (P1 F2 complex values: 16-byte
  // multiple, P1 even), so the first stage's later rounds hit it there
  if (tid == 0) bulk_prefetch_l2(plane, (unsigned)(P1 * F2 * sizeof(cx<float>)));
  // the first y unit's rows are requested before the twiddle copies, so the
  // two global-memory latencies overlap
  cx<float> v0[A1];
  {
    const int k2 = hw % R1, c = (hw / R1) * 16 + hl;
    if (hw < R1 * NG1 && c < F2) {
#pragma unroll
      for (int k1 = 0; k1 < A1; ++k1) v0[k1] = plane[(k2 + R1 * k1) * F2 + c];
    }
  }
  for (int i = tid; i < P1; i += kYzNT) tw1[i] = a.tw1[i];
  for (int i = tid; i < P2; i += kYzNT) tw2[i] = a.tw[i];
  if (S1 & 1)  // the last row pair's second row is zero
    for (int f = tid; f < F2; f += kYzNT) Zs[f * ZST + S1] = cx<float>{0.f, 0.f};
  const int wy = imod_yz(inf.wc[1], P1), wz = imod_yz(inf.wc[2], P2);
  __syncthreads();
  // y, first inverse stage: rows k2 + R k1 straight from global memory
  for (int u = hw; u < R1 * NG1; u += kYzNT / 16) {
    const int k2 = u % R1, c = (u / R1) * 16 + hl;
    if (c < F2) {
      cx<float> v[A1];
      if (u == hw) {
#pragma unroll
        for (int k1 = 0; k1 < A1; ++k1) v[k1] = v0[k1];
      } else {
#pragma unroll
        for (int k1 = 0; k1 < A1; ++k1) v[k1] = plane[(k2 + R1 * k1) * F2 + c];
      }
      dft_small<float, A1>(v, true, tw1, P1);
#pragma unroll
      for (int n1 = 1; n1 < A1; ++n1) v[n1] = c_mul(v[n1], tw_load<float>(tw1[n1 * k2], true));
#pragma unroll
      for (int n1 = 0; n1 < A1; ++n1) Y[(A1 * k2 + n1) * F2 + c] = v[n1];
    }
  }
  __syncthreads();
  // y, second inverse stage: the site window's rows into Zs[column][s1]
  for (int u = hw; u < A1 * NG1; u += kYzNT / 16) {
    const int n1 = u % A1, c = (u / A1) * 16 + hl;
    if (c < F2) {
      cx<float> v[R1];
#pragma unroll
      for (int k2 = 0; k2 < R1; ++k2) v[k2] = Y[(A1 * k2 + n1) * F2 + c];
      dft_small<float, R1>(v, true, tw1, P1);
#pragma unroll
      for (int n2 = 0; n2 < R1; ++n2) {
        int s1 = n1 + A1 * n2 - wy;
        s1 += s1 < 0 ? P1 : 0;
        if (s1 < S1) Zs[c * ZST + s1] = v[n2];
      }
    }
  }
  __syncthreads();
  // z, first inverse stage: row pairs as A + i B, Hermitian-extended
  for (int u = qw; u < R2 * NGz; u += kYzNT / 8) {
    const int k2 = u % R2, l = (u / R2) * 8 + ql;
    if (l < L) {
      cx<float> v[A2];
#pragma unroll
      for (int k1 = 0; k1 < A2; ++k1) {
        const int f = k2 + R2 * k1;
        const bool up = 2 * f <= P2;
        const int kk = up ? f : P2 - f;
        const float4 ab = *reinterpret_cast<const float4 *>(&Zs[kk * ZST + 2 * l]);  // A = (x, y), B = (z, w)
        float ai = ab.y, bi = ab.w;
        if (kk == 0 || 2 * kk == P2) ai = bi = 0.f;  // real bins
        if (!up) {
          ai = -ai;
          bi = -bi;
        }
        v[k1] = cx<float>{__fsub_rn(ab.x, bi), __fadd_rn(ai, ab.z)};
      }
      dft_small<float, A2>(v, true, tw2, P2);
#pragma unroll
      for (int n1 = 1; n1 < A2; ++n1) v[n1] = c_mul(v[n1], tw_load<float>(tw2[n1 * k2], true));
#pragma unroll
      for (int n1 = 0; n1 < A2; ++n1) W[(A2 * k2 + n1) * WS + l] = v[n1];
    }
  }
  __syncthreads();
  // z, second inverse stage: energies of rows 2 l and 2 l + 1 at z index n1 + 8 n2
  const float nscale = a.nscale_hi, escale = a.escale_hi;
  float ext = refine ? CUDART_INF_F : -CUDART_INF_F;  // plane minimum of E (refined) or maximum of -E/kT
  for (int u = qw; u < A2 * NGz; u += kYzNT / 8) {
    const int n1 = u % A2, l = (u / A2) * 8 + ql;
    if (l < L) {
      cx<float> v[R2];
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) v[k2] = W[(A2 * k2 + n1) * WS + l];
      dft_small<float, R2>(v, true, tw2, P2);
      const int s1a = 2 * l, s1b = 2 * l + 1;
      const bool oka = s1a >= inf.sa[1] && s1a <= inf.sb[1];
      const bool okb = s1b < S1 && s1b >= inf.sa[1] && s1b <= inf.sb[1];
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) {
        int s2 = n1 + A2 * n2 - wz;
        s2 += s2 < 0 ? P2 : 0;
        if (s2 < S2) {
          const bool ok2 = s2 >= inf.sa[2] && s2 <= inf.sb[2];
          float ea, eb;
          if (refine) {
            ea = (oka && ok2) ? __fmul_rn(v[n2].re, escale) : CUDART_INF_F;
            eb = (okb && ok2) ? __fmul_rn(v[n2].im, escale) : CUDART_INF_F;
            ext = fminf(ext, fminf(ea, eb));
          } else {
            ea = (oka && ok2) ? __fmul_rn(v[n2].re, nscale) : -CUDART_INF_F;
            eb = (okb && ok2) ? __fmul_rn(v[n2].im, nscale) : -CUDART_INF_F;
            ext = fmaxf(ext, fmaxf(ea, eb));
          }
          es[s1a * S2 + s2] = ea;
          if (s1b < S1) es[s1b * S2 + s2] = eb;
        }
      }
    }
  }
  // the plane's extreme value
  for (int o = 16; o > 0; o >>= 1)
    ext = refine ? fminf(ext, __shfl_xor_sync(0xffffffffu, ext, o)) : fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, o));
  if ((tid & 31) == 0) s_red[tid >> 5] = ext;
  __syncthreads();  // also publishes es
  const int nS = S1 * S2;
  if (refine) {
    // the plane's minimum lowers the pair's running minimum; translations
    // within W + 2B of it are appended to the pair's list (warp-aggregated).
    // The list is the pair's whole weight (the others lie more than W above
    // the pair's minimum and weigh less than 1e-5 of S together), so the
    // plane writes no partial of its own.
    if (tid == 0) {
      float v = s_red[0];
      for (int w = 1; w < kYzNT / 32; ++w) v = fminf(v, s_red[w]);
      float thr = -CUDART_INF_F;
      if (v < CUDART_INF_F) {
        const float run = fminf(ord2f(atomicMin(&a.rs.pmin[jk], f2ord(v))), v);
        thr = __fadd_ru(run, a.rs.win[jk % a.K]);
      }
      s_thr = thr;
      a.part[blockIdx.x] = make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const float thr = s_thr;
    const int lane = tid & 31;
    Cand *list = a.rs.cand + (long long)jk * a.rs.cap;
    const unsigned t0 = (unsigned)(s0 * S1 * S2);
    for (int b = tid & ~31; b < nS; b += kYzNT) {
      const int idx = b + lane;
      const float ef = idx < nS ? es[idx] : CUDART_INF_F;
      const bool keep = ef <= thr;
      const unsigned bal = __ballot_sync(0xffffffffu, keep);
      if (bal) {
        int base = 0;
        if (lane == 0) base = atomicAdd(&a.rs.cnt[jk], __popc(bal));
        base = __shfl_sync(0xffffffffu, base, 0);
        const int slot = base + __popc(bal & ((1u << lane) - 1u));
        // (a translation that does not fit makes k_refine flag the overflow)
        if (keep && slot < a.rs.cap) list[slot] = Cand{t0 + (unsigned)idx, ef};
      }
    }
    return;
  }
  // FP32 form: max-shifted sum of exp(-E/kT) over the plane
  float M = s_red[0];
  for (int w = 1; w < kYzNT / 32; ++w) M = fmaxf(M, s_red[w]);
  float acc = 0.f;
  if (M > -CUDART_INF_F)
    for (int idx = tid; idx < nS; idx += kYzNT) {
      const float x = es[idx];
      if (x > -CUDART_INF_F) acc += expf(__fsub_rn(x, M));
    }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __syncthreads();  // every thread has read s_red
  if ((tid & 31) == 0) s_red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kYzNT / 32; ++w) s += s_red[w];
    a.part[blockIdx.x] = make_float4(M, 0.f, M > -CUDART_INF_F ? s : 0.f, 0.f);
  }
}

template <int A1, int R1, int A2, int R2>
size_t yzinv_smem_p(int S1, int S2) {
  constexpr int P1 = A1 * R1, P2 = A2 * R2, F2 = P2 / 2 + 1;
  const int L = (S1 + 1) / 2, WS = 8 * ((L + 7) / 8);
  const size_t YW = (size_t)std::max(P1 * F2, P2 * WS);
  return sizeof(float4) * (P1 + P2) + sizeof(cx<float>) * (YW + (size_t)F2 * yz_zst(S1)) +
         sizeof(float) * (size_t)S1 * S2;
}

template <int A1, int R1, int A2, int R2>
cudaError_t launch_yzinv_p(const ZinvArgs &a, int batch, cudaStream_t st) {
  const size_t smem = yzinv_smem_p<A1, R1, A2, R2>(a.S1, a.S2);
  cudaError_t e =
      cudaFuncSetAttribute(k_yzinv<A1, R1, A2, R2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_yzinv<A1, R1, A2, R2><<<(unsigned)((long long)batch * a.K * a.S0), kYzNT, smem, st>>>(a);
  return cudaGetLastError();
}

// The compiled (y edge, z edge) pairs, each edge as A x R: every pair of the
// 8 R edges 64, 72, 80, 96, and each padded edge with its crop edge (the
// smooth edge near 5/6 of it) for 80, 84, 90, 96, 100 and 108.
#define BPMF_YZ_PAIRS(X)                                                                                        \
  X(8, 8, 8, 8) X(8, 8, 8, 9) X(8, 8, 8, 10) X(8, 8, 8, 12) X(8, 9, 8, 8) X(8, 9, 8, 9) X(8, 9, 8, 10)          \
  X(8, 9, 8, 12) X(8, 10, 8, 8) X(8, 10, 8, 9) X(8, 10, 8, 10) X(8, 10, 8, 12) X(8, 12, 8, 8) X(8, 12, 8, 9)    \
  X(8, 12, 8, 10) X(8, 12, 8, 12)                                                                              \
  X(7, 10, 7, 10) X(8, 10, 7, 10) X(7, 10, 8, 10)                                                              \
  X(7, 12, 7, 12) X(7, 12, 7, 10) X(7, 10, 7, 12)                                                              \
  X(9, 10, 9, 10) X(9, 10, 8, 10) X(8, 10, 9, 10)                                                              \
  X(10, 10, 10, 10) X(10, 10, 7, 12) X(7, 12, 10, 10)                                                          \
  X(9, 12, 9, 12) X(9, 12, 9, 10) X(9, 10, 9, 12)

size_t yz_smem(int P1, int P2, int S1, int S2) {
#define BPMF_YZ_SMEM(a1, r1, a2, r2) \
  if (P1 == a1 * r1 && P2 == a2 * r2) return yzinv_smem_p<a1, r1, a2, r2>(S1, S2);
  BPMF_YZ_PAIRS(BPMF_YZ_SMEM)
#undef BPMF_YZ_SMEM
  return 0;
}

cudaError_t yz_launch(int P1, int P2, const ZinvArgs &a, int batch, cudaStream_t st) {
#define BPMF_YZ_LAUNCH(a1, r1, a2, r2) \
  if (P1 == a1 * r1 && P2 == a2 * r2) return launch_yzinv_p<a1, r1, a2, r2>(a, batch, st);
  BPMF_YZ_PAIRS(BPMF_YZ_LAUNCH)
#undef BPMF_YZ_LAUNCH
  return cudaErrorInvalidValue;
}

}  // namespace

bool yzinv_supported(int P1, int P2, int S1, int S2, bool clash, bool export_E) {
  if (clash || export_E || S1 < 1 || S2 < 1 || S1 > P1 || S2 > P2) return false;
  const size_t smem = yz_smem(P1, P2, S1, S2);
  return smem > 0 && smem <= 227 * 1024;
}

cudaError_t launch_yzinv(const ZinvArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const int P1 = a.yplan.n, P2 = a.plan.n;
  if (!a.x2 || a.F2 != P2 / 2 + 1 || a.clash || a.export_E || !yzinv_supported(P1, P2, a.S1, a.S2, false, false) ||
      a.Qx != (long long)P1 * a.F2 || !a.tw1)
    return cudaErrorInvalidValue;
  return yz_launch(P1, P2, a, batch, st);
}

}  // namespace bpmf
