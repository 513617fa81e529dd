// The x pass of the FP32 forms on compile-time transform edges P = 8 R
// (R = 8, 9, 10, 12, 14, 15, 16: edges 64 to 128): forward DFT of the ligand's three
// channels along x, the conj-multiply-sum with every receptor spectrum (Eq.
// fft_correlation_func), inverse DFT along x, site window (the same work as
// k_xfused, organised for fewer instructions per point).
//
// Each DFT has two in-place stages (four-step factorisation, n = n1 + 8 n2,
// f = k2 + R k1):
//   forward  A: per n1, R-point DFT over n2 of x[n1 + 8 n2], times w_P^(n1 k2)
//            B: per k2, 8-point DFT over n1                 -> X[k2 + R k1]
//   inverse  B': per k2, inverse 8-point DFT over k1, times conj(w_P^(n1 k2))
//            A': per n1, inverse R-point DFT over k2        -> x[n1 + 8 n2]
// A stage unit reads and writes the same rows, so no second buffer is needed:
// the spectra live in shared memory in the permuted row order
// row 8 k2 + k1 <-> frequency k2 + R k1, and the inverse returns natural order.
//
// CTA = 2 configurations x 8 consecutive (y, zf) columns, one half-warp per
// k2 (16 R threads).  A half-warp owns one unit at a time and its 16 lanes are
// the 16 lines of a channel (configuration g = lane / 8, column l = lane % 8):
// every shared access of a half-warp is 16 consecutive float2 (no bank
// conflicts), and the index arithmetic is per unit, not per element.
// Shared-memory round trips are kept to the one transpose each DFT needs:
// stage A transforms the ligand's rows in place where one TMA box per CTA
// left them in the forward buffer (or reads them from global memory), stage B
// leaves the three channels' spectra at the half-warp's frequencies k2 + R k1
// in its registers for every receptor, the spectral product is formed there
// with the staged receptor tile inside the first inverse stage, and the last
// inverse stage writes the site-window rows straight to global memory.
//
// Each receptor's spectra for the CTA's columns (3 channels x P frequencies x
// 8 columns) are staged in one of two shared-memory tiles two receptors
// ahead: by one TMA tensor copy (cp.async.bulk.tensor, completion on an
// mbarrier per tile) when the receptor group has at most kXpMaxMaps
// receptors, else by 16-byte cp.async copies.  With two inverse buffers the
// CTA meets one barrier per receptor: the product of receptor k + 1 (other
// buffer) runs while receptor k's last stage does.  Every mbarrier wait is
// bounded: after about a second it sets the call's error flag, waits
// (bounded) for the tiles still in flight, and the CTA returns.
#include <cuda.h>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "kernels.cuh"
#include "tma.cuh"

namespace bpmf {

namespace {

constexpr int kXpLW = 8;       // columns per CTA
constexpr int kXpG = 2;        // configurations per CTA
constexpr int kXpNLF = 48;     // forward lines: 3 channels x 2 configurations x 8 columns

__device__ __forceinline__ int imod_p(int a, int m) {
  const int r = a % m;
  return r < 0 ? r + m : r;
}

__device__ __forceinline__ void cp16(void *dst, const void *src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// One receptor's spectra for this CTA's 8 columns, all P frequencies and 3
// channels, into RS[t][row][8] in the permuted row order of the forward
// spectra (row 8 k2 + k1 <-> frequency k2 + R k1): 16-byte asynchronous
// copies of column pairs (Q is even and q0 a multiple of 8, so each pair is
// 16-byte aligned and wholly inside or outside the spectrum).
template <int P, int NT>
__device__ __forceinline__ void stage_receptor(cx<float> *RS, const float2 *rh, int Q, int q0) {
  constexpr int R = P / 8;
  for (int e = threadIdx.x; e < 3 * P * 4; e += NT) {
    const int c = e & 3, tr = e >> 2, t = tr / P, row = tr - t * P;
    const int f = (row >> 3) + R * (row & 7);
    const bool v = q0 + 2 * c < Q;
    cp16(&RS[tr * kXpLW + 2 * c], v ? rh + ((long long)t * P + f) * Q + q0 + 2 * c : rh, v);
  }
}

// Launch shape of the x pass on edge P = 8 R: one half-warp per k2 (16 R
// threads), and the CTAs per SM the registers are budgeted for (the shared
// memory of P <= 80 fits four CTAs per SM, of P <= 96 three).
template <int P>
struct XpCfg {
  static constexpr int R = P / 8;
  static constexpr int NT = 16 * R;
  static constexpr int MINB = P <= 80 ? 4 : (P <= 96 ? 3 : 2);
  // on 72 and 80 the second receptor tile lies over the forward buffer's
  // last third (free once stage B has read it): four CTAs fit an SM
  static constexpr bool kAliasT1 = P == 72 || P == 80;
  // the last inverse stage has 8 units (n1); with 16 half-warps two share one
  static constexpr bool kSplitA = R == 16;
};

// Half of an inverse composite R-point DFT (R = R1 R2, decimation in time as
// in dft_small: R2 length-R1 DFTs over the inputs v[R2 n1 + n2], twiddles
// w_R^(n2 k1), then R1 length-R2 DFTs): the R1 / 2 sub-transforms k1 = h R1 / 2
// ... of half h, outputs o[i] = X[k1 + R1 k2] with k1 = h R1 / 2 + i / R2,
// k2 = i % R2.
template <int R>
__device__ __forceinline__ void idft_half(const cx<float> *v, int h, const float4 *tw, int P, cx<float> *o) {
  constexpr int R1 = 4, R2 = R / R1, H = R1 / 2;
  cx<float> b[H][R2];
#pragma unroll
  for (int n2 = 0; n2 < R2; ++n2) {
    cx<float> a[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) a[m] = v[R2 * m + n2];
    dft_small<float, R1>(a, true, tw, P);
#pragma unroll
    for (int kk = 0; kk < H; ++kk) {
      const int k1 = h * H + kk;
      cx<float> x = h ? a[H + kk] : a[kk];
      if (n2 > 0 && k1 > 0) x = tw_small_mul<float, R>(x, n2 * k1, true, tw, P);
      b[kk][n2] = x;
    }
  }
#pragma unroll
  for (int kk = 0; kk < H; ++kk) {
    dft_small<float, R2>(b[kk], true, tw, P);
#pragma unroll
    for (int k2 = 0; k2 < R2; ++k2) o[kk * R2 + k2] = b[kk][k2];
  }
}

// Shared memory of k_xpass<P>: the twiddles, the ligand spectra L [P][48]
// (reused as the two inverse buffers W [2][P][16] once the forward transform
// is done), two receptor tiles [3][P][8] (128-byte aligned TMA destinations;
// with kAliasT1 the second starts at L + 32 P, over L's last third, so the
// region is 80 P complex values instead of 96 P), and slack for the alignment.
template <int P>
constexpr size_t xpass_smem_bytes() {
  return sizeof(float4) * P + sizeof(cx<float>) * (size_t)P * (XpCfg<P>::kAliasT1 ? 80 : 96) + 128;
}

template <int P, bool TMA>
__global__ void __launch_bounds__(XpCfg<P>::NT, XpCfg<P>::MINB)
    k_xpass(XfusedArgs a, int batch, const __grid_constant__ XpassMaps maps) {
  constexpr int R = P / 8, NT = XpCfg<P>::NT;
  constexpr int NLI = 16;                    // inverse lines: 2 configurations x 8 columns
  constexpr int kTile = 3 * P * kXpLW;       // complex values of one receptor tile
  constexpr unsigned kTileBytes = kTile * sizeof(cx<float>);
  // arrivals of the two receptor tiles and of the ligand rows (TMA)
  __shared__ alignas(8) unsigned long long s_bar[3];
  extern __shared__ float4 smem[];
  // 128-byte aligned TMA destinations: the twiddles (16 P bytes, P a multiple
  // of 8) and L (384 P bytes) keep the receptor tiles aligned too
  float4 *tw = reinterpret_cast<float4 *>((reinterpret_cast<uintptr_t>(smem) + 127) & ~uintptr_t(127));  // [P]
  cx<float> *L = reinterpret_cast<cx<float> *>(tw + P);  // [P][48], then W [2][P][16]
  constexpr bool kAlias = XpCfg<P>::kAliasT1;
  // the receptor tiles [3][P][8]: T1 over L's last third (kAlias) or after T0
  cx<float> *T0 = L + (kAlias ? 56 : 48) * P;
  cx<float> *T1 = kAlias ? L + 32 * P : T0 + kTile;
  const int tid = threadIdx.x, hw = tid >> 4, hl = tid & 15;
  const int g = hl >> 3, l = hl & 7;
  const int nJG = (batch + kXpG - 1) / kXpG;
  const int j0 = (blockIdx.x % nJG) * kXpG;
  const int q0 = (blockIdx.x / nJG) * kXpLW;
  const int Q = (int)a.Q, K = a.K;
  const int j = j0 + g, q = q0 + l;
  const bool live = j < batch && q < Q;
  const long long limit = a.wait_test ? (1ll << 20) : (1ll << 31);
  const bool lig_tma = maps.lig_ok != 0;
  const int U0 = a.U0 < P ? a.U0 : P;
  // the ligand's rows for this CTA straight into L, in its row layout: one
  // box of the batch's U0 rows, issued at once (rows past a configuration's
  // own extent are loaded but not read; waiting for the extents first, to
  // load fewer rows, made the pass slower)
  if (lig_tma && tid == 0) {
    mbar_init(&s_bar[2], 1);
    mbar_arrive_expect(&s_bar[2], 384u * (unsigned)a.U0);
    tma_issue_4d(L, &maps.lig, 2 * q0, j0, 0, 0, &s_bar[2]);
  }
  for (int i = tid; i < P; i += NT) tw[i] = a.tw[i];
  // the first two receptors' spectra, asynchronously, while the ligand's are transformed
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_init(&s_bar[0], 1);
      mbar_init(&s_bar[1], 1);
      if (K > 0 && !a.wait_test) tma_load_3d(T0, &maps.m[0], 2 * q0, 0, 0, &s_bar[0], kTileBytes);
      if (!kAlias && K > 1) tma_load_3d(T1, &maps.m[1], 2 * q0, 0, 0, &s_bar[1], kTileBytes);
    }
  } else {
    if (K > 0) stage_receptor<P, NT>(T0, a.rhi[0], Q, q0);
    if (!kAlias && K > 1) stage_receptor<P, NT>(T1, a.rhi[1], Q, q0);
  }
  __syncthreads();
  // forward A: unit (n1, t), R-point DFT over n2 of rows n1 + 8 n2 of the
  // ligand's y-z spectra (rows at or beyond the configuration's box extent u0
  // are zero and not read), twiddled, into L: from the rows staged in L
  // (in place: a unit writes the rows it read), else straight from global
  // memory
  {
    const int u0 = live ? min(a.meta ? a.meta[j].u[0] : U0, U0) : 0;
    const cx<float> *ly = reinterpret_cast<const cx<float> *>(a.ly);
    if (lig_tma) {
      const bool ok = mbar_wait(&s_bar[2], 0, limit);
      if (__syncthreads_or(!ok)) {  // the CTA agrees, waits (bounded) for its copies in flight and returns
        if (tid == 0 && a.err) atomicOr(a.err, 1);
        mbar_wait(&s_bar[2], 0, limit);
        if constexpr (TMA) {
          if (K > 0 && !a.wait_test) mbar_wait(&s_bar[0], 0, limit);
          if (!kAlias && K > 1) mbar_wait(&s_bar[1], 0, limit);
        } else {
          cp_wait_all();
        }
        return;
      }
    }
    for (int u = hw; u < 8 * 3; u += R) {
      const int n1 = u & 7, t = u >> 3;
      const cx<float> *src = ly + (((long long)j * 3 + t) * a.U0 + n1) * Q + q;
      const cx<float> *stg = L + n1 * kXpNLF + t * 16 + hl;
      cx<float> v[R];
#pragma unroll
      for (int n2 = 0; n2 < R; ++n2)
        v[n2] = n1 + 8 * n2 < u0 ? (lig_tma ? stg[8 * n2 * kXpNLF] : src[(long long)8 * n2 * Q]) : cx<float>{0.f, 0.f};
      dft_small<float, R>(v, false, tw, P);
#pragma unroll
      for (int k2 = 1; k2 < R; ++k2) v[k2] = c_mul(v[k2], tw_load<float>(tw[n1 * k2], false));
      cx<float> *col = L + n1 * kXpNLF + t * 16 + hl;
#pragma unroll
      for (int k2 = 0; k2 < R; ++k2) col[8 * k2 * kXpNLF] = v[k2];
    }
  }
  __syncthreads();
  // forward B: unit k2 = hw, 8-point DFTs over n1 of the three channels' rows
  // 8 k2 + n1 -> X_t[k2 + R k1], kept in registers for every receptor
  const int k2 = hw;
  cx<float> Lr[3][8];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const cx<float> *col = L + 8 * k2 * kXpNLF + t * 16 + hl;
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) Lr[t][n1] = col[n1 * kXpNLF];
    dft_small<float, 8>(Lr[t], false, tw, P);
  }
  if constexpr (!TMA) cp_wait_all();
  __syncthreads();  // L is the inverse buffers W from here on
  // kAlias: the second receptor's spectra into T1, now that L's last third
  // has been read
  if constexpr (kAlias) {
    if (K > 1) {
      if constexpr (TMA) {
        if (tid == 0) tma_load_3d(T1, &maps.m[1], 2 * q0, 0, 0, &s_bar[1], kTileBytes);
      } else {
        stage_receptor<P, NT>(T1, a.rhi[1], Q, q0);
      }
    }
  }
  for (int k = 0; k < K; ++k) {
    const int b = k & 1;
    const cx<float> *rs0 = b ? T1 : T0;
    cx<float> *Wb = L + b * P * NLI;
    const int wm = live ? imod_p(a.info[j * K + k].wc[0], P) : 0;  // window start along x, mod P
    __builtin_assume(wm >= 0 && wm < P);
    bool ok = true;
    if constexpr (TMA) ok = mbar_wait(&s_bar[b], (k >> 1) & 1, limit);
    // product and inverse B', unit k2: P_f = sum_t R_{f,t} conj(L_t) at the
    // frequencies f = k2 + R k1, inverse 8-point DFT over k1, then
    // conj(w_P^(n1 k2)), into rows 8 k2 + n1 of W[b]
    {
      cx<float> v[8];
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) {
        // TMA tiles hold natural frequency order, the cp.async tiles row order
        const cx<float> *rs = rs0 + (TMA ? k2 + R * k1 : 8 * k2 + k1) * kXpLW + l;
        const cx<float> r0 = rs[0], r1 = rs[P * kXpLW], r2 = rs[2 * P * kXpLW];
        // sum_t R_t conj(L_t) as one fused multiply-add chain per part
        v[k1].re = __fmaf_rn(r0.re, Lr[0][k1].re,
                             __fmaf_rn(r0.im, Lr[0][k1].im,
                                       __fmaf_rn(r1.re, Lr[1][k1].re,
                                                 __fmaf_rn(r1.im, Lr[1][k1].im,
                                                           __fmaf_rn(r2.re, Lr[2][k1].re, __fmul_rn(r2.im, Lr[2][k1].im))))));
        v[k1].im = __fmaf_rn(r0.im, Lr[0][k1].re,
                             __fmaf_rn(-r0.re, Lr[0][k1].im,
                                       __fmaf_rn(r1.im, Lr[1][k1].re,
                                                 __fmaf_rn(-r1.re, Lr[1][k1].im,
                                                           __fmaf_rn(r2.im, Lr[2][k1].re, -__fmul_rn(r2.re, Lr[2][k1].im))))));
      }
      dft_small<float, 8>(v, true, tw, P);
#pragma unroll
      for (int n1 = 1; n1 < 8; ++n1) v[n1] = c_mul(v[n1], tw_load<float>(tw[n1 * k2], true));
      cx<float> *col = Wb + 8 * k2 * NLI + hl;
#pragma unroll
      for (int n1 = 0; n1 < 8; ++n1) col[n1 * NLI] = v[n1];
    }
    if constexpr (!TMA) cp_wait_all();  // receptor k + 1's tile, for the next product
    // W[b] is complete and tile b has been read.  On a timeout the CTA agrees,
    // waits (bounded) for the tiles still in flight and returns.
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && a.err) atomicOr(a.err, 1);
      if constexpr (TMA) {
        mbar_wait(&s_bar[b], (k >> 1) & 1, limit);
        if (k + 1 < K) mbar_wait(&s_bar[b ^ 1], ((k + 1) >> 1) & 1, limit);
      }
      return;
    }
    // receptor k + 2's spectra stream into tile b while this one is
    // transformed back and the next multiplied
    if (k + 2 < K) {
      if constexpr (TMA) {
        if (tid == 0) tma_load_3d(b ? T1 : T0, &maps.m[k + 2], 2 * q0, 0, 0, &s_bar[b], kTileBytes);
      } else {
        stage_receptor<P, NT>(b ? T1 : T0, a.rhi[k + 2], Q, q0);
      }
    }
    // inverse A', unit n1: inverse R-point DFT over k2 -> x[n1 + 8 n2]; the
    // rows inside the site window along x go straight to the output.  The
    // next receptor's product needs no barrier first: it writes the other W.
    cx<float> *dst = reinterpret_cast<cx<float> *>(a.x2) + ((long long)j * K + k) * a.S0 * Q + q;
    if constexpr (XpCfg<P>::kSplitA) {
      constexpr int R1 = 4, R2 = R / R1, H = R1 / 2;
      const int n1 = hw & 7, h = hw >> 3;
      const cx<float> *col = Wb + n1 * NLI + hl;
      cx<float> v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = col[8 * m * NLI];
      cx<float> o[R / 2];
      idft_half<R>(v, h, tw, P, o);
      if (live) {
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
          const int n2 = h * H + i / R2 + R1 * (i % R2);  // output k1 + R1 k2
          int s = n1 + 8 * n2 - wm;
          s += s < 0 ? P : 0;
          if (s < a.S0) dst[(long long)s * Q] = o[i];
        }
      }
    } else if (hw < 8) {
      const int n1 = hw;
      const cx<float> *col = Wb + n1 * NLI + hl;
      cx<float> v[R];
#pragma unroll
      for (int m = 0; m < R; ++m) v[m] = col[8 * m * NLI];
      dft_small<float, R>(v, true, tw, P);
      if (live) {
#pragma unroll
        for (int n2 = 0; n2 < R; ++n2) {
          int s = n1 + 8 * n2 - wm;
          s += s < 0 ? P : 0;
          if (s < a.S0) dst[(long long)s * Q] = v[n2];
        }
      }
    }
  }
}

template <int P>
size_t xpass_smem() {
  return xpass_smem_bytes<P>();
}

// Tensor maps of the receptor spectra [3][P][Q] float2 as FP32 [3][P][2Q],
// box [3][P][16 floats] (8 columns), cached by (spectrum, P, Q).
using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
std::mutex g_map_mu;
std::map<std::tuple<const void *, int, long long>, CUtensorMap> g_maps;

// the driver's tensor-map encoder (null when unavailable); call under g_map_mu
EncodeTiled tiled_encoder() {
  static EncodeTiled encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      cudaGetLastError();
      return nullptr;
    }
    encode = reinterpret_cast<EncodeTiled>(fn);
  }
  return encode;
}

bool receptor_map(const float2 *spec, int P, long long Q, CUtensorMap *out) {
  std::lock_guard<std::mutex> lk(g_map_mu);
  const auto key = std::make_tuple((const void *)spec, P, Q);
  auto it = g_maps.find(key);
  if (it != g_maps.end()) {
    *out = it->second;
    return true;
  }
  const EncodeTiled encode = tiled_encoder();
  if (!encode) return false;
  alignas(64) CUtensorMap m;
  const cuuint64_t dims[3] = {(cuuint64_t)(2 * Q), (cuuint64_t)P, 3};
  const cuuint64_t strides[2] = {(cuuint64_t)(2 * Q * sizeof(float)), (cuuint64_t)(2 * Q * sizeof(float) * P)};
  const cuuint32_t box[3] = {2 * kXpLW, (cuuint32_t)P, 3};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (encode(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2 *>(spec), dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  g_maps[key] = m;
  *out = m;
  return true;
}

// Tensor map of the ligand's y-z spectra ly [batch][3][U0][Q] float2 as FP32
// with dimensions (2Q, batch, 3, U0) and box (16 floats, 2, 3, U0): one CTA's
// rows in the forward buffer's layout [row][channel][configuration][column]
// (out-of-range configurations and columns read as zeros).  Needs two
// configurations, a 16-byte aligned ly and Q even.
bool ligand_map(const void *ly, long long Q, int U0, int batch, CUtensorMap *out) {
  if (batch < 2 || U0 < 1 || U0 > 256 || (Q & 1) || (reinterpret_cast<unsigned long long>(ly) & 15ull)) return false;
  std::lock_guard<std::mutex> lk(g_map_mu);
  const EncodeTiled encode = tiled_encoder();
  if (!encode) return false;
  const cuuint64_t row = (cuuint64_t)(2 * Q * sizeof(float));
  const cuuint64_t dims[4] = {(cuuint64_t)(2 * Q), (cuuint64_t)batch, 3, (cuuint64_t)U0};
  const cuuint64_t strides[3] = {row * 3 * U0, row * U0, row};
  const cuuint32_t box[4] = {2 * kXpLW, (cuuint32_t)kXpG, 3, (cuuint32_t)U0};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void *>(ly), dims, strides, box, estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int P>
cudaError_t launch_xpass_p(const XfusedArgs &a, int batch, cudaStream_t st) {
  const size_t smem = xpass_smem<P>();
  const long long blocks = (long long)((batch + kXpG - 1) / kXpG) * ((a.Q + kXpLW - 1) / kXpLW);
  XpassMaps maps;
  // the ligand rows of a CTA (384 U0 bytes) fit the forward buffer (384 P)
  maps.lig_ok = a.U0 <= P && ligand_map(a.ly, a.Q, a.U0, batch, &maps.lig) ? 1 : 0;
  bool tma = a.rhi_h && a.K <= kXpMaxMaps;
  for (int k = 0; tma && k < a.K; ++k) {
    // 16-byte aligned spectra whose rows are 16-byte multiples (Q even)
    tma = ((reinterpret_cast<unsigned long long>(a.rhi_h[k]) & 15ull) == 0) && receptor_map(a.rhi_h[k], P, a.Q, &maps.m[k]);
  }
  constexpr int NT = XpCfg<P>::NT;
  auto kern = tma ? k_xpass<P, true> : k_xpass<P, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)blocks, NT, smem, st>>>(a, batch, maps);
  return cudaGetLastError();
}

}  // namespace

bool xpass_supported(int P) {
  return P == 64 || P == 72 || P == 80 || P == 96 || P == 112 || P == 120 || P == 128;
}

cudaError_t launch_xpass(const XfusedArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (a.S0 > a.plan.n || a.plan.tca) return cudaErrorInvalidValue;
  if (a.Q % 2) return cudaErrorInvalidValue;  // 16-byte column pairs
  switch (a.plan.n) {
    case 64: return launch_xpass_p<64>(a, batch, st);
    case 72: return launch_xpass_p<72>(a, batch, st);
    case 80: return launch_xpass_p<80>(a, batch, st);
    case 96: return launch_xpass_p<96>(a, batch, st);
    case 112: return launch_xpass_p<112>(a, batch, st);
    case 120: return launch_xpass_p<120>(a, batch, st);
    case 128: return launch_xpass_p<128>(a, batch, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bpmf
