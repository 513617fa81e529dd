// The ligand's y-z spectra evaluated directly from its atoms (FP32 forms).
//
// The spread grid of one channel t is a sum of trilinear corner weights,
//   G_L(x, y, z) = sum_i gamma_t,i wx_i(x) wy_i(y) wz_i(z),
// so its 2D DFT over (y, z) on an x plane factorises per atom:
//   L_t(x, ky, kz) = sum_i gamma_t,i wx_i(x) A_i(ky) B_i(kz),
//   A_i(ky) = (1 - fy) w1^(ky cy) + fy w1^(ky (cy + 1)),  w1 = exp(-2 pi i / P1),
//   B_i(kz) = (1 - fz) w2^(kz cz) + fz w2^(kz (cz + 1)),  w2 = exp(-2 pi i / P2),
// with (cx, cy, cz) an atom's cell and (fx, fy, fz) its fractional offsets
// (wx = 1 - fx on plane cx, fx on plane cx + 1).  This is the spreading
// (Methodology, ligand grid) followed by the forward DFT along z (real to
// half spectrum, kz < P2/2 + 1) and y (Eq. fft_correlation_func), evaluated in
// one pass: a handful of atoms touch each plane, so a direct sum costs less
// than materialising the grid and transforming it, and it rounds less.
//
// CTA = (configuration, x plane of the ligand box).  Atom placement is the
// float-pair placement of the spreading kernel; weights and sums are FP32, in
// a fixed order (atoms in index order), so results are deterministic and do
// not depend on the batching.
#include <cuda_runtime.h>

#include <algorithm>

#include "kernels.cuh"

namespace bpmf {

constexpr int kLsAtoms = 256;  // atoms per ligand (BPMF_MAX_ATOMS)

__global__ void __launch_bounds__(256) k_ligspec(LigSpecArgs a) {
  extern __shared__ float2 s_dyn[];  // [chunk][P1] A, then [chunk][F2] B
  __shared__ int s_c[kLsAtoms][3];
  __shared__ float s_f[kLsAtoms][3];
  __shared__ int s_list[kLsAtoms];   // atoms touching this plane, in index order
  __shared__ float s_wg[kLsAtoms][3];  // wx gamma_t of the listed atoms
  __shared__ int s_cnt[9];
  const int ix = blockIdx.x, j = blockIdx.y;
  const ConfMeta m = a.meta[j];
  // planes beyond this configuration's ligand box hold no atom; the x pass
  // reads them as zeros without loading them
  if (ix >= m.u[0]) return;
  const int n = m.n_atoms;
  const ff h{a.h_hi, a.h_lo};
  // placement in float pairs, as the spreading kernel does it
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      int c;
      ff f;
      cell_ff(place_ff(a.coords[3ll * (m.atom_off + i) + d], m.lo[d], h), c, f);
      s_c[i][d] = c;
      s_f[i][d] = fminf(fmaxf(__fadd_rn(f.hi, f.lo), 0.f), 1.f);
    }
  }
  __syncthreads();
  // ordered list of the atoms on this plane (exclusive scan of the flags)
  {
    const int i = threadIdx.x;
    const bool on = i < n && (s_c[i][0] == ix || s_c[i][0] + 1 == ix);
    const unsigned bal = __ballot_sync(0xffffffffu, on);
    const int lane = i & 31, warp = i >> 5;
    if (lane == 0) s_cnt[warp] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int c = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        const int v = s_cnt[w];
        s_cnt[w] = c;
        c += v;
      }
      s_cnt[8] = c;
    }
    __syncthreads();
    if (on) {
      const int pos = s_cnt[warp] + __popc(bal & ((1u << lane) - 1u));
      s_list[pos] = i;
      const float wx = s_c[i][0] == ix ? __fsub_rn(1.f, s_f[i][0]) : s_f[i][0];
      for (int t = 0; t < 3; ++t)
        s_wg[pos][t] = __fmul_rn(wx, a.gamma[(long long)t * a.gamma_stride + m.gamma_off + i].x);
    }
    __syncthreads();
  }
  const int na = s_cnt[8];
  const int P1 = a.P1, P2 = a.P2, F2 = a.F2;
  const long long Q = a.Q;
  float2 *out[3];
  for (int t = 0; t < 3; ++t)
    out[t] = reinterpret_cast<float2 *>(a.ly) + (((long long)j * 3 + t) * a.U0 + ix) * Q;
  if (na == 0) {  // an empty plane: zero spectra
    for (long long q = threadIdx.x; q < Q; q += blockDim.x)
      for (int t = 0; t < 3; ++t) out[t][q] = make_float2(0.f, 0.f);
    return;
  }
  float2 *sA = s_dyn, *sB = s_dyn + (size_t)a.chunk * P1;
  for (int c0 = 0; c0 < na; c0 += a.chunk) {
    const int nc = min(a.chunk, na - c0);
    // per-atom factors A(ky), B(kz) from the twiddle tables; corners beyond
    // the ligand box are dropped, as the spreading drops them
    for (int e = threadIdx.x; e < nc * P1; e += blockDim.x) {
      const int q = e / P1, ky = e % P1, i = s_list[c0 + q];
      const int cy = s_c[i][1];
      const float fy = s_f[i][1];
      const float g0 = cy < a.U1 ? __fsub_rn(1.f, fy) : 0.f, g1 = cy + 1 < a.U1 ? fy : 0.f;
      const float4 t0 = a.tw1[(ky * cy) % P1], t1 = a.tw1[(ky * (cy + 1)) % P1];
      sA[e] = make_float2(__fmaf_rn(g1, t1.x, __fmul_rn(g0, t0.x)), __fmaf_rn(g1, t1.y, __fmul_rn(g0, t0.y)));
    }
    for (int e = threadIdx.x; e < nc * F2; e += blockDim.x) {
      const int q = e / F2, kz = e % F2, i = s_list[c0 + q];
      const int cz = s_c[i][2];
      const float fz = s_f[i][2];
      const float g0 = cz < a.U2 ? __fsub_rn(1.f, fz) : 0.f, g1 = cz + 1 < a.U2 ? fz : 0.f;
      const float4 t0 = a.tw2[(kz * cz) % P2], t1 = a.tw2[(kz * (cz + 1)) % P2];
      sB[e] = make_float2(__fmaf_rn(g1, t1.x, __fmul_rn(g0, t0.x)), __fmaf_rn(g1, t1.y, __fmul_rn(g0, t0.y)));
    }
    __syncthreads();
    // (ky, kz) = divmod(q, F2), stepped without a division per output
    const int dky = (int)blockDim.x / F2, dkz = (int)blockDim.x % F2;
    for (int q = threadIdx.x, ky = (int)threadIdx.x / F2, kz = (int)threadIdx.x % F2; q < (int)Q;
         q += blockDim.x, ky += dky, kz += dkz) {
      if (kz >= F2) {
        kz -= F2;
        ++ky;
      }
      float2 acc[3];
      for (int t = 0; t < 3; ++t) acc[t] = c0 == 0 ? make_float2(0.f, 0.f) : out[t][q];
      for (int e = 0; e < nc; ++e) {
        const float2 A = sA[e * P1 + ky], B = sB[e * F2 + kz];
        const float re = __fmaf_rn(A.x, B.x, -__fmul_rn(A.y, B.y));
        const float im = __fmaf_rn(A.x, B.y, __fmul_rn(A.y, B.x));
        for (int t = 0; t < 3; ++t) {
          const float wg = s_wg[c0 + e][t];
          acc[t].x = __fmaf_rn(wg, re, acc[t].x);
          acc[t].y = __fmaf_rn(wg, im, acc[t].y);
        }
      }
      for (int t = 0; t < 3; ++t) out[t][q] = acc[t];
    }
    __syncthreads();
  }
}

cudaError_t launch_ligspec(const LigSpecArgs &a_in, int batch, cudaStream_t st) {
  if (batch <= 0 || a_in.U0 <= 0) return cudaSuccess;
  LigSpecArgs a = a_in;
  // atoms whose factors fit in 96 KB of shared memory at once, and no more
  // than a plane can hold (the ligand's atoms): a small ligand keeps the
  // footprint small and more CTAs resident
  const int cap = a.nmax > 0 ? std::min(a.nmax, kLsAtoms) : kLsAtoms;
  a.chunk = (int)std::max<size_t>(1, std::min<size_t>(cap, (96 * 1024) / (sizeof(float2) * (a.P1 + a.F2))));
  const size_t smem = sizeof(float2) * (size_t)a.chunk * (a.P1 + a.F2);
  cudaError_t e = cudaFuncSetAttribute(k_ligspec, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_ligspec<<<dim3(a.U0, batch), 256, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bpmf
