// Refined form (BPMF_MODE_REFINE): the FP32 correlation gives every
// translation's energy with an error below a bound B (8 eps sqrt(log2 P^3)
// sum_t rms(G_t) ||gamma_t||); only translations whose FP32 energy lies
// within W + 2B of the configuration's FP32 minimum can carry a weight above
// e^(-W/kT) of the largest, so only they are re-evaluated exactly: the direct
// sum the FFT correlation equals (trilinear interpolation of each receptor
// grid at every atom, Eqs. general_form / receptor_grid / correlation_func),
// in FP64.  The window W = kT max(20, ln(1e5 n)) (n translations in the site
// window) keeps the weight of the translations left at their FP32 values
// below 1e-5 of S.
//
// k_window (W + 2B per receptor), k_threshold (per pair: T = FP32 minimum +
// W + 2B), then k_refine, one CTA per (configuration, receptor, s0 plane);
// planes whose minimum lies above T keep the FP32 partial of k_zinv (all
// their weights lie below e^(-W/kT) of the largest), the others:
//   * every FP32 energy <= T is a candidate; a warp evaluates its
//     candidates together (lanes over atoms, FP64, shuffle reduction);
//   * S = sum over candidates of exp(-E_exact/kT) + sum over the others of
//     exp(-E_fp32/kT), max-shifted, written as the plane's LSE partial (the
//     merge is unchanged), and the exported energies (exact where refined)
//     when asked.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "kernels.cuh"

namespace bpmf {

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 trilinear interpolation of one grid at p (grid units); a position on
// the last node uses the cell below it.
__device__ __forceinline__ double trilinear64(const float *G, int N0, int N1, int N2, double px, double py,
                                              double pz) {
  const int cx = min(max((int)floor(px), 0), N0 - 2), cy = min(max((int)floor(py), 0), N1 - 2),
            cz = min(max((int)floor(pz), 0), N2 - 2);
  const double fx = px - cx, fy = py - cy, fz = pz - cz;
  const long long sy = N2, sx = (long long)N1 * N2;
  const float *g = G + cx * sx + cy * sy + cz;
  const double c00 = (double)g[0] * (1.0 - fz) + (double)g[1] * fz;
  const double c01 = (double)g[sy] * (1.0 - fz) + (double)g[sy + 1] * fz;
  const double c10 = (double)g[sx] * (1.0 - fz) + (double)g[sx + 1] * fz;
  const double c11 = (double)g[sx + sy] * (1.0 - fz) + (double)g[sx + sy + 1] * fz;
  const double c0 = c00 * (1.0 - fy) + c01 * fy, c1 = c10 * (1.0 - fy) + c11 * fy;
  return c0 * (1.0 - fx) + c1 * fx;
}

__global__ void __launch_bounds__(256) k_refine(RefineArgs a) {
  __shared__ double s_g[3][256];    // atom positions in the ligand-box frame (grid units), FP64
  __shared__ double s_gam[3][256];  // gamma_t,i, FP64
  __shared__ double s_mx[8], s_sm[8];
  __shared__ float s_non[8];
  const int s0 = blockIdx.x % a.S0;
  const int pair = blockIdx.x / a.S0;  // j * K + k
  const int j = pair / a.K, k = pair % a.K;
  // the pair's threshold (k_threshold): a plane whose FP32 minimum lies above
  // it has no candidate, and the FP32 partial k_zinv wrote for it stands
  const float Tf = a.thresh[pair];
  const float *pm = a.plane_min + (long long)pair * a.S0;
  if (!(pm[s0] <= Tf)) return;
  const ConfMeta m = a.meta[j];
  const PairInfo inf = a.info[pair];
  const RefTab t = a.tabs[k];
  const int n = m.n_atoms;
  const float Mf = a.pmin_pair[pair];
  const double M = (double)Mf;
  const double kT = a.kT;
  {
    const double h = a.h;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const float *x = a.coords + 3ll * (m.atom_off + i);
      for (int d = 0; d < 3; ++d) s_g[d][i] = ((double)x[d] - (double)m.lo[d]) / h + 2.0;
      for (int c = 0; c < 3; ++c) s_gam[c][i] = a.gamma64[(long long)c * a.gamma_stride + m.gamma_off + i];
    }
    __syncthreads();
  }
  const int nP = a.S1 * a.S2;
  const float *E = a.E + (long long)blockIdx.x * nP;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double mx = -CUDART_INF, sm = 0.0;  // exact candidates, max-shifted (per warp, identical on its lanes)
  // the others, relative to exp(-M / kT), per thread: each lies below
  // e^(-W/kT) of the largest weight, so single precision is ample for them
  float non_f = 0.f;
  const float ikT = a.ikT;
  double *expo = (a.export_E && pair == 0) ? a.export_E + (long long)s0 * nP : nullptr;
  if (Mf < CUDART_INF_F) {
    for (int b0 = warp * 32; b0 < nP; b0 += blockDim.x) {
      const int idx = b0 + lane;
      const float e = idx < nP ? E[idx] : CUDART_INF_F;
      const bool fin = e < CUDART_INF_F;
      const bool cand = fin && e <= Tf;
      if (fin && !cand) non_f += __expf(-(e - Mf) * ikT);
      if (expo && idx < nP && !cand) expo[idx] = fin ? (double)e : CUDART_INF;
      unsigned bal = __ballot_sync(0xffffffffu, cand);
      while (bal) {
        const int src = __ffs(bal) - 1;
        bal &= bal - 1;
        const int ci = b0 + src;
        const int s2 = ci % a.S2, s1 = ci / a.S2;
        const double m0 = inf.w0[0] + s0, m1 = inf.w0[1] + s1, m2 = inf.w0[2] + s2;
        double part = 0.0;
        for (int i = lane; i < n; i += 32) {
          const double px = s_g[0][i] + m0, py = s_g[1][i] + m1, pz = s_g[2][i] + m2;
          for (int c = 0; c < 3; ++c)
            part += s_gam[c][i] *
                    trilinear64(t.grid + (long long)c * t.N0 * t.N1 * t.N2, t.N0, t.N1, t.N2, px, py, pz);
        }
        const double ex = warp_sum_d(part);
        const double v = -ex / kT;
        if (v > mx) {
          sm = sm * exp(mx - v) + 1.0;
          mx = v;
        } else {
          sm += exp(v - mx);
        }
        if (expo && lane == 0) expo[ci] = ex;
      }
    }
  }
  // CTA: combine the warps' exact sums and the threads' FP32 remainders into
  // this plane's LSE partial {level hi, level lo, sum relative to the level}
  for (int o = 16; o > 0; o >>= 1) non_f += __shfl_xor_sync(0xffffffffu, non_f, o);
  const float non = non_f;
  if (lane == 0) {
    s_mx[warp] = mx;
    s_sm[warp] = sm;
    s_non[warp] = non;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double MX = -CUDART_INF;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) MX = fmax(MX, s_mx[w]);
    double S = 0.0, NON = 0.0;  // (NON summed in order from FP32 warp sums)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (s_mx[w] > -CUDART_INF) S += s_mx[w] == MX ? s_sm[w] : s_sm[w] * exp(s_mx[w] - MX);
      NON += s_non[w];
    }
    if (!(MX > -CUDART_INF) && NON > 0.0) {  // no candidate here: level of the FP32 minimum
      MX = -M / kT;
      S = NON;
    } else if (MX > -CUDART_INF && NON > 0.0) {
      S += NON * exp(-M / kT - MX);
    }
    const float hi = (float)MX;
    a.part[blockIdx.x] = MX > -CUDART_INF ? make_float4(hi, (float)(MX - (double)hi), (float)S, 0.f)
                                          : make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
  }
}

// The window W + 2B of every receptor of a batch (one thread each): the FP32
// correlation error bound B = 8 eps sqrt(log2 P^3) sum_t rms(G_t) ||gamma_t||
// and W = kT max(20, ln(1e5 n)), n = S0 S1 S2 translations.
__global__ void k_window(const RefTab *tabs, int K, double g0, double g1, double g2, double log2P3, double kT,
                         double nS, double *window) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= K) return;
  const RefTab t = tabs[k];
  const double vol = t.vol;
  const double B = 8.0 * 5.9604644775390625e-08 * sqrt(log2P3) *
                   (sqrt(t.sumsq[0] / vol) * g0 + sqrt(t.sumsq[1] / vol) * g1 + sqrt(t.sumsq[2] / vol) * g2);
  window[k] = kT * fmax(20.0, log(1e5 * nS)) + 2.0 * B;
}

// Per (configuration, receptor): the FP32 minimum over its planes and the
// threshold, that minimum plus the receptor's window, rounded up to FP32.
__global__ void k_threshold(const float *plane_min, int n_pairs, int S0, int K, const double *window, float *pmin_pair,
                            float *thresh) {
  const int pr = blockIdx.x * blockDim.x + threadIdx.x;
  if (pr >= n_pairs) return;
  float mn = CUDART_INF_F;
  for (int q = 0; q < S0; ++q) mn = fminf(mn, plane_min[(long long)pr * S0 + q]);
  pmin_pair[pr] = mn;
  thresh[pr] = mn < CUDART_INF_F ? __double2float_ru((double)mn + window[pr % K]) : -CUDART_INF_F;
}

cudaError_t launch_refine(const RefineArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  k_window<<<(a.K + 127) / 128, 128, 0, st>>>(a.tabs, a.K, a.gnorm[0], a.gnorm[1], a.gnorm[2], a.log2P3, a.kT,
                                              (double)a.S0 * a.S1 * a.S2, a.window);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int n_pairs = batch * a.K;
  k_threshold<<<(n_pairs + 127) / 128, 128, 0, st>>>(a.plane_min, n_pairs, a.S0, a.K, a.window, a.pmin_pair,
                                                     a.thresh);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_refine<<<(unsigned)((long long)batch * a.K * a.S0), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// gamma_t,i in FP64 (Eqs. electrostatic, repulsive_LJ, attractive_LJ): q,
// sqrt(eps) R^p_rep, sqrt(eps) R^p_att.
__global__ void k_gamma64(const float *q, const float *eps, const float *R, int n, int p_rep, int p_att,
                          double *g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double se = sqrt((double)eps[i]), r = (double)R[i];
  double rr = 1.0, ra = 1.0;
  for (int p = 0; p < p_rep; ++p) rr *= r;
  for (int p = 0; p < p_att; ++p) ra *= r;
  g[i] = (double)q[i];
  g[(long long)n + i] = se * rr;
  g[2ll * n + i] = se * ra;
}

cudaError_t launch_gamma64(const float *q, const float *eps, const float *R, int n, int p_rep, int p_att, double *g,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gamma64<<<(n + 127) / 128, 128, 0, st>>>(q, eps, R, n, p_rep, p_att, g);
  return cudaGetLastError();
}

// Sum of squares of each of the three grids (FP64), for the FP32 error bound.
__global__ void k_sumsq(const float *g, long long vol, double *out) {
  __shared__ double s_d[256];
  const int c = blockIdx.y;
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < vol; i += (long long)gridDim.x * blockDim.x) {
    const double v = g[(long long)c * vol + i];
    acc += v * v;
  }
  s_d[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out + c, s_d[0]);
}

cudaError_t launch_sumsq(const float *g, long long vol, double *out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(double), st);
  if (e != cudaSuccess) return e;
  k_sumsq<<<dim3(sm_count(), 3), 256, 0, st>>>(g, vol, out);
  return cudaGetLastError();
}

}  // namespace bpmf
