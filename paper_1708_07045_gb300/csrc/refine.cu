// Refined form (BPMF_MODE_REFINE): the FP32 correlation gives every
// translation's energy with an error that stays below a bound B
// (8 eps32 sqrt(log2 P^3) sum_t rms(G_t) ||gamma_t||, the typical roundoff
// growth of an FFT correlation); only translations whose FP32 energy lies
// within W + 2B of the configuration's FP32 minimum can carry a weight above
// e^(-W/kT) of the largest, so only they are re-evaluated exactly: the direct
// sum the FFT correlation equals (trilinear interpolation of each receptor
// grid at every atom, Eqs. general_form / receptor_grid / correlation_func),
// in float-pair arithmetic built from FP32 instructions (about 2^-44
// relative).  The window W = kT max(20, ln(1e5 n)) (n translations in the
// site window) keeps the weight of all the other translations below 1e-5 of
// S together (at most 6e-6 kcal/mol on kT log Z); they are left out.
//
// Per batch:
//   k_refine_init  -- W + 2B and B per receptor; reset each pair's running
//                     minimum (or, in a second pass, set it to the first
//                     pass's final minimum) and candidate count;
//   k_zinv         -- (kernels.cu) each plane lowers its pair's running
//                     minimum and appends the translations within W + 2B of
//                     it to the pair's list (a superset of those within
//                     W + 2B of the final minimum); it writes no partial;
//   k_refine       -- one CTA per pair: the final threshold from the final
//                     minimum; every listed translation below it is
//                     re-evaluated exactly (a warp per translation, lanes
//                     over atoms) and checked against its FP32 energy
//                     (|E_fp32 - E_exact| <= B, the certificate); their
//                     weights, summed in order-independent fixed point, are
//                     the pair's partial in the merge.
// The set below the final threshold does not depend on the order in which
// the planes ran, so results are the same on every run.  A failed check sets
// a flag that makes bpmf_eval recompute the ligand in float pairs; an
// overflowing list, one that makes it run the ligand again from the stored
// minima.
#include <cuda_runtime.h>

#include <algorithm>
#include <math_constants.h>

#include "kernels.cuh"

namespace bpmf {

// W + 2B and B of every receptor, and the per-pair reset (one thread each).
__global__ void k_refine_init(RefineArgs a, int n_pairs, float nS) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_pairs) {
    // a second pass starts from the first pass's minimum: an FP32 energy of a
    // valid translation, so at least E_min - B, and the lists hold no more
    // than the final window (plus what lower FP32 values add)
    a.rs.pmin[i] = (a.seeded && a.store) ? a.store[a.order[i / a.K] * a.Kall + a.kmap[i % a.K]] : f2ord(CUDART_INF_F);
    a.rs.cnt[i] = 0;
    a.rs.lvl[i] = 0ull;  // below every key
    a.rs.wsum[i] = 0ull;
    a.rs.done[i] = 0u;
  }
  if (i < a.K) {
    const RefTab t = a.tabs[i];
    const float B = a.bound_scale * 8.f * 5.9604644775390625e-08f * sqrtf(a.log2P3) *
                    (sqrtf(t.sumsq[0] / t.vol) * a.gnorm[0] + sqrtf(t.sumsq[1] / t.vol) * a.gnorm[1] +
                     sqrtf(t.sumsq[2] / t.vol) * a.gnorm[2]);
    a.win[i] = a.kT * fmaxf(20.f, logf(1e5f * nS)) + 2.f * B;
    a.bnd[i] = B * a.check_scale;
  }
}

cudaError_t launch_refine_init(const RefineArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const int n_pairs = batch * a.K;
  const int n = n_pairs > a.K ? n_pairs : a.K;
  k_refine_init<<<(n + 127) / 128, 128, 0, st>>>(a, n_pairs, (float)a.S0 * a.S1 * a.S2);
  return cudaGetLastError();
}

__device__ __forceinline__ ff lerp_ff(ff a, ff b, ff w0, ff w1) { return s_add(s_mul(a, w0), s_mul(b, w1)); }

// Float-pair trilinear interpolation of one FP32 grid: cell (cx, cy, cz),
// fractions f (weights 1 - f, f per axis), as nested linear interpolations
// along z, then y, then x.
__device__ __forceinline__ ff trilinear_ff(const float *g, long long sx, long long sy, const ff w[3][2]) {
  const ff c00 = s_norm(lerp_ff(ff{g[0], 0.f}, ff{g[1], 0.f}, w[2][0], w[2][1]));
  const ff c01 = s_norm(lerp_ff(ff{g[sy], 0.f}, ff{g[sy + 1], 0.f}, w[2][0], w[2][1]));
  const ff c10 = s_norm(lerp_ff(ff{g[sx], 0.f}, ff{g[sx + 1], 0.f}, w[2][0], w[2][1]));
  const ff c11 = s_norm(lerp_ff(ff{g[sx + sy], 0.f}, ff{g[sx + sy + 1], 0.f}, w[2][0], w[2][1]));
  const ff c0 = s_norm(lerp_ff(c00, c01, w[1][0], w[1][1]));
  const ff c1 = s_norm(lerp_ff(c10, c11, w[1][0], w[1][1]));
  return s_norm(lerp_ff(c0, c1, w[0][0], w[0][1]));
}

__device__ __forceinline__ float d_ff(ff a, ff b) {  // a - b, rounded to FP32
  return __fadd_rn(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

// Weights are summed in 64-bit fixed point (scale 2^40 relative to the
// pair's level, every weight <= 1): integer adds are exact and
// order-independent, so the result does not depend on the order in which
// k_zinv appended the translations nor on how the list is split among CTAs.
constexpr double kFixScale = 1099511627776.0;  // 2^40 (lists of up to 2^23 translations: sums < 2^63)

// Ordered 64-bit key of a normalised float pair (hi, then lo): a larger value,
// a larger key, so atomicMax on keys keeps the largest pair.
__device__ __forceinline__ unsigned long long ff_key(ff x) {
  return ((unsigned long long)f2ord(x.hi) << 32) | (unsigned long long)f2ord(x.lo);
}
__device__ __forceinline__ ff key_ff(unsigned long long k) {
  return ff{ord2f((unsigned)(k >> 32)), ord2f((unsigned)(k & 0xffffffffull))};
}

// Pass 1, CTA c of gridDim.y per pair (blockIdx.x = pair): the exact -E/kT of
// every listed translation below the final threshold in its share of the
// list (a warp per translation, lanes over atoms), the certificate check, and
// the largest exact value into the pair's level.
__global__ void __launch_bounds__(256) k_refine(RefineArgs a) {
  __shared__ ff s_g[3][256];    // atom positions in the ligand-box frame (grid units)
  __shared__ ff s_gam[3][256];  // gamma_t,i
  __shared__ unsigned long long s_key;
  const int pair = blockIdx.x;  // j * K + k
  const int j = pair / a.K, k = pair % a.K;
  const int n_list = min(a.rs.cnt[pair], a.rs.cap);
  if (threadIdx.x == 0) {
    s_key = 0ull;
    if (blockIdx.y == 0) {
      if (a.rs.cnt[pair] > a.rs.cap) atomicOr(a.rs.fail, 2);  // list overflow (bit 1)
      if (a.store) a.store[a.order[j] * a.Kall + a.kmap[k]] = a.rs.pmin[pair];
    }
  }
  const float Emin = ord2f(a.rs.pmin[pair]);
  // the final threshold (k_zinv listed against thresholds at least as high)
  const float T = __fadd_ru(Emin, a.rs.win[k]);
  const float B = a.rs.bnd[k];
  const ConfMeta m = a.meta[j];
  const PairInfo inf = a.info[pair];
  const RefTab tb = a.tabs[k];
  const int n = m.n_atoms;
  const ff h{a.h_hi, a.h_lo};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int d = 0; d < 3; ++d) s_g[d][i] = place_ff(a.coords[3ll * (m.atom_off + i) + d], m.lo[d], h);
    for (int c = 0; c < 3; ++c) {
      const float2 g = a.gamma[(long long)c * a.gamma_stride + m.gamma_off + i];
      s_gam[c][i] = ff{g.x, g.y};
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const ff nikT{a.nikT_hi, a.nikT_lo};
  const long long vol = (long long)tb.N0 * tb.N1 * tb.N2;
  const long long sx = (long long)tb.N1 * tb.N2, sy = tb.N2;
  const Cand *list = a.rs.cand + (long long)pair * a.rs.cap;
  float2 *ex = a.rs.exact + (long long)pair * a.rs.cap;
  double *expo = (a.export_E && pair == 0) ? a.export_E : nullptr;
  ff Xe{-CUDART_INF_F, 0.f};  // max exact
  bool bad = false;
  const int step = (int)gridDim.y * nwarp * 32;
  for (int b0 = ((int)blockIdx.y * nwarp + warp) * 32; b0 < n_list; b0 += step) {
    const int idx = b0 + lane;
    Cand cd{0u, CUDART_INF_F};
    if (idx < n_list) cd = list[idx];
    const bool cand = idx < n_list && cd.e <= T;
    unsigned bal = __ballot_sync(0xffffffffu, cand);
    while (bal) {
      const int src = __ffs(bal) - 1;
      bal &= bal - 1;
      const unsigned t = __shfl_sync(0xffffffffu, cd.t, src);
      const float ef = __shfl_sync(0xffffffffu, cd.e, src);

      const int s2 = (int)(t % (unsigned)a.S2), s01 = (int)(t / (unsigned)a.S2);
      const int s1 = s01 % a.S1, s0 = s01 / a.S1;
      const int mt[3] = {inf.w0[0] + s0, inf.w0[1] + s1, inf.w0[2] + s2};
      ff part{0.f, 0.f};
      for (int i = lane; i < n; i += 32) {
        int c[3];
        ff w[3][2];
        for (int d = 0; d < 3; ++d) {
          const ff p = s_norm(s_add(s_g[d][i], ff{(float)mt[d], 0.f}));
          ff f;
          cell_ff(p, c[d], f);
          const int Nd = d == 0 ? tb.N0 : (d == 1 ? tb.N1 : tb.N2);
          if (c[d] > Nd - 2) {  // a position on the last node uses the cell below it
            f = s_norm(s_add(f, ff{(float)(c[d] - (Nd - 2)), 0.f}));
            c[d] = Nd - 2;
          }
          if (c[d] < 0) {
            f = s_norm(s_add(f, ff{(float)c[d], 0.f}));
            c[d] = 0;
          }
          w[d][0] = s_norm(s_sub(ff{1.f, 0.f}, f));
          w[d][1] = f;
        }
        const float *g0 = tb.grid + c[0] * sx + c[1] * sy + c[2];
        for (int ch = 0; ch < 3; ++ch)
          part = s_norm(s_add(part, s_mul(s_gam[ch][i], trilinear_ff(g0 + ch * vol, sx, sy, w))));
      }
      for (int o = 16; o > 0; o >>= 1) {
        const ff other{__shfl_xor_sync(0xffffffffu, part.hi, o), __shfl_xor_sync(0xffffffffu, part.lo, o)};
        part = s_norm(s_add(part, other));
      }
      // the certificate: the FP32 energy lies within B of the exact one
      if (fabsf(d_ff(ff{ef, 0.f}, part)) > B) bad = true;
      const ff x = s_norm(s_mul(part, nikT));
      if (ff_gt(x, Xe)) Xe = x;
      if (lane == src) {
        ex[idx] = make_float2(x.hi, x.lo);
        if (expo) expo[t] = (double)part.hi + (double)part.lo;
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(a.rs.fail, 1);  // certificate (bit 0)
  for (int o = 16; o > 0; o >>= 1) {
    const ff o2{__shfl_xor_sync(0xffffffffu, Xe.hi, o), __shfl_xor_sync(0xffffffffu, Xe.lo, o)};
    if (ff_gt(o2, Xe)) Xe = o2;
  }
  if (lane == 0 && Xe.hi > -CUDART_INF_F) atomicMax(&s_key, ff_key(Xe));
  __syncthreads();
  if (gridDim.y > 1) {  // the level over every CTA of the pair; k_refine_sum sums
    if (threadIdx.x == 0 && s_key) atomicMax(&a.rs.lvl[pair], s_key);
    return;
  }
  // one CTA per pair: it holds the level already and sums the weights itself
  // (the same fixed-point sum k_refine_sum forms)
  const unsigned long long key = s_key;
  if (!key) {  // no translation below the threshold (no valid translation)
    if (threadIdx.x == 0) {
      a.part_ref[2 * pair] = make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
      a.part_ref[2 * pair + 1] = make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
    }
    return;
  }
  __shared__ unsigned long long s_we;
  if (threadIdx.x == 0) s_we = 0ull;
  __syncthreads();
  const ff L = key_ff(key);
  unsigned long long wt = 0ull;
  for (int idx = threadIdx.x; idx < n_list; idx += blockDim.x)
    if (list[idx].e <= T) {
      const float2 xe = ex[idx];
      wt += (unsigned long long)__double2ll_rn((double)expf(d_ff(ff{xe.x, xe.y}, L)) * kFixScale);
    }
  if (wt) atomicAdd(&s_we, wt);
  __syncthreads();
  if (threadIdx.x == 0) {
    const double sw = (double)s_we / kFixScale;  // exact to double rounding
    const float sw_hi = (float)sw;
    a.part_ref[2 * pair] = make_float4(L.hi, L.lo, sw_hi, (float)(sw - (double)sw_hi));
    a.part_ref[2 * pair + 1] = make_float4(L.hi, L.lo, 0.f, 0.f);
  }
}

// Pass 2, the same CTAs: the weight exp(x - L) of every re-evaluated
// translation in the CTA's share, in fixed point relative to the pair's level
// L, added to the pair's sum; the last CTA of the pair writes its partial
// {L, sum} for the merge (none when nothing lies below the threshold).
__global__ void __launch_bounds__(256) k_refine_sum(RefineArgs a) {
  __shared__ unsigned long long s_we;
  __shared__ bool s_last;
  const int pair = blockIdx.x;
  const int k = pair % a.K;
  const int n_list = min(a.rs.cnt[pair], a.rs.cap);
  const unsigned long long key = a.rs.lvl[pair];
  const float T = __fadd_ru(ord2f(a.rs.pmin[pair]), a.rs.win[k]);
  if (threadIdx.x == 0) s_we = 0ull;
  __syncthreads();
  const Cand *list = a.rs.cand + (long long)pair * a.rs.cap;
  const float2 *ex = a.rs.exact + (long long)pair * a.rs.cap;
  unsigned long long wt = 0ull;
  if (key) {
    const ff L = key_ff(key);  // the largest exact value: every weight <= 1
    const int step = (int)(gridDim.y * blockDim.x);
    for (int idx = (int)(blockIdx.y * blockDim.x + threadIdx.x); idx < n_list; idx += step)
      if (list[idx].e <= T) {
        const float2 xe = ex[idx];
        wt += (unsigned long long)__double2ll_rn((double)expf(d_ff(ff{xe.x, xe.y}, L)) * kFixScale);
      }
  }
  if (wt) atomicAdd(&s_we, wt);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (s_we) atomicAdd(&a.rs.wsum[pair], s_we);
    __threadfence();
    s_last = atomicAdd(&a.rs.done[pair], 1u) == gridDim.y - 1;
  }
  __syncthreads();
  if (s_last && threadIdx.x == 0) {
    __threadfence();
    if (!key) {  // no translation below the threshold (no valid translation)
      a.part_ref[2 * pair] = make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
      a.part_ref[2 * pair + 1] = make_float4(-CUDART_INF_F, 0.f, 0.f, 0.f);
      return;
    }
    const ff L = key_ff(key);
    const double sw = (double)atomicAdd(&a.rs.wsum[pair], 0ull) / kFixScale;  // exact to double rounding
    const float sw_hi = (float)sw;
    a.part_ref[2 * pair] = make_float4(L.hi, L.lo, sw_hi, (float)(sw - (double)sw_hi));
    a.part_ref[2 * pair + 1] = make_float4(L.hi, L.lo, 0.f, 0.f);
  }
}

// CTAs per pair: one (and one kernel) when the pairs fill the SMs; else
// enough to cover the GPU twice over, at most 64 per pair (long lists on few
// pairs, e.g. one wide site window), and k_refine_sum as the second pass.
cudaError_t launch_refine(const RefineArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  const long long pairs = (long long)batch * a.K;
  const int n_sm = sm_count();
  const int C = pairs >= n_sm ? 1 : (int)std::min<long long>(64, (2ll * n_sm + pairs - 1) / pairs);
  const dim3 grid((unsigned)pairs, (unsigned)C);
  k_refine<<<grid, 256, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || C == 1) return e;
  k_refine_sum<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}


}  // namespace bpmf
