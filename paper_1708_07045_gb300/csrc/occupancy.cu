// Steric clashes (Eq. occupancy_grid): a translation clashes when an occupied
// node of the ligand occupancy grid lands on an occupied node of the receptor
// occupancy grid, i.e. when the correlation of the two grids is positive.
//
// The grids are binary, so the correlation's sign is computed exactly with bit
// operations instead of a fourth FFT channel:
//   * the receptor grid becomes bit rows along z with one dilation per run
//     length, D_v(z) = OR_{t <= v} occ(z + t), v < 32 (k_occ_table, once per
//     receptor);
//   * each configuration's occupied ligand nodes become runs of at most 32
//     nodes along z (k_occ_runs);
//   * for 32 translations along z at once, a run of length v + 1 hits where
//     the level-v row it lands on has a set bit: one funnel shift (k_clash).
// Node occupancy of the ligand is decided in IEEE single precision, each
// operation rounded in a fixed order (position, threshold, squared distance),
// so that it is a function of the FP32 inputs alone.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cstdint>

#include "kernels.cuh"

namespace bpmf {

// 2^(-1/3): squared ratio of the occupancy radius 2^(-1/6) R to R
#define OCC_R2_SCALE 0.79370052598409973737585281963615f

// ---------------------------------------------------------------- receptor
__global__ void k_occ_table(const unsigned char *occ, int N0, int N1, int N2, int W, uint32_t *tab) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)N0 * N1) return;
  const int X = (int)(t / N1), Y = (int)(t % N1);
  const int Q0 = N0 + 2 * kOccXYPad, Q1 = N1 + 2 * kOccXYPad;
  const unsigned char *row = occ + ((long long)X * N1 + Y) * N2;
  const long long lvs = (long long)Q0 * W * Q1;  // level stride
  uint32_t *base = tab + (long long)(X + kOccXYPad) * W * Q1 + (Y + kOccXYPad);
  // level 0: the bits themselves
  for (int w = 0; w < W; ++w) {
    uint32_t v = 0;
    for (int b = 0; b < 32; ++b) {
      const int z = 32 * w + b - kOccZPad;
      if (z >= 0 && z < N2 && row[z]) v |= 1u << b;
    }
    base[(long long)w * Q1] = v;
  }
  // level v from level v-1: D_v(z) = D_{v-1}(z) | occ(z + v)
  const uint32_t *raw = base;
  for (int lv = 1; lv < kOccLevels; ++lv) {
    const uint32_t *src = base + (lv - 1) * lvs;
    uint32_t *dst = base + lv * lvs;
    for (int w = 0; w < W; ++w) {
      const uint32_t r0 = raw[(long long)w * Q1], r1 = (w + 1 < W) ? raw[(long long)(w + 1) * Q1] : 0u;
      dst[(long long)w * Q1] = src[(long long)w * Q1] | __funnelshift_r(r0, r1, lv);
    }
  }
}

cudaError_t launch_occ_table(const unsigned char *occ, int N0, int N1, int N2, int W, uint32_t *tab,
                             cudaStream_t st) {
  const long long n = (long long)N0 * N1;
  if (n <= 0) return cudaSuccess;
  const size_t words = (size_t)kOccLevels * (N0 + 2 * kOccXYPad) * W * (N1 + 2 * kOccXYPad);
  cudaError_t e = cudaMemsetAsync(tab, 0, words * sizeof(uint32_t), st);  // zero margins
  if (e != cudaSuccess) return e;
  k_occ_table<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(occ, N0, N1, N2, W, tab);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ ligand
constexpr int kRowIntervals = 192;  // disjoint z intervals one row can hold (>= ceil(extent / 2))

__device__ __forceinline__ bool node_occupied(float s2, float pz, float thr, int c) {
  const float dz = __fsub_rn((float)c, pz);
  return __fadd_rn(s2, __fmul_rn(dz, dz)) < thr;
}

// rb CTAs per configuration: atom positions in the ligand-box frame, then,
// for each CTA's share of the (a, b) rows, the occupied-node intervals of a
// row, merged and split into runs of at most 32 nodes.
__global__ void __launch_bounds__(256) k_occ_runs(OccRunsArgs a) {
  __shared__ float s_p[3][256], s_thr[256];
  __shared__ float s_red[4][8];
  __shared__ int s_cnt[8];
  __shared__ int s_base;
  const int cfg = blockIdx.x / a.rb, part = blockIdx.x % a.rb;
  const ConfMeta m = a.meta[cfg];
  const int n = m.n_atoms;
  const int tid = threadIdx.x;
  float pmin[3] = {CUDART_INF_F, CUDART_INF_F, CUDART_INF_F}, pmax[3] = {-CUDART_INF_F, -CUDART_INF_F,
                                                                          -CUDART_INF_F};
  float rmax = 0.f;
  for (int i = tid; i < n; i += blockDim.x) {
    const float *x = a.coords + 3ll * (m.atom_off + i);
    for (int d = 0; d < 3; ++d) {
      const float p = __fadd_rn(__fdiv_rn(__fsub_rn(x[d], m.lo[d]), a.h), 2.0f);
      s_p[d][i] = p;
      pmin[d] = fminf(pmin[d], p);
      pmax[d] = fmaxf(pmax[d], p);
    }
    const float r = __fdiv_rn(a.R[m.gamma_off + i], a.h);
    s_thr[i] = __fmul_rn(__fmul_rn(r, r), OCC_R2_SCALE);
    rmax = fmaxf(rmax, fabsf(r));
  }
  // block reductions of the position range and the largest radius
  for (int o = 16; o > 0; o >>= 1) {
    for (int d = 0; d < 3; ++d) {
      pmin[d] = fminf(pmin[d], __shfl_xor_sync(0xffffffffu, pmin[d], o));
      pmax[d] = fmaxf(pmax[d], __shfl_xor_sync(0xffffffffu, pmax[d], o));
    }
    rmax = fmaxf(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
  }
  if ((tid & 31) == 0) {
    for (int d = 0; d < 3; ++d) {
      s_red[d][tid >> 5] = pmin[d];
    }
    s_red[3][tid >> 5] = rmax;
  }
  __syncthreads();
  float lo3[3], hi3[3], R0 = 0.f;
  for (int d = 0; d < 3; ++d) lo3[d] = CUDART_INF_F;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
    for (int d = 0; d < 3; ++d) lo3[d] = fminf(lo3[d], s_red[d][w]);
    R0 = fmaxf(R0, s_red[3][w]);
  }
  __syncthreads();
  if ((tid & 31) == 0)
    for (int d = 0; d < 3; ++d) s_red[d][tid >> 5] = pmax[d];
  __syncthreads();
  for (int d = 0; d < 3; ++d) {
    hi3[d] = -CUDART_INF_F;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) hi3[d] = fmaxf(hi3[d], s_red[d][w]);
  }
  int alo = (int)floorf(lo3[0] - R0) - 1, ahi = (int)ceilf(hi3[0] + R0) + 1;
  int blo = (int)floorf(lo3[1] - R0) - 1, bhi = (int)ceilf(hi3[1] + R0) + 1;
  // a row holds at most ceil(nC / 2) disjoint intervals; a longer z extent
  // belongs to a box no receptor grid of at most 256 nodes admits (no valid
  // translation), and such a configuration gets no runs
  bool sane = n > 0 && R0 < 1e4f;
  for (int d = 0; d < 3; ++d) sane = sane && fabsf(lo3[d]) < 1e6f && fabsf(hi3[d]) < 1e6f;
  if (!sane) {
    alo = blo = 0;
    ahi = bhi = -1;
  }
  const int clo = sane ? (int)floorf(lo3[2] - R0) - 1 : 0, chi = sane ? (int)ceilf(hi3[2] + R0) + 1 : -1;
  const int nC = chi - clo + 1;
  const int nA = ahi - alo + 1, nB = bhi - blo + 1;
  // (sane bounds keep nA, nB below 2e6 + 2e4; rows beyond 2^31 do not occur
  // for boxes a receptor grid of at most 256 nodes admits)
  const long long rows_ll = (nA > 0 && nB > 0 && nC <= 2 * kRowIntervals) ? (long long)nA * nB : 0;
  const long long rows = rows_ll < (1ll << 30) ? rows_ll : 0;
  OccRun *out = a.runs + (long long)cfg * 2 * a.cap;
  // this CTA's share of the rows; its runs go to space reserved with an
  // atomic add per chunk (the order of chunks across CTAs is free: the clash
  // flags are an OR over runs, and k_occ_sort orders runs by length)
  const int rpp = (int)((rows + a.rb - 1) / a.rb);
  const int row_lo = part * rpp, row_hi = min((int)rows, row_lo + rpp);
  short iv_lo[kRowIntervals], iv_hi[kRowIntervals];
  for (int r0 = row_lo; r0 < row_hi; r0 += blockDim.x) {
    const int row = r0 + tid;
    int nI = 0;
    int ra = 0, rb = 0;
    if (row < row_hi) {
      ra = alo + row / nB;
      rb = blo + row % nB;
      for (int i = 0; i < n; ++i) {
        const float dx = __fsub_rn((float)ra, s_p[0][i]), dy = __fsub_rn((float)rb, s_p[1][i]);
        const float s2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        const float thr = s_thr[i];
        if (!(s2 < thr)) continue;
        const float pz = s_p[2][i];
        // the occupied nodes of one atom in a row form an interval around
        // the node nearest p_z (the rounded squared distance is monotone in
        // |c - p_z|)
        const int cn = (int)rintf(pz);
        if (!node_occupied(s2, pz, thr, cn)) continue;
        int c0 = cn, c1 = cn;
        while (c0 > clo && node_occupied(s2, pz, thr, c0 - 1)) --c0;
        while (c1 < chi && node_occupied(s2, pz, thr, c1 + 1)) ++c1;
        // insert [c0, c1] into the sorted list of disjoint intervals, merging
        // overlapping or adjacent ones
        int k = 0;
        while (k < nI && iv_hi[k] < c0 - 1) ++k;
        int e = k;
        while (e < nI && iv_lo[e] <= c1 + 1) {
          c0 = min(c0, (int)iv_lo[e]);
          c1 = max(c1, (int)iv_hi[e]);
          ++e;
        }
        const int removed = e - k;
        if (removed == 0) {
          if (nI < kRowIntervals) {
            for (int t = nI; t > k; --t) {
              iv_lo[t] = iv_lo[t - 1];
              iv_hi[t] = iv_hi[t - 1];
            }
            ++nI;
          }
        } else if (removed > 1) {
          for (int t = k + 1; t + removed - 1 < nI; ++t) {
            iv_lo[t] = iv_lo[t + removed - 1];
            iv_hi[t] = iv_hi[t + removed - 1];
          }
          nI -= removed - 1;
        }
        iv_lo[k] = (short)c0;
        iv_hi[k] = (short)c1;
      }
    }
    // runs of at most 32 nodes
    int cnt = 0;
    for (int k = 0; k < nI; ++k) cnt += (iv_hi[k] - iv_lo[k] + kOccLevels) / kOccLevels;
    // exclusive prefix within the chunk: within the warp by shuffles, then
    // over the warp totals; one atomic add reserves the chunk's space
    const int lane = tid & 31, warp = tid >> 5;
    int incl = cnt;
    for (int d = 1; d < 32; d <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) s_cnt[warp] = incl;
    __syncthreads();
    int o = incl - cnt;
    for (int w = 0; w < warp; ++w) o += s_cnt[w];
    if (tid == blockDim.x - 1) s_base = atomicAdd(a.n_runs + cfg, o + cnt);
    __syncthreads();
    o += s_base;
    for (int k = 0; k < nI; ++k) {
      for (int c = iv_lo[k]; c <= iv_hi[k]; c += kOccLevels) {
        const int len = min(kOccLevels, iv_hi[k] - c + 1);
        if (o < a.cap) {
          OccRun rr;
          rr.a = (short)ra;
          rr.b = (short)rb;
          rr.c0 = (short)c;
          rr.dc = 0;
          rr.lv = (unsigned char)(len - 1);
          out[o] = rr;
        }
        ++o;
      }
    }
    __syncthreads();
  }
}

// One CTA per configuration: stable partition of its runs by length, longest
// first, into the second half of its buffer, so that the clash test meets
// long runs (the ones likeliest to hit) first and walks neighbouring rows of
// one table.  Warp w owns the lengths lv = w, w + 16: it counts them with
// ballots over the run list, then writes each length's runs in order.
__global__ void __launch_bounds__(512) k_occ_sort(OccRunsArgs a) {
  __shared__ int s_len[kOccLevels];
  const int tid = threadIdx.x;
  const OccRun *out = a.runs + (long long)blockIdx.x * 2 * a.cap;
  OccRun *sorted = a.runs + (long long)blockIdx.x * 2 * a.cap + a.cap;
  const int nr = min(a.n_runs[blockIdx.x], a.cap);
  const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int lv = warp; lv < kOccLevels; lv += nw) {
    int c = 0;
    for (int r0 = 0; r0 < nr; r0 += 32) {
      const int r = r0 + lane;
      c += __popc(__ballot_sync(0xffffffffu, r < nr && out[r].lv == lv));
    }
    if (lane == 0) s_len[lv] = c;
  }
  __syncthreads();
  if (tid == 0) {  // longest first
    int c = 0;
    for (int lv = kOccLevels - 1; lv >= 0; --lv) {
      const int n = s_len[lv];
      s_len[lv] = c;
      c += n;
    }
  }
  __syncthreads();
  for (int lv = warp; lv < kOccLevels; lv += nw) {
    int o = s_len[lv];
    for (int r0 = 0; r0 < nr; r0 += 32) {
      const int r = r0 + lane;
      OccRun rr;
      const bool mt = r < nr && (rr = out[r]).lv == lv;
      const unsigned bal = __ballot_sync(0xffffffffu, mt);
      if (mt) sorted[o + __popc(bal & ((1u << lane) - 1u))] = rr;
      o += __popc(bal);
    }
  }
  __syncthreads();
  if (tid == 0) a.n_runs[blockIdx.x] = nr;
}

cudaError_t launch_occ_runs(const OccRunsArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(a.n_runs, 0, sizeof(int) * batch, st);
  if (e != cudaSuccess) return e;
  k_occ_runs<<<batch * a.rb, 256, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_occ_sort<<<batch, 512, 0, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- clash
__device__ __forceinline__ uint32_t occ_word(const uint32_t *row, int w, int W, int N1) {
  return (w >= 0 && w < W) ? __ldg(row + (long long)w * N1) : 0u;
}

// One CTA per (configuration, receptor, tile of T0 x T1 translations in
// (s0, s1)); every thread owns one (s0, s1) and the flags of all s2 in
// 64-translation groups (two 32-bit words).  Runs come sorted by length (see
// k_occ_runs), so consecutive runs read neighbouring rows of one table (the
// L1 serves them); a warp stops once every flag of its lanes is set.  Each
// chunk of runs is first turned into table-word offsets and shift amounts
// shared by the whole CTA; when every row and word the CTA can touch lies in
// the table, the inner loop needs no bounds checks.
constexpr int kClashChunk = 2048;

__global__ void __launch_bounds__(256) k_clash(ClashArgs a) {
  __shared__ uint2 s_ri[kClashChunk];  // {table-word offset, bit shift}
  const int n0 = (a.S0 + a.T0 - 1) / a.T0, n1 = (a.S1 + a.T1 - 1) / a.T1;
  const int tile = blockIdx.x % (n0 * n1);
  const int pair = blockIdx.x / (n0 * n1);  // j * K + k
  const int j = pair / a.K, k = pair % a.K;
  const int ty = threadIdx.x / a.T1, tx = threadIdx.x % a.T1;
  const int s0_t = (tile / n1) * a.T0, s1_t = (tile % n1) * a.T1;
  const int s0 = s0_t + ty, s1 = s1_t + tx;
  const bool active = ty < a.T0 && s0 < a.S0 && s1 < a.S1;
  const OccTab t = a.tabs[k];
  const PairInfo inf = a.info[pair];
  const bool valid = active && t.tab && s0 >= inf.sa[0] && s0 <= inf.sb[0] && s1 >= inf.sa[1] && s1 <= inf.sb[1];
  uint32_t *dst = a.clash + (((long long)pair * a.S0 + s0) * a.S1 + s1) * a.CW;
  const int nr = t.tab ? a.n_runs[j] : 0;
  const OccRun *runs = a.runs + (long long)j * 2 * a.cap + a.cap;  // level-sorted half
  const int ys = t.N1 + 2 * kOccXYPad, xs = t.W * ys, lvs = (t.N0 + 2 * kOccXYPad) * xs;  // < 2^31 words
  // translations the CTA evaluates (valid lanes only)
  const int v0lo = max(s0_t, inf.sa[0]), v0hi = min(min(s0_t + a.T0, a.S0) - 1, inf.sb[0]);
  const int v1lo = max(s1_t, inf.sa[1]), v1hi = min(min(s1_t + a.T1, a.S1) - 1, inf.sb[1]);
  const int zb0 = inf.w0[2] + kOccZPad;
  const int npairs = (a.CW + 1) / 2;
  uint32_t acc[2][4];  // up to 8 flag words (S2 <= 256)
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[0][q] = acc[1][q] = 0u;
  const uint32_t *base = t.tab + (long long)(inf.w0[0] + (valid ? s0 : v0lo) + kOccXYPad) * xs +
                         (inf.w0[1] + (valid ? s1 : v1lo) + kOccXYPad);
  for (int c0r = 0; c0r < nr && v0lo <= v0hi && v1lo <= v1hi; c0r += kClashChunk) {
    const int nc = min(kClashChunk, nr - c0r);
    __syncthreads();
    int amin = 1 << 30, namax = 1 << 30, bmin = 1 << 30, nbmax = 1 << 30, wmin = 1 << 30, nwmax = 1 << 30;
    for (int r = threadIdx.x; r < nc; r += blockDim.x) {
      const OccRun rr = runs[c0r + r];
      const int bA = zb0 + rr.c0;
      const int wA = bA >> 5;
      s_ri[r] = make_uint2((unsigned)(rr.lv * lvs + rr.a * xs + rr.b + wA * ys), (unsigned)(bA & 31));
      amin = min(amin, (int)rr.a);
      namax = min(namax, -(int)rr.a);
      bmin = min(bmin, (int)rr.b);
      nbmax = min(nbmax, -(int)rr.b);
      wmin = min(wmin, wA);
      nwmax = min(nwmax, -wA);
    }
    // CTA-wide extremes (six minima over the warps)
    int v[6] = {amin, namax, bmin, nbmax, wmin, nwmax};
#pragma unroll
    for (int q = 0; q < 6; ++q)
      for (int o = 16; o > 0; o >>= 1) v[q] = min(v[q], __shfl_xor_sync(0xffffffffu, v[q], o));
    __shared__ int s_v[6][8];
    if ((threadIdx.x & 31) == 0)
#pragma unroll
      for (int q = 0; q < 6; ++q) s_v[q][threadIdx.x >> 5] = v[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      v[q] = s_v[q][0];
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v[q] = min(v[q], s_v[q][w]);
    }
    // every row and word in the table: no checks in the loop
    const bool fast = inf.w0[0] + v0lo + v[0] >= -kOccXYPad && inf.w0[0] + v0hi - v[1] < t.N0 + kOccXYPad &&
                      inf.w0[1] + v1lo + v[2] >= -kOccXYPad && inf.w0[1] + v1hi - v[3] < t.N1 + kOccXYPad &&
                      v[4] >= 0 && -v[5] + 2 * (npairs - 1) + 2 < t.W;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g >= npairs) break;
      uint32_t a0 = acc[0][g], a1 = acc[1][g];
      const int nb0 = min(32, a.S2 - 64 * g), nb1 = min(32, a.S2 - 64 * g - 32);
      const uint32_t full0 = nb0 >= 32 ? 0xffffffffu : ((1u << nb0) - 1u);
      const uint32_t full1 = nb1 <= 0 ? 0u : (nb1 >= 32 ? 0xffffffffu : ((1u << nb1) - 1u));
      const int gofs = 2 * g * ys;
      for (int r0 = 0; r0 < nc; r0 += 16) {
        const bool done = !valid || ((a0 & full0) == full0 && (a1 & full1) == full1);
        if (__all_sync(0xffffffffu, done)) break;
        const int r1 = min(nc, r0 + 16);
        if (fast) {
          if (valid) {
            const uint32_t *bg = base + gofs;
            int r = r0;
            for (; r + 4 <= r1; r += 4) {  // four runs' loads in flight
              uint2 ri[4];
              uint32_t l[4][3];
#pragma unroll
              for (int q = 0; q < 4; ++q) ri[q] = s_ri[r + q];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                const uint32_t *p = bg + (int)ri[q].x;
                l[q][0] = __ldg(p);
                l[q][1] = __ldg(p + ys);
                l[q][2] = __ldg(p + 2 * ys);
              }
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                a0 |= __funnelshift_r(l[q][0], l[q][1], ri[q].y);
                a1 |= __funnelshift_r(l[q][1], l[q][2], ri[q].y);
              }
            }
            for (; r < r1; ++r) {
              const uint2 ri = s_ri[r];
              const uint32_t *p = bg + (int)ri.x;
              const uint32_t l0 = __ldg(p), l1 = __ldg(p + ys), l2 = __ldg(p + 2 * ys);
              a0 |= __funnelshift_r(l0, l1, ri.y);
              a1 |= __funnelshift_r(l1, l2, ri.y);
            }
          }
        } else if (valid) {
          for (int r = r0; r < r1; ++r) {
            const OccRun rr = runs[c0r + r];
            const int X = inf.w0[0] + s0 + rr.a, Y = inf.w0[1] + s1 + rr.b;
            if (X < 0 || X >= t.N0 || Y < 0 || Y >= t.N1) continue;
            const uint32_t *row = t.tab + (long long)rr.lv * lvs + (long long)(X + kOccXYPad) * xs + (Y + kOccXYPad);
            const int bA = zb0 + 64 * g + rr.c0;
            const int wA = bA >> 5, shA = bA & 31;
            const uint32_t l0 = occ_word(row, wA, t.W, ys), l1 = occ_word(row, wA + 1, t.W, ys),
                           l2 = occ_word(row, wA + 2, t.W, ys);
            a0 |= __funnelshift_r(l0, l1, shA);
            a1 |= __funnelshift_r(l1, l2, shA);
          }
        }
      }
      acc[0][g] = a0;
      acc[1][g] = a1;
    }
  }
  if (active)
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (2 * g < a.CW) dst[2 * g] = acc[0][g];
      if (2 * g + 1 < a.CW) dst[2 * g + 1] = acc[1][g];
    }
}

cudaError_t launch_clash(ClashArgs a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (a.CW > 8) return cudaErrorInvalidValue;  // flags of at most 256 translations along z per thread
  a.T1 = std::min(a.S1, 256);
  a.T0 = std::max(1, std::min(a.S0, 256 / a.T1));
  const long long tiles = (long long)((a.S0 + a.T0 - 1) / a.T0) * ((a.S1 + a.T1 - 1) / a.T1);
  k_clash<<<(unsigned)(tiles * batch * a.K), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace bpmf
