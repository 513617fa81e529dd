// Radix-32 Stockham stage as a dense tensor-core contraction (split-bf16).
//
// For every column (line l, butterfly i) the stage computes
//   y[r'] = sum_r w32^(r r') * (w_P^(r j stride) * x[i + r P/32])
// which, with complex values interleaved (k = 2r + re/im), is the real
// 64 x 64 matrix A (rows m = 2r' + c') times a 64-vector.  A and the twiddled
// data are each split into three bf16 parts (x = x_hi + x_mid + x_lo, about
// 24 significant bits) and the product is taken as the six terms of order up
// to 2^-16: A_mid x_mid + A_lo x_hi + A_hi x_lo + A_mid x_hi + A_hi x_mid +
// A_hi x_hi (smallest first), with mma.sync m16n8k16 (bf16 in, FP32
// accumulate): relative error near FP32's per stage.  A's fragments are
// precomputed on the host in mma register order
// ([dir][term 3][mtile 4][kchunk 4][lane 32] x uint4) and read through the
// read-only cache.
#pragma once
#include <cuda_bf16.h>

#include "arith.cuh"

namespace bpmf {

__device__ __forceinline__ void split_bf16(float v, float &hi, float &mid, float &lo) {
  hi = __bfloat162float(__float2bfloat16_rn(v));
  const float r = __fsub_rn(v, hi);  // exact
  mid = __bfloat162float(__float2bfloat16_rn(r));
  lo = __fsub_rn(r, mid);            // exact; rounded to bf16 when packed
}
__device__ __forceinline__ unsigned pk_bf16(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const unsigned *>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint4 &a, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a.x), "r"(a.y), "r"(a.z), "r"(a.w), "r"(b0), "r"(b1));
}

// One radix-32 stage over nlines lines (element n of line l at buf[n es + l ls]).
// Every warp of the CTA takes 8-column tiles in turn; tca points to the
// fragment table, tw to the stage twiddle table (exp(-2 pi i k / P)).
__device__ inline void tc_dft32_stage(const cx<float> *src, cx<float> *dst, int es, int ls, int nlines, int P, int Ns,
                               const float4 *tw, bool inv, const uint4 *tca) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int gid = lane >> 2, tig = lane & 3;
  const int nb = P / 32;
  const int ncol = nb * nlines;
  const int tstride = P / (Ns * 32);
  const uint4 *A = tca + (inv ? 3 * 4 * 4 * 32 : 0);  // [term][mtile][kchunk][lane]
  for (int n0 = warp * 8; n0 < ncol; n0 += nwarps * 8) {
    // B fragments: column n0 + gid, values r = 8q + tig and 8q + tig + 4
    const int col = n0 + gid;
    const bool live = col < ncol;
    const int l = live ? col % nlines : 0, i = live ? col / nlines : 0;
    const int j = i % Ns;
    unsigned bh[4][2], bm[4][2], bl[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = 8 * q + tig + 4 * h;
        cx<float> v{0.f, 0.f};
        if (live) {
          v = src[(i + r * nb) * es + l * ls];
          if (Ns > 1 && r > 0) v = c_mul(v, tw_load<float>(tw[r * j * tstride], inv));
        }
        float rh, rm, rl, ih, im, il;
        split_bf16(v.re, rh, rm, rl);
        split_bf16(v.im, ih, im, il);
        bh[q][h] = pk_bf16(rh, ih);
        bm[q][h] = pk_bf16(rm, im);
        bl[q][h] = pk_bf16(rl, il);
      }
    // output: columns n0 + 2 tig, n0 + 2 tig + 1 of the warp's tile
    int oc[2], ol[2];
    bool ok[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int c = n0 + 2 * tig + e;
      ok[e] = c < ncol;
      const int cl = ok[e] ? c % nlines : 0, ci = ok[e] ? c / nlines : 0;
      oc[e] = (ci / Ns) * Ns * 32 + ci % Ns;
      ol[e] = cl;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const uint4 ah = __ldg(&A[((0 * 4 + t) * 4 + q) * 32 + lane]);
        const uint4 am = __ldg(&A[((1 * 4 + t) * 4 + q) * 32 + lane]);
        const uint4 al = __ldg(&A[((2 * 4 + t) * 4 + q) * 32 + lane]);
        mma_bf16(acc, am, bm[q][0], bm[q][1]);
        mma_bf16(acc, al, bh[q][0], bh[q][1]);
        mma_bf16(acc, ah, bl[q][0], bl[q][1]);
        mma_bf16(acc, am, bh[q][0], bh[q][1]);
        mma_bf16(acc, ah, bm[q][0], bm[q][1]);
        mma_bf16(acc, ah, bh[q][0], bh[q][1]);
      }
      // rows m = 16 t + gid (+8): output r' = m / 2, real (m even) or imaginary part
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int m = 16 * t + gid + 8 * hh;
        const int rp = m >> 1;
#pragma unroll
        for (int e = 0; e < 2; ++e)
          if (ok[e]) {
            float *d = reinterpret_cast<float *>(&dst[(oc[e] + rp * Ns) * es + ol[e] * ls]);
            d[m & 1] = acc[2 * hh + e];
          }
      }
    }
  }
}

}  // namespace bpmf
