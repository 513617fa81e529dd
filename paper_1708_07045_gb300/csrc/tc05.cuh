// Radix-32 Stockham stage of the split-bf16 form on the fifth-generation
// tensor cores (tcgen05): the same contraction as tc_dft.cuh (the real
// 64 x 64 DFT-32 matrix F times the twiddled data, both split into bf16
// hi + mid + lo, the six terms of order up to 2^-16), issued as tcgen05.mma
// with the accumulator in tensor memory.
//
// Per tile of 128 stage columns (column = (butterfly i, line l)):
//   1. every thread writes its share of the tile X [128 rows][64 reals] as
//      three bf16 parts into shared memory, K-major core-matrix layout
//      (8 rows x 16 bytes per core matrix; 128 bytes between core matrices
//      along K, 1024 bytes between 8-row groups), a warp filling one core
//      matrix per part at a time;
//   2. one thread issues 4 K-steps x 6 terms of tcgen05.mma.kind::f16
//      (M = 128 rows, N = 64 outputs, K = 16), D[row][n] += sum_k X[row][k]
//      F[n][k], into a 64-column TMEM accumulator, and commits them to an
//      mbarrier;
//   3. after a bounded wait, warp w reads TMEM lanes 32 (w % 4) .. + 31
//      (rows), columns 32 (w / 4) .. + 31 (outputs), with tcgen05.ld and
//      writes the outputs to the stage's destination.
// F's three parts for both directions live in global memory in the same
// core-matrix layout (bpmf_api.cu builds them) and are copied to shared
// memory once per stage call.  A wait that runs out sets *err (if given) and
// leaves the remaining outputs unwritten; no thread waits forever.
#pragma once
#include <cuda_bf16.h>

#include "arith.cuh"

namespace bpmf {

constexpr int kTc05Rows = 128;                               // stage columns per tile (MMA M)
constexpr int kTc05PartBytes = kTc05Rows * 64 * 2;           // one bf16 part of the data tile
constexpr int kTc05FBytes = 64 * 64 * 2;                     // one bf16 part of F
constexpr int kTc05Smem = 3 * kTc05PartBytes + 3 * kTc05FBytes + 1024;  // + alignment slack

__device__ __forceinline__ unsigned tc05_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

// element (row, k) of a K-major bf16 tile in core-matrix layout
__device__ __forceinline__ int tc05_off(int row, int k) {
  return (row >> 3) * 512 + (k >> 3) * 64 + (row & 7) * 8 + (k & 7);
}

__device__ __forceinline__ unsigned long long tc05_desc(unsigned addr) {
  unsigned long long d = (unsigned long long)((addr >> 4) & 0x3FFF);
  d |= (unsigned long long)(128u >> 4) << 16;   // leading byte offset: next core matrix along K
  d |= (unsigned long long)(1024u >> 4) << 32;  // stride byte offset: next 8-row group
  d |= 1ull << 46;                              // descriptor version; no swizzle
  return d;
}

__device__ __forceinline__ void tc05_mma(unsigned tmem, unsigned long long ad, unsigned long long bd, bool acc) {
  // kind::f16: D f32, A and B bf16, both K-major, N = 64, M = 128
  constexpr unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc ? 1u : 0u)
      : "memory");
}

// Bounded wait (about 2^31 SM cycles) on an mbarrier phase; false if it ran out.
__device__ __forceinline__ bool tc05_wait(unsigned bar, unsigned parity) {
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

// One radix-32 stage over nlines lines (element n of line l at buf[n es + l ls]);
// all threads of the CTA call it (blockDim.x a multiple of 256); only the
// split-bf16 instantiations of the kernels compile it.  scratch:
// kTc05Smem bytes of shared memory; fmat: F parts [dir][3][64 x 64] bf16.
__device__ __forceinline__ void tc05_dft32_stage(const cx<float> *src, cx<float> *dst, int es, int ls, int nlines, int P,
                                        int Ns, const float4 *tw, bool inv, const __nv_bfloat16 *fmat,
                                        unsigned char *scratch, int *err) {
  __shared__ unsigned s_tmem;
  __shared__ alignas(8) unsigned long long s_bar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
  unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(scratch) + 1023) & ~uintptr_t(1023));
  __nv_bfloat16 *xa = reinterpret_cast<__nv_bfloat16 *>(base);                          // [3][128 x 64]
  __nv_bfloat16 *fa = reinterpret_cast<__nv_bfloat16 *>(base + 3 * kTc05PartBytes);    // [3][64 x 64]
  // F for this direction (already in core-matrix layout): 16-byte copies
  {
    const uint4 *g = reinterpret_cast<const uint4 *>(fmat + (inv ? 3 * 64 * 64 : 0));
    uint4 *d = reinterpret_cast<uint4 *>(fa);
    for (int e = tid; e < 3 * kTc05FBytes / 16; e += nt) d[e] = g[e];
  }
  if (warp == 0)
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;\n" ::"r"(tc05_u32(&s_tmem))
                 : "memory");
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc05_u32(&s_bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const unsigned tmem = s_tmem;
  const int nb = P / 32;
  const int ncol = nb * nlines;
  const int tstride = P / (Ns * 32);
  unsigned parity = 0;
  bool timed_out = false;
  for (int c0 = 0; c0 < ncol; c0 += kTc05Rows) {
    // 1. the tile's data, twiddled and split, rows = columns c0 .. c0 + 127;
    // a warp takes 8 rows x 4 consecutive values, one 128-byte core matrix
    // per part (no bank conflicts)
    for (int e = tid; e < kTc05Rows * 32; e += nt) {
      const int ln = e & 31, rest = e >> 5;
      const int row = ((rest >> 3) << 3) + (ln >> 2), r = ((rest & 7) << 2) + (ln & 3), col = c0 + row;
      cx<float> v{0.f, 0.f};
      if (col < ncol) {
        const int l = col % nlines, i = col / nlines, j = i % Ns;
        v = src[(i + r * nb) * es + l * ls];
        if (Ns > 1 && r > 0) v = c_mul(v, tw_load<float>(tw[r * j * tstride], inv));
      }
      const int o = tc05_off(row, 2 * r);
      float h[2] = {v.re, v.im};
#pragma unroll
      for (int part = 0; part < 3; ++part) {
        __nv_bfloat162 b;
        b.x = __float2bfloat16_rn(h[0]);
        b.y = __float2bfloat16_rn(h[1]);
        *reinterpret_cast<__nv_bfloat162 *>(xa + part * (kTc05PartBytes / 2) + o) = b;
        h[0] = __fsub_rn(h[0], __bfloat162float(b.x));  // exact remainders
        h[1] = __fsub_rn(h[1], __bfloat162float(b.y));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // 2. 24 MMAs, the smallest terms first: (data part, matrix part)
    if (tid == 0) {
      constexpr int terms[6][2] = {{1, 1}, {0, 2}, {2, 0}, {0, 1}, {1, 0}, {0, 0}};
      for (int ks = 0; ks < 4; ++ks)
#pragma unroll
        for (int t = 0; t < 6; ++t) {
          const unsigned xaddr = tc05_u32(xa) + terms[t][0] * kTc05PartBytes + ks * 256;
          const unsigned faddr = tc05_u32(fa) + terms[t][1] * kTc05FBytes + ks * 256;
          tc05_mma(tmem, tc05_desc(xaddr), tc05_desc(faddr), ks > 0 || t > 0);
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       tc05_u32(&s_bar))
                   : "memory");
    }
    const bool ok = tc05_wait(tc05_u32(&s_bar), parity);
    parity ^= 1u;
    if (__syncthreads_or(!ok)) {  // wait once more (bounded) for the MMAs in flight, then stop
      tc05_wait(tc05_u32(&s_bar), parity ^ 1u);
      timed_out = true;
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // 3. outputs: warp w -> rows 32 (w % 4) + lane, output columns 32 (w / 4) ..
    if (warp < 8) {
      const int row = 32 * (warp & 3) + lane, cbase = 32 * (warp >> 2), col = c0 + row;
      float out[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        unsigned r[16];
        const unsigned taddr = tmem + ((unsigned)(32 * (warp & 3)) << 16) + (unsigned)(cbase + 16 * half);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
        for (int q = 0; q < 16; ++q) out[16 * half + q] = __uint_as_float(r[q]);
      }
      if (col < ncol) {
        const int l = col % nlines, i = col / nlines;
        const int oc = (i / Ns) * Ns * 32 + i % Ns;
#pragma unroll
        for (int q = 0; q < 16; ++q) {  // output r' = cbase / 2 + q: (re, im) at columns 2 r', 2 r' + 1
          const int rp = cbase / 2 + q;
          dst[(oc + rp * Ns) * es + l * ls] = cx<float>{out[2 * q], out[2 * q + 1]};
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();  // the tile buffers and the accumulator are free again
  }
  if (timed_out && tid == 0 && err) atomicOr(err, 1);
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;\n" ::"r"(tmem) : "memory");
  __syncthreads();
}

}  // namespace bpmf
