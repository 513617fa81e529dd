// Hot-path kernels: ligand spreading, forward R2C/C2C passes, the fused
// x-pass (forward ligand DFT, conj-multiply-sum with every receptor spectrum,
// inverse DFT, site window), the inverse y-pass, the inverse C2R z-pass fused
// with the site mask and a max-shifted log-sum-exp, and the FP64 merge into
// log Z_jk, the BPMF per receptor and the standard binding free energy.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "kernels.cuh"

namespace bpmf {

// --------------------------------------------------------------------------
// small helpers
// Streaming multiprocessors of the current device (queried once per device).
int sm_count() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
      cudaGetLastError();
      v = 1;
    }
    cache[dev] = v;
  }
  return cache[dev];
}

__device__ __forceinline__ int imod(int a, int m) {
  int r = a % m;
  return r < 0 ? r + m : r;
}

// Threads per CTA and minimum resident CTAs per SM: float-pair kernels use
// smaller CTAs capped at 128 registers so that 4 can share an SM.
template <class T>
struct KCfg {
  static constexpr int threads = 256, min_blocks = 2, xlw = 8, xconf = 2, x_min_blocks = 3, a_min_blocks = 3,
                       z_min_blocks = 3, zi_min_blocks = 3;
};
template <>
struct KCfg<ff> {
  static constexpr int threads = 128, min_blocks = 4, xlw = 8, xconf = 1, x_min_blocks = 4, a_min_blocks = 4,
                       z_min_blocks = 4, zi_min_blocks = 2;
};

template <class T>
__device__ __forceinline__ void st_cx(void *base, long long idx, cx<T> v) {
  reinterpret_cast<cx<T> *>(base)[idx] = c_norm(v);
}
template <class T>
__device__ __forceinline__ cx<T> ld_cx(const void *base, long long idx) {
  return reinterpret_cast<const cx<T> *>(base)[idx];
}

// receptor spectrum element from hi / lo planes
__device__ __forceinline__ cx<float> ld_rec(const float2 *hi, const float2 *, long long idx, float) {
  float2 a = hi[idx];
  return cx<float>{a.x, a.y};
}
__device__ __forceinline__ cx<ff> ld_rec(const float2 *hi, const float2 *lo, long long idx, ff) {
  float2 a = hi[idx], b = lo[idx];
  return cx<ff>{ff{a.x, b.x}, ff{a.y, b.y}};
}

__device__ __forceinline__ void load_tw(float4 *s_tw, const float4 *tw, int P) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) s_tw[i] = tw[i];
}

// Asynchronous global -> shared copy of one element (8 or 16 bytes), zero
// filled when !valid (no bytes are read then).  All copies a thread issues are
// in flight together; cp_async_wait_all() + __syncthreads() publish them.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? BYTES : 0;
  if constexpr (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(s), "l"(src), "n"(BYTES), "r"(n)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <class T>
__device__ __forceinline__ void cp_cx(cx<T> *dst, const void *base, long long idx, bool valid) {
  const cx<T> *b = reinterpret_cast<const cx<T> *>(base);
  cp_async<sizeof(cx<T>)>(dst, valid ? b + idx : b, valid);
}

// --------------------------------------------------------------------------
// generalised charges (Eqs. electrostatic, repulsive_LJ, attractive_LJ):
// gamma = (q, sqrt(eps) R^p_rep, sqrt(eps) R^p_att), carried as float pairs
// {hi, lo}: g[t * n + i].
__device__ __forceinline__ ff ff_sqrt(float a) {
  const float s = __fsqrt_rn(a);
  if (s == 0.f) return ff{0.f, 0.f};
  const float r = __fmaf_rn(-s, s, a);  // exact residual a - s^2
  return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

__global__ void k_gamma(const float *q, const float *eps, const float *R, int n, int p_rep, int p_att, float2 *g) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const ff se = ff_sqrt(eps[i]);
  const ff r{R[i], 0.f};
  ff pr{1.f, 0.f}, pa{1.f, 0.f};
  for (int k = 0; k < p_rep; ++k) pr = s_mul(pr, r);
  for (int k = 0; k < p_att; ++k) pa = s_mul(pa, r);
  const ff gr = s_norm(s_mul(se, pr)), ga = s_norm(s_mul(se, pa));
  g[i] = make_float2(q[i], 0.f);
  g[n + i] = make_float2(gr.hi, gr.lo);
  g[2 * n + i] = make_float2(ga.hi, ga.lo);
}

cudaError_t launch_gamma(const float *q, const float *eps, const float *R, int n, int p_rep, int p_att, float2 *gamma,
                         cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_gamma<<<(n + 127) / 128, 128, 0, st>>>(q, eps, R, n, p_rep, p_att, gamma);
  return cudaGetLastError();
}

// per-configuration coordinate bounds (placement, "FFT-based BPMF Estimation")
__global__ void k_minmax(const float *xyz, const int *off, const int *nat, int n_conf, float *out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_conf) return;
  const float *x = xyz + 3ll * off[j];
  float lo[3] = {x[0], x[1], x[2]}, hi[3] = {x[0], x[1], x[2]};
  for (int i = 1; i < nat[j]; ++i)
    for (int d = 0; d < 3; ++d) {
      lo[d] = fminf(lo[d], x[3 * i + d]);
      hi[d] = fmaxf(hi[d], x[3 * i + d]);
    }
  for (int d = 0; d < 3; ++d) {
    out[6 * j + d] = lo[d];
    out[6 * j + 3 + d] = hi[d];
  }
}

cudaError_t launch_minmax(const float *coords, const int *off, const int *nat, int n_conf, float *out,
                          cudaStream_t st) {
  if (n_conf <= 0) return cudaSuccess;
  k_minmax<<<(n_conf + 127) / 128, 128, 0, st>>>(coords, off, nat, n_conf, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// (a) spreading.  CTA = (configuration, x-plane of the ligand box).  Each atom
// is placed (lowest coordinate 2 spacings above plane 0) with its grid-unit
// position carried as a float pair, then its 8 trilinear corner weights times
// gamma_t (float-pair products) are accumulated in shared memory in 64-bit
// fixed point (per-channel power-of-two scale from sum |gamma|): the sums are
// exact, order independent and deterministic.  Each node is written once as a
// float pair {hi, lo}.
constexpr int kMaxAtoms = 256;

__global__ void __launch_bounds__(256) k_spread(SpreadArgs a) {
  const int ix = blockIdx.x;
  const int j = blockIdx.y;
  const ConfMeta m = a.meta[j];
  __shared__ int s_c[kMaxAtoms][3];
  __shared__ ff s_f[kMaxAtoms][3];
  __shared__ float s_red[3][8];
  __shared__ int s_e[3];
  extern __shared__ unsigned long long s_plane[];  // [U1][U2]
  const int n = m.n_atoms;
  const ff h{a.h_hi, a.h_lo};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    for (int d = 0; d < 3; ++d) {
      // g = (x - lo) / h + 2 in float-pair precision, then its cell and fraction
      const ff g = place_ff(a.coords[3ll * (m.atom_off + i) + d], m.lo[d], h);
      int c;
      ff f;
      cell_ff(g, c, f);
      s_c[i][d] = c;
      s_f[i][d] = f;
    }
  }
  // per-channel fixed-point scale
  float sa[3] = {0.f, 0.f, 0.f};
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int t = 0; t < 3; ++t) sa[t] += fabsf(a.gamma[(long long)t * a.gamma_stride + m.gamma_off + i].x);
  for (int t = 0; t < 3; ++t) {
    float v = sa[t];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_red[t][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += s_red[threadIdx.x][w];
    // 2^e * (sum |gamma| * 1.01) < 2^60 keeps every partial sum in range
    s_e[threadIdx.x] = v > 0.f ? 59 - ilogbf(v * 1.01f) : 0;
  }
  __syncthreads();
  const int plane = a.U1 * a.U2;
  // the plane is accumulated in chunks of whole y rows that fit the shared buffer
  const int rows = a.chunk_rows;
  const ff one{1.f, 0.f};
  for (int t = 0; t < 3; ++t) {
    const int e = s_e[t];
    float2 *dst = a.box + (((long long)j * 3 + t) * a.U0 + ix) * plane;
    for (int y0 = 0; y0 < a.U1; y0 += rows) {
      const int ny = min(rows, a.U1 - y0), cells = ny * a.U2;
      for (int i = threadIdx.x; i < cells; i += blockDim.x) s_plane[i] = 0ull;
      __syncthreads();
      for (int it = threadIdx.x; it < n * 8; it += blockDim.x) {
        const int i = it >> 3, dx = (it >> 2) & 1, dy = (it >> 1) & 1, dz = it & 1;
        if (s_c[i][0] + dx != ix) continue;
        const int y = s_c[i][1] + dy - y0, z = s_c[i][2] + dz;
        if (y < 0 || y >= ny || z >= a.U2) continue;
        const ff wx = dx ? s_f[i][0] : s_sub(one, s_f[i][0]);
        const ff wy = dy ? s_f[i][1] : s_sub(one, s_f[i][1]);
        const ff wz = dz ? s_f[i][2] : s_sub(one, s_f[i][2]);
        const float2 g2 = a.gamma[(long long)t * a.gamma_stride + m.gamma_off + i];
        const ff v = s_norm(s_mul(s_mul(s_mul(wx, wy), wz), ff{g2.x, g2.y}));
        const long long iv = __float2ll_rn(ldexpf(v.hi, e)) + __float2ll_rn(ldexpf(v.lo, e));
        atomicAdd(&s_plane[y * a.U2 + z], (unsigned long long)iv);
      }
      __syncthreads();
      for (int i = threadIdx.x; i < cells; i += blockDim.x) {
        const long long v = (long long)s_plane[i];
        const float hi = __ll2float_rn(v);
        const float lo = __ll2float_rn(v - __float2ll_rn(hi));  // exact remainder, then rounded
        dst[(long long)y0 * a.U2 + i] = make_float2(ldexpf(hi, -e), ldexpf(lo, -e));
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_spread(const SpreadArgs &a_in, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  SpreadArgs a = a_in;
  // at most 96 KB of 64-bit accumulators per CTA, in whole y rows
  a.chunk_rows = std::max(1, std::min(a.U1, (int)((96 * 1024) / (sizeof(unsigned long long) * std::max(a.U2, 1)))));
  const size_t smem = sizeof(unsigned long long) * (size_t)a.chunk_rows * a.U2;
  // static + dynamic shared memory may pass the 48 KB default: always opt in
  cudaError_t e = cudaFuncSetAttribute(k_spread, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_spread<<<dim3(a.U0, batch), 256, smem, st>>>(a);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// (b) R2C along the contiguous axis: two real rows packed as one complex line.
template <class T, bool TC = false>
__global__ void __launch_bounds__(KCfg<T>::threads, KCfg<T>::z_min_blocks) k_zfwd(ZfwdArgs a) {
  extern __shared__ float4 smem[];
  const int P = a.plan.n, L = a.L, ls = P + 1, F = P / 2 + 1;
  float4 *s_tw = smem;
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem + P);
  cx<T> *b1 = b0 + L * ls;
  load_tw(s_tw, a.tw, P);
  const long long r0 = (long long)blockIdx.x * 2 * L;
  for (int idx = threadIdx.x; idx < L * P; idx += blockDim.x) {
    const int l = idx / P, n = idx % P;
    const long long ra = r0 + 2 * l, rb = ra + 1;
    const bool va = n < a.w_in && ra < a.n_rows, vb = n < a.w_in && rb < a.n_rows;
    cx<T> *d = &b0[l * ls + n];
    if (a.in_pairs) {
      // float-pair rows: row ra -> real part, row rb -> imaginary part
      const float2 *in2 = reinterpret_cast<const float2 *>(a.in);
      if constexpr (sizeof(T) == 8) {
        cp_async<8>(&d->re, va ? in2 + ra * a.in_stride + n : in2, va);
        cp_async<8>(&d->im, vb ? in2 + rb * a.in_stride + n : in2, vb);
      } else {
        cp_async<4>(&d->re, va ? &in2[ra * a.in_stride + n].x : a.in, va);
        cp_async<4>(&d->im, vb ? &in2[rb * a.in_stride + n].x : a.in, vb);
      }
    } else {
      const float x = va ? a.in[ra * a.in_stride + n] : 0.f;
      const float y = vb ? a.in[rb * a.in_stride + n] : 0.f;
      *d = cx<T>{s_from<T>(x), s_from<T>(y)};
    }
  }
  cp_async_wait_all();
  __syncthreads();
  cx<T> *res = cta_fft_auto<T, 16, KCfg<T>::threads, true, false, TC>(b0, b1, 1, ls, L, a.plan, s_tw, false);
  const T half = s_from<T>(0.5f);
  for (int idx = threadIdx.x; idx < L * F; idx += blockDim.x) {
    const int l = idx / F, k = idx % F;
    const long long ra = r0 + 2 * l, rb = ra + 1;
    const cx<T> zk = res[l * ls + k];
    const cx<T> zn = c_conj(res[l * ls + (k == 0 ? 0 : P - k)]);
    // A = (Z_k + conj Z_{P-k}) / 2,  B = -i (Z_k - conj Z_{P-k}) / 2
    const cx<T> s = c_add(zk, zn), d = c_sub(zk, zn);
    if (ra < a.n_rows) st_cx<T>(a.out, ra * a.out_stride + k, cx<T>{s_mul(s.re, half), s_mul(s.im, half)});
    if (rb < a.n_rows) st_cx<T>(a.out, rb * a.out_stride + k, cx<T>{s_mul(d.im, half), s_neg(s_mul(d.re, half))});
  }
}

// Kernels whose plan has a tcgen05 stage get kTc05Smem bytes of scratch at
// the end of their dynamic shared memory.
inline size_t with_tc05(FftPlan &pl, size_t smem) {
  if (!pl.tc05_f) return smem;
  pl.tc05_off = (int)smem;
  return smem + kTc05Smem;
}

template <class T>
cudaError_t launch_zfwd(const ZfwdArgs &a_in, cudaStream_t st) {
  if (a_in.n_rows <= 0) return cudaSuccess;
  ZfwdArgs a = a_in;
  const int P = a.plan.n;
  const size_t smem = with_tc05(a.plan, sizeof(float4) * P + 2 * sizeof(cx<T>) * (size_t)a.L * (P + 1));
  const long long blocks = (a.n_rows + 2 * a.L - 1) / (2 * a.L);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, KCfg<T>::threads, smem, st>>>(a);
    return cudaGetLastError();
  };
  if constexpr (std::is_same<T, float>::value)
    if (a.plan.tca) return go(k_zfwd<T, true>);
  return go(k_zfwd<T, false>);
}

// --------------------------------------------------------------------------
// C2C along a strided axis for a tile of LW consecutive innermost indices
// (LWC > 0: LW fixed at compile time, so tile indices are shifts and masks).
template <class T, int LWC, bool TC = false>
__global__ void __launch_bounds__(KCfg<T>::threads, KCfg<T>::a_min_blocks) k_axis(AxisArgs a) {
  extern __shared__ float4 smem[];
  const int P = a.plan.n, LW = LWC > 0 ? LWC : a.LW;
  float4 *s_tw = smem;
  cx<T> *b0 = reinterpret_cast<cx<T> *>(smem + P);
  cx<T> *b1 = b0 + P * LW;
  __shared__ long long s_in[64], s_out[64];  // per tile column: base offsets of input / output
  __shared__ int s_w0[64];                   // per tile column: output window start mod P
  load_tw(s_tw, a.tw, P);
  // columns are the flattened (outer, inner) pairs, so a tile never wastes
  // lanes on a short inner edge
  const long long ncols = a.n_outer * a.inner;
  const long long c0 = (long long)blockIdx.x * LW;
  if (threadIdx.x < LW) {
    const long long c = c0 + threadIdx.x;
    const long long o = c < ncols ? c / a.inner : 0, i = c < ncols ? c % a.inner : 0;
    s_in[threadIdx.x] = c < ncols ? o * a.in_os + i : -1;
    s_out[threadIdx.x] = c < ncols ? o * a.out_os + i : -1;
    s_w0[threadIdx.x] = a.info ? imod(a.info[o / a.w0_div].wc[a.axis], P) : 0;
  }
  __syncthreads();
  const int n_in = a.n_in < P ? a.n_in : P;
  for (int idx = threadIdx.x; idx < n_in * LW; idx += blockDim.x) {
    const int n = idx / LW, l = idx % LW;
    const long long base = s_in[l];
    cp_cx<T>(&b0[idx], a.in, base + n * a.inner, base >= 0);
  }
  for (int idx = n_in * LW + threadIdx.x; idx < P * LW; idx += blockDim.x) b0[idx] = c_zero<T>();
  cp_async_wait_all();
  __syncthreads();
  cx<T> *res = cta_fft_auto<T, (LWC > 0 ? LWC : 16), KCfg<T>::threads, false, true, TC>(b0, b1, LW, 1, LW, a.plan,
                                                                                 s_tw, a.inverse != 0);
  // outputs s < n_out <= P, read at (w0 + s) mod P
  for (int idx = threadIdx.x; idx < a.n_out * LW; idx += blockDim.x) {
    const int s = idx / LW, l = idx % LW;
    const long long base = s_out[l];
    const int m = s_w0[l] + s;
    if (base < 0) continue;
    const cx<T> v = res[(m >= P ? m - P : m) * LW + l];
    if constexpr (std::is_same<T, ff>::value) {
      if (a.out_hi) {  // split into the hi / lo planes
        const cx<ff> w = c_norm(v);
        a.out_hi[base + s * a.inner] = make_float2(w.re.hi, w.im.hi);
        a.out_lo[base + s * a.inner] = make_float2(w.re.lo, w.im.lo);
        continue;
      }
    }
    st_cx<T>(a.out, base + s * a.inner, v);
  }
}

template <class T, int LWC>
cudaError_t launch_axis_lw(const AxisArgs &a_in, cudaStream_t st) {
  AxisArgs a = a_in;
  const int P = a.plan.n;
  const size_t smem = with_tc05(a.plan, sizeof(float4) * P + 2 * sizeof(cx<T>) * (size_t)P * a.LW);
  const long long blocks = (a.n_outer * a.inner + a.LW - 1) / a.LW;
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, KCfg<T>::threads, smem, st>>>(a);
    return cudaGetLastError();
  };
  if constexpr (std::is_same<T, float>::value)
    if (a.plan.tca) return go(k_axis<T, LWC, true>);
  return go(k_axis<T, LWC, false>);
}

template <class T>
cudaError_t launch_axis(const AxisArgs &a, cudaStream_t st) {
  if (a.n_outer <= 0 || a.inner <= 0) return cudaSuccess;
  if (a.LW < 1 || a.LW > 64 || a.n_out > a.plan.n) return cudaErrorInvalidValue;
  if (a.LW == 32) return launch_axis_lw<T, 32>(a, st);
  if (a.LW == 16) return launch_axis_lw<T, 16>(a, st);
  if (a.LW == 8) return launch_axis_lw<T, 8>(a, st);
  return launch_axis_lw<T, 0>(a, st);
}

// --------------------------------------------------------------------------
// (b)+(c)+(d, first inverse pass) along x.  CTA = (G configurations, tile of
// LW consecutive (y, zf) columns).  Forward DFT of the 3 ligand channels of
// each configuration, then for each receptor k: P_k = sum_t R_{k,t} conj(L_t),
// inverse DFT, keep the site window along x.  Each receptor element is loaded
// once per CTA and used for all G configurations; the ligand spectra never
// leave shared memory.
template <class T, int KP, bool TC = false>
__global__ void __launch_bounds__(KCfg<T>::threads, KCfg<T>::x_min_blocks) k_xfused(XfusedArgs a, int batch) {
  extern __shared__ float4 smem[];
  constexpr int LW = KCfg<T>::xlw, G = KCfg<T>::xconf, LG = G * LW, L3 = 3 * LG;
  constexpr int LK = KP * LG;  // inverse lines per pass: KP receptors x G configurations x LW columns
  constexpr int LB = L3 > 2 * LK ? L3 : 2 * LK;
  const int P = a.plan.n;
  float4 *s_tw = smem;
  // R = [bB: LB lines][bA: L3 lines]; the forward transform runs bA -> bB ->
  // ..., and whichever buffer holds its result, the other P (L3 + LB) - P L3
  // elements form one contiguous free region of at least 2 LK lines
  cx<T> *R = reinterpret_cast<cx<T> *>(smem + P);
  cx<T> *bB = R;
  cx<T> *bA = R + P * LB;
  load_tw(s_tw, a.tw, P);
  // tile-major order: CTAs resident together share a column tile across many
  // configurations, so that tile's receptor spectra are served from L2
  const int nJG = (batch + G - 1) / G;
  const int j0 = (blockIdx.x % nJG) * G;
  const long long q0 = (long long)(blockIdx.x / nJG) * LW;
  const int U0 = a.U0 < P ? a.U0 : P;
  // ligand columns: c = (g * 3 + t) * LW + l
  for (int idx = threadIdx.x; idx < U0 * L3; idx += blockDim.x) {
    const int x = idx / L3, c = idx % L3, gt = c / LW, l = c % LW;
    const int j = j0 + gt / 3, t = gt % 3;
    const long long q = q0 + l;
    // rows beyond a configuration's own ligand box are zero (not read)
    const bool in_box = j < batch && (!a.meta || x < a.meta[j].u[0]);
    cp_cx<T>(&bA[idx], a.ly, (((long long)j * 3 + t) * a.U0 + x) * a.Q + q, q < a.Q && in_box);
  }
  for (int idx = U0 * L3 + threadIdx.x; idx < P * L3; idx += blockDim.x) bA[idx] = c_zero<T>();
  cp_async_wait_all();
  __syncthreads();
  cx<T> *Lsp = cta_fft_auto<T, L3, KCfg<T>::threads, false, false, TC>(bA, bB, L3, 1, L3, a.plan, s_tw, false);
  cx<T> *W1 = (Lsp == bB) ? R + P * L3 : R;
  cx<T> *W2 = W1 + P * LK;
  __shared__ int s_wm[KP * G];  // per (receptor of the pass, configuration): site window start along x, mod P
  for (int k0 = 0; k0 < a.K; k0 += KP) {
    if (threadIdx.x < KP * G) {
      const int kk = threadIdx.x / G, j = j0 + (int)threadIdx.x % G;
      s_wm[threadIdx.x] = (j < batch && k0 + kk < a.K) ? imod(a.info[j * a.K + k0 + kk].wc[0], P) : 0;
    }
    // inverse line c = (kk * G + g) * LW + l
    for (int idx = threadIdx.x; idx < P * LW; idx += blockDim.x) {
      const int x = idx / LW, l = idx % LW;
      const long long q = q0 + l;
#pragma unroll
      for (int kk = 0; kk < KP; ++kk) {
        cx<T> r0 = c_zero<T>(), r1 = c_zero<T>(), r2 = c_zero<T>();
        if (q < a.Q && k0 + kk < a.K) {
          const float2 *rh = a.rhi[k0 + kk];
          const float2 *rl = a.rlo ? a.rlo[k0 + kk] : nullptr;
          const long long ri = (long long)x * a.Q + q, rs = (long long)P * a.Q;
          r0 = ld_rec(rh, rl, ri, T{});
          r1 = ld_rec(rh, rl, ri + rs, T{});
          r2 = ld_rec(rh, rl, ri + 2 * rs, T{});
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
          const cx<T> *lx = Lsp + x * L3 + g * 3 * LW + l;
          const cx<T> acc = c_add(c_add(c_mulconj(r0, lx[0]), c_mulconj(r1, lx[LW])), c_mulconj(r2, lx[2 * LW]));
          W1[x * LK + (kk * G + g) * LW + l] = c_norm(acc);
        }
      }
    }
    __syncthreads();
    cx<T> *res = cta_fft_auto<T, LK, KCfg<T>::threads, false, false, TC>(W1, W2, LK, 1, LK, a.plan, s_tw, true);
    for (int idx = threadIdx.x; idx < a.S0 * LK; idx += blockDim.x) {
      const int s = idx / LK, c = idx % LK, kg = c / LW, l = c % LW;
      const int k = k0 + kg / G, j = j0 + kg % G;
      const long long q = q0 + l;
      if (q < a.Q && j < batch && k < a.K) {
        const int m = s_wm[kg] + s;  // s < S0 <= P
        st_cx<T>(a.x2, (((long long)j * a.K + k) * a.S0 + s) * a.Q + q, res[(m >= P ? m - P : m) * LK + c]);
      }
    }
    __syncthreads();
  }
}

template <class T, int KP>
size_t xfused_smem(int P) {
  constexpr int LW = KCfg<T>::xlw, G = KCfg<T>::xconf, L3 = 3 * G * LW, LK = KP * G * LW;
  constexpr int LB = L3 > 2 * LK ? L3 : 2 * LK;
  return sizeof(float4) * P + sizeof(cx<T>) * (size_t)P * (L3 + LB);
}

template <class T, int KP>
cudaError_t launch_xfused_kp(const XfusedArgs &a_in, int batch, cudaStream_t st) {
  constexpr int LW = KCfg<T>::xlw, G = KCfg<T>::xconf;
  XfusedArgs a = a_in;
  const size_t smem = with_tc05(a.plan, xfused_smem<T, KP>(a.plan.n));
  const long long blocks = (long long)((batch + G - 1) / G) * ((a.Q + LW - 1) / LW);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)blocks, KCfg<T>::threads, smem, st>>>(a, batch);
    return cudaGetLastError();
  };
  if constexpr (std::is_same<T, float>::value)
    if (a.plan.tca) return go(k_xfused<T, KP, true>);
  return go(k_xfused<T, KP, false>);
}

// Two receptors per inverse pass (twice the lines per transform stage) when
// several receptors share the pass and the larger shared-memory footprint
// still leaves x_min_blocks CTAs per SM.
template <class T>
cudaError_t launch_xfused(const XfusedArgs &a, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  if (a.K >= 2 && !a.plan.tc05_f && xfused_smem<T, 2>(a.plan.n) * KCfg<T>::x_min_blocks <= 227 * 1024)
    return launch_xfused_kp<T, 2>(a, batch, st);
  return launch_xfused_kp<T, 1>(a, batch, st);
}

// --------------------------------------------------------------------------
// (d) last inverse pass: C2R along z of two packed rows, 1/(P0 P1 P2) scale,
// site mask, then a max-shifted log-sum-exp over this CTA's (s1, s2) plane.
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__device__ __forceinline__ bool ff_gt(float a, float b) { return a > b; }

template <class T, int NY, bool TC = false>
__global__ void __launch_bounds__(256, KCfg<T>::zi_min_blocks) k_zinv(ZinvArgs a) {
  extern __shared__ float4 smem[];
  const int P = a.plan.n, F = a.F2, ls = P + 1;
  const int Lc = a.Lc;  // row pairs per chunk (all of them when they fit)
  const int b1n = Lc * ls > 2 * Lc * F ? Lc * ls : 2 * Lc * F;
  float4 *s_tw = smem;
  cx<T> *b0, *b1;
  T *xs;  // [2 Lc * S2]
  float4 *s_tw1 = nullptr;
  if constexpr (NY == 0) {
    b0 = reinterpret_cast<cx<T> *>(smem + P);
    b1 = b0 + Lc * ls;
    xs = reinterpret_cast<T *>(b1 + b1n);
  } else {
    // [tw (P2)][tw1 (P1)][b1][b0][xs]: the y pass's two buffers (2 P1 NY
    // elements) overlay b0 and xs, which are free until the z transform
    s_tw1 = smem + P;
    b1 = reinterpret_cast<cx<T> *>(s_tw1 + a.yplan.n);
    b0 = b1 + b1n;
    xs = reinterpret_cast<T *>(b0 + Lc * ls);
  }
  // refined form: the FP32 energies of the chunk, after xs
  float *es = reinterpret_cast<float *>(xs + 2 * Lc * a.S2);
  __shared__ T s_red[8];
  __shared__ float s_sum[8];
  __shared__ float s_thr;
  load_tw(s_tw, a.tw, P);
  const int s0 = blockIdx.x % a.S0;
  const int jk = blockIdx.x / a.S0;  // j * K + k
  const PairInfo inf = a.info[jk];
  const bool row_ok = (s0 >= inf.sa[0] && s0 <= inf.sb[0]);
  // refined form (FP32 only): candidate lists of the exact re-evaluation
  const bool refine = std::is_same<T, float>::value && a.rs.cand != nullptr;
  if constexpr (NY > 0) {
    // y inverse of this CTA's plane in sub-passes of NY columns (the per-line
    // arithmetic of k_axis's two-stage plan, so the values are the same);
    // the site window rows land in b1 as the z pass's staged input
    const int P1 = a.yplan.n;
    load_tw(s_tw1, a.tw1, P1);
    if (row_ok) {  // uniform over the CTA
      cx<T> *yb = b0;
      const int w1 = imod(inf.wc[1], P1);
      const long long plane = (long long)blockIdx.x * a.Qx;
      for (int c0 = 0; c0 < F; c0 += NY) {
        __syncthreads();
        for (int idx = threadIdx.x; idx < P1 * NY; idx += blockDim.x) {
          const int ky = idx / NY, l = idx % NY;
          cp_cx<T>(&yb[idx], a.x2, plane + (long long)ky * F + c0 + l, c0 + l < F);
        }
        cp_async_wait_all();
        __syncthreads();
        cx<T> *res = cta_fft_auto<T, NY, 256, false, true>(yb, yb + P1 * NY, NY, 1, NY, a.yplan, s_tw1, true);
        for (int idx = threadIdx.x; idx < a.S1 * NY; idx += blockDim.x) {
          const int s1 = idx / NY, l = idx % NY;
          const int m = w1 + s1;  // s1 < S1 <= P1
          if (c0 + l < F) b1[s1 * F + c0 + l] = res[(m >= P1 ? m - P1 : m) * NY + l];
        }
      }
    }
  }
  const T nscale = s_mk<T>(a.nscale_hi, a.nscale_lo);
  const T escale = s_mk<T>(a.escale_hi, a.escale_lo);
  // running max-shifted sum over the chunks: M_run and s_run relative to it
  T M_run = s_mk<T>(-CUDART_INF_F, 0.f);
  float s_run = 0.f;
  for (int r0 = 0; r0 < a.S1; r0 += 2 * Lc) {
    const int nrow = min(2 * Lc, a.S1 - r0), L = (nrow + 1) / 2;
    const long long base = ((long long)blockIdx.x * a.S1 + r0) * F;
    // stage this chunk's [rows][F2] half spectra with asynchronous copies,
    // then pack row pairs as z = A + iB with Hermitian extension
    cx<T> *stg = b1;
    __syncthreads();
    if (NY == 0 && row_ok) {  // fused: the y pass has staged the one chunk already
      for (int idx = threadIdx.x; idx < nrow * F; idx += blockDim.x) cp_cx<T>(&stg[idx], a.y2, base + idx, true);
      cp_async_wait_all();
    }
    __syncthreads();
    // (l, n) = divmod(idx, P), stepped without a division per element
    const int dl = (int)blockDim.x / P, dn = (int)blockDim.x % P;
    for (int idx = threadIdx.x, l = (int)threadIdx.x / P, n = (int)threadIdx.x % P; idx < L * P;
         idx += blockDim.x, l += dl, n += dn) {
      if (n >= P) {
        n -= P;
        ++l;
      }
      const int ra = 2 * l, rb = ra + 1;
      cx<T> A = c_zero<T>(), B = c_zero<T>();
      const bool up = n <= P / 2;
      const int kk = up ? n : P - n;
      const bool real_bin = (kk == 0) || (2 * kk == P);
      if (row_ok) {
        A = stg[ra * F + kk];
        if (rb < nrow) B = stg[rb * F + kk];
      }
      if (real_bin) {
        A.im = s_zero<T>();
        B.im = s_zero<T>();
      }
      if (!up) {
        A = c_conj(A);
        B = c_conj(B);
      }
      b0[l * ls + n] = c_norm(cx<T>{s_sub(A.re, B.im), s_add(A.im, B.re)});
    }
    __syncthreads();
    cx<T> *res = cta_fft_auto<T, 20, 256, true, (std::is_same<T, float>::value && NY > 0), TC>(b0, b1, 1, ls, L, a.plan, s_tw, true);
    const int nS = nrow * a.S2;
    T vmax = s_mk<T>(-CUDART_INF_F, 0.f);
    float emin = CUDART_INF_F;  // refined form: plane minimum of the energies
    // (r, s2) = divmod(idx, S2) stepped the same way; z index (wc + s2) mod P
    // from its value at s2 = 0 (s2 < S2 <= P)
    const int dr = (int)blockDim.x / a.S2, ds = (int)blockDim.x % a.S2;
    const int zb = imod(inf.wc[2], P);
    for (int idx = threadIdx.x, r = (int)threadIdx.x / a.S2, s2 = (int)threadIdx.x % a.S2; idx < nS;
         idx += blockDim.x, r += dr, s2 += ds) {
      if (s2 >= a.S2) {
        s2 -= a.S2;
        ++r;
      }
      const int s1 = r0 + r;
      const int zi = zb + s2 >= P ? zb + s2 - P : zb + s2;
      bool ok = row_ok && s1 >= inf.sa[1] && s1 <= inf.sb[1] && s2 >= inf.sa[2] && s2 <= inf.sb[2];
      if (ok && a.clash) {  // a clashing translation has infinite energy (it stays counted in n)
        const uint32_t w = a.clash[((long long)blockIdx.x * a.S1 + s1) * a.CW + (s2 >> 5)];
        ok = !((w >> (s2 & 31)) & 1u);
      }
      T x = s_mk<T>(-CUDART_INF_F, 0.f);
      float ef = CUDART_INF_F;
      if (ok) {
        const cx<T> z = res[(r >> 1) * ls + zi];
        const T val = (r & 1) ? z.im : z.re;
        if (refine) {
          ef = s_hi(s_norm(s_mul(val, escale)));
          emin = fminf(emin, ef);
        } else {
          x = s_norm(s_mul(val, nscale));
          if (ff_gt(x, vmax)) vmax = x;
        }
      }
      if (refine)
        es[idx] = ef;
      else
        xs[idx] = x;
      if (a.export_E && jk == 0) {
        double e = CUDART_INF;
        if (ok) {
          const cx<T> z = res[(r >> 1) * ls + zi];
          const T E = s_norm(s_mul((r & 1) ? z.im : z.re, escale));
          e = (double)s_hi(E) + (double)s_lo(E);
        }
        a.export_E[((long long)s0 * a.S1 + s1) * a.S2 + s2] = e;
      }
    }
    if (refine) {
      // the chunk's minimum lowers the pair's running minimum; translations
      // within W + 2B of it are appended to the pair's list (warp-aggregated).
      // The list is the pair's whole weight: every translation left out lies
      // more than W above the pair's minimum (its FP32 energy exceeds the
      // final minimum + W + 2B), and together they weigh less than 1e-5 of S,
      // so the plane writes no partial of its own
      for (int o = 16; o > 0; o >>= 1) emin = fminf(emin, __shfl_xor_sync(0xffffffffu, emin, o));
      if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = emin;
      __syncthreads();
      if (threadIdx.x == 0) {
        float v = s_sum[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fminf(v, s_sum[w]);
        float thr = -CUDART_INF_F;
        if (v < CUDART_INF_F) {
          const float run = fminf(ord2f(atomicMin(&a.rs.pmin[jk], f2ord(v))), v);
          thr = __fadd_ru(run, a.rs.win[jk % a.K]);
        }
        s_thr = thr;
      }
      __syncthreads();
      const float thr = s_thr;
      const int lane = threadIdx.x & 31;
      Cand *list = a.rs.cand + (long long)jk * a.rs.cap;
      const unsigned t0 = (unsigned)((s0 * a.S1 + r0) * a.S2);
      for (int b = (int)(threadIdx.x & ~31u); b < nS; b += blockDim.x) {
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
      continue;  // the next chunk's first barrier orders these reads of es before its writes
    }
    // block max of the chunk
    for (int o = 16; o > 0; o >>= 1) {
      T other = s_mk<T>(__shfl_xor_sync(0xffffffffu, s_hi(vmax), o), __shfl_xor_sync(0xffffffffu, s_lo(vmax), o));
      if (ff_gt(other, vmax)) vmax = other;
    }
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = vmax;
    __syncthreads();
    T M = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (ff_gt(s_red[w], M)) M = s_red[w];
    float acc = 0.f;
    if (s_hi(M) > -CUDART_INF_F) {
      for (int idx = threadIdx.x; idx < nS; idx += blockDim.x) {
        const T x = xs[idx];
        if (s_hi(x) > -CUDART_INF_F) {
          const float d = __fadd_rn(__fsub_rn(s_hi(x), s_hi(M)), __fsub_rn(s_lo(x), s_lo(M)));
          acc += expf(d);
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = acc;
    __syncthreads();
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += s_sum[w];
    // combine with the earlier chunks (one chunk: M_run = M, s_run = s)
    if (s_hi(M) > -CUDART_INF_F) {
      if (!(s_hi(M_run) > -CUDART_INF_F)) {
        M_run = M;
        s_run = s;
      } else if (ff_gt(M, M_run)) {
        s_run = s_run * expf(__fadd_rn(__fsub_rn(s_hi(M_run), s_hi(M)), __fsub_rn(s_lo(M_run), s_lo(M)))) + s;
        M_run = M;
      } else {
        s_run += s * expf(__fadd_rn(__fsub_rn(s_hi(M), s_hi(M_run)), __fsub_rn(s_lo(M), s_lo(M_run))));
      }
    }
  }
  if (threadIdx.x == 0) a.part[blockIdx.x] = make_float4(s_hi(M_run), s_lo(M_run), s_run, 0.f);
}

template <class T>
size_t zinv_smem(const ZinvArgs &a, int Lc) {
  const int P = a.plan.n;
  const size_t b1n = std::max((size_t)Lc * (P + 1), (size_t)2 * Lc * a.F2);
  const size_t es = a.rs.cand ? sizeof(float) * (size_t)2 * Lc * a.S2 : 0;  // refined form's FP32 energies
  return sizeof(float4) * P + sizeof(cx<T>) * ((size_t)Lc * (P + 1) + b1n) + sizeof(T) * (size_t)2 * Lc * a.S2 + es +
         (a.plan.tc05_f ? (size_t)kTc05Smem : 0);  // tcgen05 scratch (placed last)
}

// Fused y + z inverse (FP32): y sub-pass width for F2 columns (two sub-passes
// of at most 21 or 25 lines), 0 when F2 is wider
int zinv_ny(int F2) { return F2 <= 42 ? 21 : (F2 <= 50 ? 25 : 0); }

size_t zinv_fused_smem(int P1, int P2, int S1, int S2, bool refine) {
  const int F2 = P2 / 2 + 1, Lc = (S1 + 1) / 2, NY = zinv_ny(F2);
  const size_t b1n = std::max((size_t)Lc * (P2 + 1), (size_t)2 * Lc * F2);
  const size_t tail = std::max(sizeof(cx<float>) * Lc * (P2 + 1) + sizeof(float) * 2 * Lc * S2 * (refine ? 2 : 1),
                               sizeof(cx<float>) * 2 * P1 * NY);
  return sizeof(float4) * (P1 + P2) + sizeof(cx<float>) * b1n + tail;
}

bool zinv_fused_fits(int P1, int P2, int S1, int S2, bool refine) {
  return zinv_ny(P2 / 2 + 1) > 0 && S1 <= P1 && zinv_fused_smem(P1, P2, S1, S2, refine) * 3 <= 227 * 1024;
}

template <class T, int NY, bool TC = false>
cudaError_t launch_zinv_k(const ZinvArgs &a, size_t smem, int batch, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_zinv<T, NY, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_zinv<T, NY, TC><<<(unsigned)((long long)batch * a.K * a.S0), 256, smem, st>>>(a);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_zinv(const ZinvArgs &a_in, int batch, cudaStream_t st) {
  if (batch <= 0) return cudaSuccess;
  ZinvArgs a = a_in;
  const int L = (a.S1 + 1) / 2;
  if (a.x2) {  // fused y + z inverse: FP32 only, the whole window in one chunk
    if constexpr (std::is_same<T, float>::value) {
      const int P1 = a.yplan.n;
      const bool refine = a.rs.cand != nullptr;
      if (!zinv_fused_fits(P1, a.plan.n, a.S1, a.S2, refine) || a.F2 != a.plan.n / 2 + 1)
        return cudaErrorInvalidValue;
      a.Lc = L;
      const size_t smem = zinv_fused_smem(P1, a.plan.n, a.S1, a.S2, refine);
      return zinv_ny(a.F2) == 21 ? launch_zinv_k<float, 21>(a, smem, batch, st)
                                 : launch_zinv_k<float, 25>(a, smem, batch, st);
    }
    return cudaErrorInvalidValue;
  }
  // all row pairs of the site window in one chunk when they fit in shared
  // memory (227 KB per CTA), else the largest chunk that does
  int Lc = L;
  while (Lc > 1 && zinv_smem<T>(a, Lc) > 227 * 1024) --Lc;
  if (zinv_smem<T>(a, Lc) > 227 * 1024) return cudaErrorInvalidValue;
  a.Lc = Lc;
  const size_t smem = zinv_smem<T>(a, Lc);
  if (a.plan.tc05_f) a.plan.tc05_off = (int)(smem - kTc05Smem);
  if constexpr (std::is_same<T, float>::value)
    if (a.plan.tca) return launch_zinv_k<T, 0, true>(a, smem, batch, st);
  return launch_zinv_k<T, 0>(a, smem, batch, st);
}

// --------------------------------------------------------------------------
// FP64 merge (Eq. sample_mean_BPMF pooled over every valid pose; Eqs.
// standard_binding_fe / binding_FE_estimate with uniform receptor weights):
//   log S_jk = M* + ln sum_c s_c exp(M_c - M*)      over the S0 partials
//   log Z_jk = log S_jk - ln n_jk
//   B_k      = -kT [ LSE_j log S_jk - ln sum_j n_jk ]
//   dG       = -kT [ LSE_k (-B_k / kT) - ln K ] - kT ln(V_site C)
__global__ void __launch_bounds__(128) k_merge_pairs(MergeArgs a) {
  const int JK = a.J * a.Kg;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= JK) return;
  const int j = p / a.Kg, kg = p % a.Kg;
  const int k = a.kmap ? a.kmap[kg] : kg;
  const float4 *pp = a.part + (long long)p * a.S0;
  double Mx = -CUDART_INF;
  for (int c = 0; c < a.S0; ++c)
    if (pp[c].z > 0.f) Mx = fmax(Mx, (double)pp[c].x + (double)pp[c].y);
  // refined form: the pair's re-evaluated translations (their weight sum as
  // a float pair)
  double X = -CUDART_INF;  // largest exact -E/kT
  float4 rc{0.f, 0.f, 0.f, 0.f};
  if (a.part_ref) {
    rc = a.part_ref[2ll * p];
    const float4 rx = a.part_ref[2ll * p + 1];
    if (rc.z > 0.f) {
      X = (double)rx.x + (double)rx.y;
      Mx = fmax(Mx, (double)rc.x + (double)rc.y);
    }
  }
  double s = 0.0;
  if (Mx > -CUDART_INF) {
    for (int c = 0; c < a.S0; ++c)
      if (pp[c].z > 0.f) s += (double)pp[c].z * exp((double)pp[c].x + (double)pp[c].y - Mx);
    if (rc.z > 0.f) s += ((double)rc.z + (double)rc.w) * exp((double)rc.x + (double)rc.y - Mx);
  }
  // the dominant state: the largest -E/kT, exact where the pair was refined
  const double Xd = X > -CUDART_INF ? X : Mx;
  // processing position -> caller's configuration order
  const long long q = (long long)(a.order ? a.order[j] : j) * a.K + k;
  const long long n = a.nvalid[q];
  const double ls = (s > 0.0 && n > 0) ? Mx + log(s) : -CUDART_INF;
  a.logS[q] = ls;
  a.logZ[q] = n > 0 ? ls - log((double)n) : -CUDART_INF;
  if (a.nvalid_out) a.nvalid_out[q] = n;
  // dominant-state energy: the largest -E/kT of all partials, back to kcal/mol
  if (a.emin) a.emin[q] = (Xd > -CUDART_INF && n > 0) ? -a.kT * Xd : CUDART_INF;
}

__global__ void __launch_bounds__(256) k_merge(MergeArgs a) {
  __shared__ double s_d[256];
  __shared__ long long s_l[256];
  const double *logS = a.logS;
  __syncthreads();
  long long ntot_all = 0;
  for (int k = 0; k < a.K; ++k) {
    double mx = -CUDART_INF;
    long long nt = 0;
    for (int j = threadIdx.x; j < a.J; j += blockDim.x) {
      mx = fmax(mx, logS[(long long)j * a.K + k]);
      nt += a.nvalid[(long long)j * a.K + k];
    }
    s_d[threadIdx.x] = mx;
    s_l[threadIdx.x] = nt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + o]);
        s_l[threadIdx.x] += s_l[threadIdx.x + o];
      }
      __syncthreads();
    }
    const double M = s_d[0];
    const long long ntot = s_l[0];
    __syncthreads();
    double acc = 0.0;
    if (M > -CUDART_INF)
      for (int j = threadIdx.x; j < a.J; j += blockDim.x) {
        const double v = logS[(long long)j * a.K + k];
        if (v > -CUDART_INF) acc += exp(v - M);
      }
    s_d[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double B = (ntot > 0 && s_d[0] > 0.0) ? -a.kT * (M + log(s_d[0]) - log((double)ntot)) : CUDART_INF;
      a.bpmf[k] = B;
    }
    ntot_all += ntot;
    __syncthreads();
  }
  // dominant-state estimates (Section "Dominant state"): the minimum
  // interaction energy per receptor, its minimum and exponential average over
  // receptors
  if (a.dom && a.emin) {
    for (int k = 0; k < a.K; ++k) {
      double mn = CUDART_INF;
      for (int j = threadIdx.x; j < a.J; j += blockDim.x) mn = fmin(mn, a.emin[(long long)j * a.K + k]);
      s_d[threadIdx.x] = mn;
      __syncthreads();
      for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) s_d[threadIdx.x] = fmin(s_d[threadIdx.x], s_d[threadIdx.x + o]);
        __syncthreads();
      }
      if (threadIdx.x == 0) a.dom[k] = s_d[0];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      double mn = CUDART_INF;
      for (int k = 0; k < a.K; ++k) mn = fmin(mn, a.dom[k]);
      double s = 0.0;
      if (mn < CUDART_INF)
        for (int k = 0; k < a.K; ++k) s += exp(-(a.dom[k] - mn) / a.kT);
      a.dom[a.K] = mn;
      a.dom[a.K + 1] = mn < CUDART_INF ? mn - a.kT * (log(s) - log((double)a.K)) : CUDART_INF;
    }
  }
  if (threadIdx.x == 0 && a.dG) {
    double mx = -CUDART_INF;
    for (int k = 0; k < a.K; ++k) mx = fmax(mx, -a.bpmf[k] / a.kT);
    double s = 0.0;
    if (mx > -CUDART_INF)
      for (int k = 0; k < a.K; ++k) s += exp(-a.bpmf[k] / a.kT - mx);
    const double nmean = (double)ntot_all / ((double)a.J * a.K);
    a.dG[0] = (s > 0.0 && nmean > 0.0)
                  ? -a.kT * (mx + log(s) - log((double)a.K)) - a.kT * log(a.vsite_scale * nmean)
                  : CUDART_INF;
  }
}

cudaError_t launch_merge_pairs(const MergeArgs &a, cudaStream_t st) {
  const int JK = a.J * a.Kg;
  if (JK > 0) k_merge_pairs<<<(JK + 127) / 128, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_merge(const MergeArgs &a, cudaStream_t st) {
  k_merge<<<1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
__global__ void k_split_ff(const cx<ff> *spec, float2 *hi, float2 *lo, long long n) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  cx<ff> v = spec[i];
  hi[i] = make_float2(v.re.hi, v.im.hi);
  lo[i] = make_float2(v.re.lo, v.im.lo);
}

cudaError_t launch_split_ff(const void *spec, float2 *hi, float2 *lo, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_split_ff<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<const cx<ff> *>(spec), hi, lo, n);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// The receptor grids cropped to the box [c0, c0 + e) and zero-padded to the
// extents E >= e (CTA row blockIdx.y = channel t), with out null only summed:
//   out[t][i][j][l] = grid[t][c0_0 + i][c0_1 + j][c0_2 + l] (i, j, l < e), else 0,
// and the sum of squares of each channel's crop (the FP32 error bound of the
// refined form) in float pairs and in a fixed order, so that the bound, and
// with it the set of refined translations, is the same on every run: CTA b
// of channel t owns the (i, j) rows [b rpb, (b + 1) rpb), a warp one row at a
// time with its lanes along l; the warps' sums are added in order into
// part[t][b], and the last CTA to finish adds each channel's partials by a
// fixed tree and resets the counter.
__global__ void __launch_bounds__(256) k_crop_sq(const float *grid, int N0, int N1, int N2, int c00, int c01, int c02,
                                                 int e0, int e1, int e2, int E0, int E1, int E2, int rpb, float *out,
                                                 float2 *part, unsigned *count, float *sumsq) {
  __shared__ float s_h[256], s_l[256];
  __shared__ bool s_last;
  const int t = blockIdx.y, b = blockIdx.x, nb = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rows = E0 * E1;
  const int r1 = min((b + 1) * rpb, rows);
  ff acc{0.f, 0.f};
  for (int row = b * rpb + warp; row < r1; row += 8) {
    const int ix = row / E1, jy = row - ix * E1;
    const bool in = ix < e0 && jy < e1;
    const float *src = grid + (((long long)t * N0 + c00 + ix) * N1 + c01 + jy) * N2 + c02;
    float *dst = out ? out + (((long long)t * E0 + ix) * E1 + jy) * E2 : nullptr;
    for (int l = lane; l < E2; l += 32) {
      const float v = (in && l < e2) ? src[l] : 0.f;
      if (dst) dst[l] = v;
      acc = s_norm(s_add(acc, s_mul(ff{v, 0.f}, ff{v, 0.f})));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const ff other{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)};
    acc = s_norm(s_add(acc, other));
  }
  if (lane == 0) {
    s_h[warp] = acc.hi;
    s_l[warp] = acc.lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ff sum{0.f, 0.f};
    for (int w = 0; w < 8; ++w) sum = s_norm(s_add(sum, ff{s_h[w], s_l[w]}));
    part[t * nb + b] = make_float2(sum.hi, sum.lo);
    __threadfence();
    s_last = atomicAdd(count, 1u) == 3u * nb - 1u;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int c = 0; c < 3; ++c) {
    const float2 pv = threadIdx.x < nb ? __ldcg(&part[c * nb + threadIdx.x]) : make_float2(0.f, 0.f);
    s_h[threadIdx.x] = pv.x;
    s_l[threadIdx.x] = pv.y;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        const ff r = s_norm(s_add(ff{s_h[threadIdx.x], s_l[threadIdx.x]}, ff{s_h[threadIdx.x + o], s_l[threadIdx.x + o]}));
        s_h[threadIdx.x] = r.hi;
        s_l[threadIdx.x] = r.lo;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) sumsq[c] = __fadd_rn(s_h[0], s_l[0]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *count = 0u;  // for the next call on this scratch (stream order)
}

namespace {
// CTAs per channel: at most 255, so that the partials and the counter fit
// the kSumsqScratch float2 of scratch
constexpr int kCropSqBlocks = (kSumsqScratch - 1) / 3;

cudaError_t launch_crop_sq(const float *grid, const int N[3], const int c0[3], const int e[3], const int E[3],
                           float *out, float *sumsq, float2 *scratch, cudaStream_t st) {
  const int rows = E[0] * E[1];
  const int nb = std::max(1, std::min(kCropSqBlocks, (rows + 15) / 16));
  const int rpb = (rows + nb - 1) / nb;
  unsigned *count = reinterpret_cast<unsigned *>(scratch + kSumsqScratch - 1);
  cudaError_t err = cudaMemsetAsync(count, 0, sizeof(unsigned), st);
  if (err != cudaSuccess) return err;
  k_crop_sq<<<dim3(nb, 3), 256, 0, st>>>(grid, N[0], N[1], N[2], c0[0], c0[1], c0[2], e[0], e[1], e[2], E[0], E[1],
                                         E[2], rpb, out, scratch, count, sumsq);
  return cudaGetLastError();
}
}  // namespace

cudaError_t launch_crop(const float *grid, const int N[3], const int c0[3], const int e[3], const int E[3],
                        float *out, float *sumsq, float2 *scratch, cudaStream_t st) {
  for (int d = 0; d < 3; ++d)
    if (c0[d] < 0 || e[d] < 1 || c0[d] + e[d] > N[d] || E[d] < e[d]) return cudaErrorInvalidValue;
  // the padding adds zeros: the sums of squares of the padded crop are the crop's
  return launch_crop_sq(grid, N, c0, e, E, out, sumsq, scratch, st);
}

cudaError_t launch_sumsq(const float *g, const int N[3], float *out, float *sumsq, float2 *scratch, cudaStream_t st) {
  if ((long long)N[0] * N[1] * N[2] <= 0) return cudaMemsetAsync(sumsq, 0, 3 * sizeof(float), st);
  const int c0[3] = {0, 0, 0};
  return launch_crop_sq(g, N, c0, N, N, out, sumsq, scratch, st);
}

// explicit instantiations
template cudaError_t launch_zfwd<float>(const ZfwdArgs &, cudaStream_t);
template cudaError_t launch_zfwd<ff>(const ZfwdArgs &, cudaStream_t);
template cudaError_t launch_axis<float>(const AxisArgs &, cudaStream_t);
template cudaError_t launch_axis<ff>(const AxisArgs &, cudaStream_t);
template cudaError_t launch_xfused<float>(const XfusedArgs &, int, cudaStream_t);
template cudaError_t launch_xfused<ff>(const XfusedArgs &, int, cudaStream_t);
template cudaError_t launch_zinv<float>(const ZinvArgs &, int, cudaStream_t);
template cudaError_t launch_zinv<ff>(const ZinvArgs &, int, cudaStream_t);

}  // namespace bpmf
