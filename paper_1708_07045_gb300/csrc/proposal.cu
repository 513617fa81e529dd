// Learned proposal over ligand configurations: configuration features, a
// small MLP (bf16 tensor-core GEMMs, FP32 accumulation, FP32 master weights
// with Adam), the proposal q = mix * softmax(pred) + (1 - mix) / J sampled by
// inverse CDF on caller-supplied uniforms, and the importance-weighted FP64
// estimator of the BPMF (Eq. sample_mean_BPMF with configurations drawn from
// q instead of uniformly).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>

#include "proposal.cuh"

namespace bpmf {

// ----------------------------------------------------------------- features
// 3x3 symmetric eigen-decomposition by cyclic Jacobi (FP32, fixed sweeps).
__device__ void jacobi3(float a[3][3], float v[3][3], float w[3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) v[i][j] = i == j ? 1.f : 0.f;
  for (int sweep = 0; sweep < 12; ++sweep) {
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        const float apq = a[p][q];
        if (fabsf(apq) < 1e-30f) continue;
        const float theta = (a[q][q] - a[p][p]) / (2.f * apq);
        const float t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
        const float c = 1.f / sqrtf(t * t + 1.f), s = t * c;
        for (int k = 0; k < 3; ++k) {  // rotate columns p, q
          const float akp = a[k][p], akq = a[k][q];
          a[k][p] = c * akp - s * akq;
          a[k][q] = s * akp + c * akq;
        }
        for (int k = 0; k < 3; ++k) {  // rotate rows p, q
          const float apk = a[p][k], aqk = a[q][k];
          a[p][k] = c * apk - s * aqk;
          a[q][k] = s * apk + c * aqk;
        }
        for (int k = 0; k < 3; ++k) {
          const float vkp = v[k][p], vkq = v[k][q];
          v[k][p] = c * vkp - s * vkq;
          v[k][q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < 3; ++i) w[i] = a[i][i];
}

__device__ float dihedral(const float *a, const float *b, const float *c, const float *d, float *sn, float *cs) {
  float b1[3], b2[3], b3[3], n1[3], n2[3], m[3];
  for (int i = 0; i < 3; ++i) {
    b1[i] = b[i] - a[i];
    b2[i] = c[i] - b[i];
    b3[i] = d[i] - c[i];
  }
  n1[0] = b1[1] * b2[2] - b1[2] * b2[1];
  n1[1] = b1[2] * b2[0] - b1[0] * b2[2];
  n1[2] = b1[0] * b2[1] - b1[1] * b2[0];
  n2[0] = b2[1] * b3[2] - b2[2] * b3[1];
  n2[1] = b2[2] * b3[0] - b2[0] * b3[2];
  n2[2] = b2[0] * b3[1] - b2[1] * b3[0];
  const float lb2 = sqrtf(b2[0] * b2[0] + b2[1] * b2[1] + b2[2] * b2[2]) + 1e-30f;
  m[0] = (n1[1] * b2[2] - n1[2] * b2[1]) / lb2;
  m[1] = (n1[2] * b2[0] - n1[0] * b2[2]) / lb2;
  m[2] = (n1[0] * b2[1] - n1[1] * b2[0]) / lb2;
  const float x = n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2];
  const float y = m[0] * n2[0] + m[1] * n2[1] + m[2] * n2[2];
  const float r = sqrtf(x * x + y * y) + 1e-30f;
  *cs = x / r;
  *sn = y / r;
  return 0.f;
}

// One thread per configuration; layout of the 24 features is documented in
// include/bpmf.h (bpmf_features).
__global__ void k_features(const float *coords, const int *conf_off, const int *conf_nat, const int *conf_lig,
                           const float *q, const float *eps, const float *R, const int *lig_atom_off, int n_conf,
                           float h, float *out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_conf) return;
  const float *x = coords + 3ll * conf_off[j];
  const int n = conf_nat[j];
  const int li = conf_lig[j];
  float c[3] = {0.f, 0.f, 0.f}, lo[3] = {x[0], x[1], x[2]}, hi[3] = {x[0], x[1], x[2]};
  for (int i = 0; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      c[d] += x[3 * i + d];
      lo[d] = fminf(lo[d], x[3 * i + d]);
      hi[d] = fmaxf(hi[d], x[3 * i + d]);
    }
  for (int d = 0; d < 3; ++d) c[d] /= (float)n;
  float g[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};  // gyration tensor
  for (int i = 0; i < n; ++i) {
    float r[3] = {x[3 * i] - c[0], x[3 * i + 1] - c[1], x[3 * i + 2] - c[2]};
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) g[a][b] += r[a] * r[b];
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) g[a][b] /= (float)n;
  float v[3][3], w[3];
  jacobi3(g, v, w);
  // sort axes by moment, ascending
  int o[3] = {0, 1, 2};
  for (int a = 0; a < 2; ++a)
    for (int b = a + 1; b < 3; ++b)
      if (w[o[b]] < w[o[a]]) {
        int t = o[a];
        o[a] = o[b];
        o[b] = t;
      }
  float e[3][3];  // e[axis][component]
  for (int a = 0; a < 3; ++a)
    for (int d = 0; d < 3; ++d) e[a][d] = v[d][o[a]];
  // sign convention: positive third moment along the first two axes
  for (int a = 0; a < 2; ++a) {
    float m3 = 0.f;
    for (int i = 0; i < n; ++i) {
      const float p = (x[3 * i] - c[0]) * e[a][0] + (x[3 * i + 1] - c[1]) * e[a][1] + (x[3 * i + 2] - c[2]) * e[a][2];
      m3 += p * p * p;
    }
    if (m3 < 0.f)
      for (int d = 0; d < 3; ++d) e[a][d] = -e[a][d];
  }
  e[2][0] = e[0][1] * e[1][2] - e[0][2] * e[1][1];  // right-handed frame
  e[2][1] = e[0][2] * e[1][0] - e[0][0] * e[1][2];
  e[2][2] = e[0][0] * e[1][1] - e[0][1] * e[1][0];
  // rotation matrix M with columns e_a (principal frame -> lab) to quaternion
  const float m00 = e[0][0], m11 = e[1][1], m22 = e[2][2];
  const float m21 = e[1][2], m12 = e[2][1], m02 = e[2][0], m20 = e[0][2], m10 = e[0][1], m01 = e[1][0];
  float qw, qx, qy, qz;
  const float tr = m00 + m11 + m22;
  if (tr > 0.f) {
    const float s = sqrtf(tr + 1.f) * 2.f;
    qw = 0.25f * s;
    qx = (m21 - m12) / s;
    qy = (m02 - m20) / s;
    qz = (m10 - m01) / s;
  } else if (m00 > m11 && m00 > m22) {
    const float s = sqrtf(1.f + m00 - m11 - m22) * 2.f;
    qw = (m21 - m12) / s;
    qx = 0.25f * s;
    qy = (m01 + m10) / s;
    qz = (m02 + m20) / s;
  } else if (m11 > m22) {
    const float s = sqrtf(1.f + m11 - m00 - m22) * 2.f;
    qw = (m02 - m20) / s;
    qx = (m01 + m10) / s;
    qy = 0.25f * s;
    qz = (m12 + m21) / s;
  } else {
    const float s = sqrtf(1.f + m22 - m00 - m11) * 2.f;
    qw = (m10 - m01) / s;
    qx = (m02 + m20) / s;
    qy = (m12 + m21) / s;
    qz = 0.25f * s;
  }
  if (qw < 0.f) qw = -qw, qx = -qx, qy = -qy, qz = -qz;
  float *f = out + 24ll * j;
  f[0] = qw;
  f[1] = qx;
  f[2] = qy;
  f[3] = qz;
  for (int d = 0; d < 3; ++d) f[4 + d] = ceilf(__fdiv_rn(hi[d] - lo[d], h)) + 4.f;  // ligand-box extents (nodes)
  for (int a = 0; a < 3; ++a) f[7 + a] = w[o[a]];                                   // principal moments (A^2)
  f[10] = sqrtf(fmaxf(w[0] + w[1] + w[2], 0.f));                                     // radius of gyration
  {
    const float *a0 = x, *an = x + 3 * (n - 1);
    f[11] = sqrtf((an[0] - a0[0]) * (an[0] - a0[0]) + (an[1] - a0[1]) * (an[1] - a0[1]) +
                  (an[2] - a0[2]) * (an[2] - a0[2]));  // end-to-end distance
  }
  for (int k = 0; k < 2; ++k) {  // first two torsions (atoms 0-3, 1-4)
    float sn = 0.f, cs = 1.f;
    if (n >= 4 + k) dihedral(x + 3 * k, x + 3 * (k + 1), x + 3 * (k + 2), x + 3 * (k + 3), &sn, &cs);
    f[12 + 2 * k] = sn;
    f[13 + 2 * k] = cs;
  }
  for (int b = 0; b < 8; ++b) f[16 + b] = 0.f;  // atom-type counts: (R > 1.75, eps > 0.125, q > 0)
  const int a0 = lig_atom_off[li];
  for (int i = 0; i < n; ++i) {
    const int bin = (R[a0 + i] > 1.75f ? 4 : 0) + (eps[a0 + i] > 0.125f ? 2 : 0) + (q[a0 + i] > 0.f ? 1 : 0);
    f[16 + bin] += 1.f;
  }
}

cudaError_t launch_features(const float *coords, const int *conf_off, const int *conf_nat, const int *conf_lig,
                            const float *q, const float *eps, const float *R, const int *lig_atom_off, int n_conf,
                            float h, float *out, cudaStream_t st) {
  if (n_conf <= 0) return cudaSuccess;
  k_features<<<(n_conf + 127) / 128, 128, 0, st>>>(coords, conf_off, conf_nat, conf_lig, q, eps, R, lig_atom_off,
                                                   n_conf, h, out);
  return cudaGetLastError();
}

// --------------------------------------------------------------- bf16 GEMM
// C[m][n] = sum_k opA(A)[m][k] * B[k][n] (+ bias[n]) on the tensor cores:
// mma.sync m16n8k16 with bf16 operands rounded from FP32 memory and FP32
// accumulation.  Strides give transposed views; opA optionally applies ReLU
// (forward) or the ReLU derivative mask of Zmask (backward) while loading A.
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const unsigned *>(&v);
}

__device__ __forceinline__ float load_a(const GemmArgs &g, int m, int k) {
  if (m >= g.M || k >= g.K) return 0.f;
  float v = g.A[(long long)m * g.sam + (long long)k * g.sak];
  if (g.a_op == 1) v = fmaxf(v, 0.f);
  return v;
}
__device__ __forceinline__ float load_b(const GemmArgs &g, int k, int n) {
  if (k >= g.K || n >= g.N) return 0.f;
  return g.B[(long long)k * g.sbk + (long long)n * g.sbn];
}

// one warp per 16 x 8 output tile
__global__ void k_gemm_bf16(GemmArgs g) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = (g.N + 7) / 8;
  const int tm = warp / tiles_n, tn = warp % tiles_n;
  if (tm * 16 >= g.M) return;
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = tm * 16, n0 = tn * 8;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  for (int k0 = 0; k0 < g.K; k0 += 16) {
    const int kc = k0 + tig * 2;
    const unsigned a0 = pack_bf16(load_a(g, m0 + gid, kc), load_a(g, m0 + gid, kc + 1));
    const unsigned a1 = pack_bf16(load_a(g, m0 + gid + 8, kc), load_a(g, m0 + gid + 8, kc + 1));
    const unsigned a2 = pack_bf16(load_a(g, m0 + gid, kc + 8), load_a(g, m0 + gid, kc + 9));
    const unsigned a3 = pack_bf16(load_a(g, m0 + gid + 8, kc + 8), load_a(g, m0 + gid + 8, kc + 9));
    const unsigned b0 = pack_bf16(load_b(g, kc, n0 + gid), load_b(g, kc + 1, n0 + gid));
    const unsigned b1 = pack_bf16(load_b(g, kc + 8, n0 + gid), load_b(g, kc + 9, n0 + gid));
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  const int r0 = m0 + gid, r1 = m0 + gid + 8, cc = n0 + tig * 2;
  const float acc[4] = {c0, c1, c2, c3};
  const int rows[4] = {r0, r0, r1, r1}, cols[4] = {cc, cc + 1, cc, cc + 1};
  for (int i = 0; i < 4; ++i)
    if (rows[i] < g.M && cols[i] < g.N) {
      float v = acc[i] + (g.bias ? g.bias[cols[i]] : 0.f);
      g.C[(long long)rows[i] * g.scm + cols[i]] = g.accumulate ? g.C[(long long)rows[i] * g.scm + cols[i]] + v : v;
    }
}

cudaError_t launch_gemm_bf16(const GemmArgs &g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  const long long warps = (long long)((g.M + 15) / 16) * ((g.N + 7) / 8);
  const int threads = 128;
  k_gemm_bf16<<<(unsigned)((warps * 32 + threads - 1) / threads), threads, 0, st>>>(g);
  return cudaGetLastError();
}

// ------------------------------------------------------------- elementwise
// loss = mean (y - t)^2 over B rows; dy = 2 (y - t) / B
__global__ void k_mse(const float *y, const float *t, int B, float *dy, float *loss) {
  __shared__ float s[256];
  float acc = 0.f;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / (float)B;
    acc += d * d;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = s[0] / (float)B;
}

// column sums of dZ (optionally masked by Z > 0): bias gradients
__global__ void k_colsum(const float *D, const float *Z, int B, int N, float *out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float acc = 0.f;
  for (int i = 0; i < B; ++i) {
    const float d = D[(long long)i * N + n];
    if (!Z || Z[(long long)i * N + n] > 0.f) acc += d;
  }
  out[n] = acc;
}

// Adam on the FP32 master parameters
__global__ void k_adam(float *w, const float *gw, float *m, float *v, long long n, float lr, float b1, float b2,
                       float epsl, float bc1, float bc2) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gw[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + epsl);
}

// dZ = dA * (Z > 0), in place
__global__ void k_mask_relu_grad(float *D, const float *Z, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && Z[i] <= 0.f) D[i] = 0.f;
}

// out[b][j] = (x[b][j] - shift[j]) / scale[j]   (invert: x * scale + shift)
__global__ void k_affine(const float *x, const float *shift, const float *scale, int B, int N, int invert,
                         float *out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)B * N) return;
  const int j = (int)(i % N);
  out[i] = invert ? x[i] * scale[j] + shift[j] : (x[i] - shift[j]) / scale[j];
}

cudaError_t launch_mask_relu_grad(float *D, const float *Z, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_mask_relu_grad<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(D, Z, n);
  return cudaGetLastError();
}
cudaError_t launch_affine(const float *x, const float *shift, const float *scale, int B, int N, int invert, float *out,
                          cudaStream_t st) {
  const long long n = (long long)B * N;
  if (n <= 0) return cudaSuccess;
  k_affine<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, shift, scale, B, N, invert, out);
  return cudaGetLastError();
}

cudaError_t launch_mse(const float *y, const float *t, int B, float *dy, float *loss, cudaStream_t st) {
  k_mse<<<1, 256, 0, st>>>(y, t, B, dy, loss);
  return cudaGetLastError();
}
cudaError_t launch_colsum(const float *D, const float *Z, int B, int N, float *out, cudaStream_t st) {
  k_colsum<<<(N + 127) / 128, 128, 0, st>>>(D, Z, B, N, out);
  return cudaGetLastError();
}
cudaError_t launch_adam(float *w, const float *gw, float *m, float *v, long long n, float lr, float b1, float b2,
                        float epsl, float bc1, float bc2, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_adam<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, gw, m, v, n, lr, b1, b2, epsl, bc1, bc2);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- proposal
// q_j = mix * softmax(pred / tau)_j + (1 - mix) / J in FP64; cumulative sums;
// then index_s = first j with cdf_j > u_s (inverse CDF of caller-supplied
// uniforms).
__global__ void k_proposal(const float *pred, int J, double mix, double tau, const double *u, int M, double *q,
                           double *cdf, int *idx, double *q_s) {
  __shared__ double s_d[256];
  // max
  double mx = -CUDART_INF;
  for (int j = threadIdx.x; j < J; j += blockDim.x) mx = fmax(mx, (double)pred[j] / tau);
  s_d[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + o]);
    __syncthreads();
  }
  const double M0 = s_d[0];
  __syncthreads();
  double acc = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) acc += exp((double)pred[j] / tau - M0);
  s_d[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
    __syncthreads();
  }
  const double Zs = s_d[0];
  for (int j = threadIdx.x; j < J; j += blockDim.x)
    q[j] = mix * exp((double)pred[j] / tau - M0) / Zs + (1.0 - mix) / J;
  __syncthreads();
  if (threadIdx.x == 0) {  // sequential prefix sum: deterministic, J is modest
    double c = 0.0;
    for (int j = 0; j < J; ++j) {
      c += q[j];
      cdf[j] = c;
    }
  }
  __syncthreads();
  const double total = cdf[J - 1];
  for (int s = threadIdx.x; s < M; s += blockDim.x) {
    const double x = u[s] * total;
    int lo = 0, hi = J - 1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cdf[mid] > x) hi = mid;
      else lo = mid + 1;
    }
    idx[s] = lo;
    q_s[s] = q[lo] / total;
  }
}

cudaError_t launch_proposal(const float *pred, int J, double mix, double tau, const double *u, int M, double *q,
                            double *cdf, int *idx, double *q_s, cudaStream_t st) {
  k_proposal<<<1, 256, 0, st>>>(pred, J, mix, tau, u, M, q, cdf, idx, q_s);
  return cudaGetLastError();
}

// Training targets of the proposal for one ligand (FP64 log-sum-exp over
// receptors, Eq. sample_mean_BPMF's per-configuration weight):
//   ls_j = ln sum_k n_jk exp(log Z_jk)   (-inf without a valid translation)
//   t_j  = max(ls_j - max_j' ls_j', -clip)
// The proposal only needs the ranking within a ligand; the offset between
// ligands and the tail below -clip carry no information for it.
__global__ void k_config_targets(const double *logZ, const long long *n_valid, int J, int K, double clip,
                                 double *ls, float *t) {
  __shared__ double s_d[256];
  double mx = -CUDART_INF;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    double m = -CUDART_INF;
    for (int k = 0; k < K; ++k)
      if (n_valid[(long long)j * K + k] > 0)
        m = fmax(m, logZ[(long long)j * K + k] + log((double)n_valid[(long long)j * K + k]));
    double v = -CUDART_INF;
    if (m > -CUDART_INF) {
      double acc = 0.0;
      for (int k = 0; k < K; ++k)
        if (n_valid[(long long)j * K + k] > 0)
          acc += exp(logZ[(long long)j * K + k] + log((double)n_valid[(long long)j * K + k]) - m);
      v = m + log(acc);
    }
    ls[j] = v;
    mx = fmax(mx, v);
  }
  s_d[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + o]);
    __syncthreads();
  }
  const double M0 = s_d[0];
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    const double v = ls[j];
    t[j] = (float)((M0 > -CUDART_INF && v > -CUDART_INF) ? fmax(v - M0, -clip) : -clip);
  }
}

cudaError_t launch_config_targets(const double *logZ, const long long *n_valid, int J, int K, double clip, double *ls,
                                  float *t, cudaStream_t st) {
  k_config_targets<<<1, 256, 0, st>>>(logZ, n_valid, J, K, clip, ls, t);
  return cudaGetLastError();
}

// Exact relative variance of the importance-sampling estimate of
// Z = sum_j S_j from one draw of q (FP64):  chi2 = sum_j S_j^2 / (q_j Z^2) - 1,
// with q_j = mix softmax(pred / tau)_j + (1 - mix) / J and S_j = exp(ls_j)
// (-inf: S_j = 0).  M independent draws have relative variance chi2 / M.
__global__ void k_proposal_chi2(const float *pred, const double *ls, int J, double mix, double tau, double *out) {
  __shared__ double s_d[256], s_e[256];
  double mp = -CUDART_INF, ms = -CUDART_INF;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    mp = fmax(mp, (double)pred[j] / tau);
    ms = fmax(ms, ls[j]);
  }
  s_d[threadIdx.x] = mp;
  s_e[threadIdx.x] = ms;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + o]);
      s_e[threadIdx.x] = fmax(s_e[threadIdx.x], s_e[threadIdx.x + o]);
    }
    __syncthreads();
  }
  const double MP = s_d[0], MS = s_e[0];
  __syncthreads();
  double zp = 0.0, zs = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    zp += exp((double)pred[j] / tau - MP);
    if (ls[j] > -CUDART_INF) zs += exp(ls[j] - MS);
  }
  s_d[threadIdx.x] = zp;
  s_e[threadIdx.x] = zs;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s_d[threadIdx.x] += s_d[threadIdx.x + o];
      s_e[threadIdx.x] += s_e[threadIdx.x + o];
    }
    __syncthreads();
  }
  const double ZP = s_d[0], ZS = s_e[0];
  __syncthreads();
  double acc = 0.0;
  for (int j = threadIdx.x; j < J; j += blockDim.x) {
    if (!(ls[j] > -CUDART_INF)) continue;
    const double q = mix * exp((double)pred[j] / tau - MP) / ZP + (1.0 - mix) / J;
    const double w = exp(ls[j] - MS) / ZS;
    acc += w * w / q;
  }
  s_d[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = ZS > 0.0 ? s_d[0] - 1.0 : CUDART_INF;
}

cudaError_t launch_proposal_chi2(const float *pred, const double *ls, int J, double mix, double tau, double *out,
                                 cudaStream_t st) {
  k_proposal_chi2<<<1, 256, 0, st>>>(pred, ls, J, mix, tau, out);
  return cudaGetLastError();
}

// Importance-weighted BPMF per receptor (FP64):
//   Z_k ~ (1/M) sum_s S_{j_s k} / q_{j_s},  S = exp(logZ + ln n)
//   B_k = -kT [ ln Z_k - ln N_k ],  N_k = total valid translations of all J
__global__ void k_is_estimate(const double *logZ_s, const long long *n_s, const double *q_s, int M, int K,
                              const long long *n_tot, double kT, double *bpmf) {
  __shared__ double s_d[256];
  for (int k = 0; k < K; ++k) {
    double mx = -CUDART_INF;
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
      const long long n = n_s[(long long)s * K + k];
      if (n > 0) mx = fmax(mx, logZ_s[(long long)s * K + k] + log((double)n) - log(q_s[s]));
    }
    s_d[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + o]);
      __syncthreads();
    }
    const double M0 = s_d[0];
    __syncthreads();
    double acc = 0.0;
    if (M0 > -CUDART_INF)
      for (int s = threadIdx.x; s < M; s += blockDim.x) {
        const long long n = n_s[(long long)s * K + k];
        if (n > 0) acc += exp(logZ_s[(long long)s * K + k] + log((double)n) - log(q_s[s]) - M0);
      }
    s_d[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0)
      bpmf[k] = (s_d[0] > 0.0 && n_tot[k] > 0) ? -kT * (M0 + log(s_d[0] / M) - log((double)n_tot[k])) : CUDART_INF;
    __syncthreads();
  }
}

cudaError_t launch_is_estimate(const double *logZ_s, const long long *n_s, const double *q_s, int M, int K,
                               const long long *n_tot, double kT, double *bpmf, cudaStream_t st) {
  k_is_estimate<<<1, 256, 0, st>>>(logZ_s, n_s, q_s, M, K, n_tot, kT, bpmf);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Sampling importance resampling of poses with weight exp(-E / kT) (FP64).
// The draw over all (configuration, translation) poses of one receptor is
// taken exactly in two stages: the configuration j with probability
// S_j / sum_j S_j (S_j = n_j exp(log Z_j), the sum of exp(-E/kT) over j's
// valid translations), then, within j, the translation with probability
// exp(-E_s / kT) / S_j.  Each stage is an inverse CDF on caller uniforms:
// the first index whose cumulative weight exceeds u * total.
//
// Cumulative weights: thread t owns the contiguous chunk [t C, (t+1) C) of
// the n weights; chunk sums, their exclusive prefix (thread 0, in order),
// then every thread writes its chunk's prefix.  The order of additions is
// fixed, so draws are deterministic.
template <class W>
__device__ double block_cdf(int n, W weight, double *cdf, double *s_d) {
  const int C = (n + blockDim.x - 1) / blockDim.x;
  const int b = threadIdx.x * C, e = min(n, b + C);
  double acc = 0.0;
  for (int i = b; i < e; ++i) acc += weight(i);
  s_d[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double c = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      const double v = s_d[t];
      s_d[t] = c;
      c += v;
    }
  }
  __syncthreads();
  double c = s_d[threadIdx.x];
  for (int i = b; i < e; ++i) {
    c += weight(i);
    cdf[i] = c;
  }
  __syncthreads();
  return cdf[n - 1];
}

__device__ int inverse_cdf(const double *cdf, int n, double x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cdf[mid] > x) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__device__ double block_max(double v, double *s_d) {
  s_d[threadIdx.x] = v;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] = fmax(s_d[threadIdx.x], s_d[threadIdx.x + o]);
    __syncthreads();
  }
  const double r = s_d[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(256) k_sir_configs(const double *logZ, const long long *nvalid, int J, int K, int k,
                                                     const double *u, int M, double *cdf, int *conf) {
  __shared__ double s_d[256];
  auto logS = [&](int j) {
    const long long n = nvalid[(long long)j * K + k];
    return n > 0 ? logZ[(long long)j * K + k] + log((double)n) : -CUDART_INF;
  };
  double mx = -CUDART_INF;
  for (int j = threadIdx.x; j < J; j += blockDim.x) mx = fmax(mx, logS(j));
  const double M0 = block_max(mx, s_d);
  double total = 0.0;
  if (M0 > -CUDART_INF)
    total = block_cdf(J, [&](int j) {
      const double v = logS(j);
      return v > -CUDART_INF ? exp(v - M0) : 0.0;
    }, cdf, s_d);
  for (int s = threadIdx.x; s < M; s += blockDim.x) conf[s] = total > 0.0 ? inverse_cdf(cdf, J, u[s] * total) : -1;
}

__global__ void __launch_bounds__(256) k_sir_translations(const double *E, int nS, double kT, const double *u,
                                                          const int *conf, int j, int M, double *cdf, int *pick) {
  __shared__ double s_d[256];
  double mx = -CUDART_INF;
  for (int i = threadIdx.x; i < nS; i += blockDim.x) mx = fmax(mx, -E[i] / kT);
  const double M0 = block_max(mx, s_d);
  double total = 0.0;
  if (M0 > -CUDART_INF)
    total = block_cdf(nS, [&](int i) {
      const double v = -E[i] / kT;
      return v > -CUDART_INF ? exp(v - M0) : 0.0;
    }, cdf, s_d);
  for (int s = threadIdx.x; s < M; s += blockDim.x)
    if (conf[s] == j) pick[s] = total > 0.0 ? inverse_cdf(cdf, nS, u[s] * total) : -1;
}

cudaError_t launch_sir_configs(const double *logZ, const long long *nvalid, int J, int K, int k, const double *u,
                               int M, double *cdf, int *conf, cudaStream_t st) {
  if (J <= 0 || M <= 0) return cudaSuccess;
  k_sir_configs<<<1, 256, 0, st>>>(logZ, nvalid, J, K, k, u, M, cdf, conf);
  return cudaGetLastError();
}

cudaError_t launch_sir_translations(const double *E, int nS, double kT, const double *u, const int *conf, int j, int M,
                                    double *cdf, int *pick, cudaStream_t st) {
  if (nS <= 0 || M <= 0) return cudaSuccess;
  k_sir_translations<<<1, 256, 0, st>>>(E, nS, kT, u, conf, j, M, cdf, pick);
  return cudaGetLastError();
}

// --------------------------------------------------------------------------
// Bootstrap of the pooled BPMF and the standard binding free energy over
// configurations (FP64).  Replicate r fills its J slots with configurations
// j = min(J - 1, floor(u J)) and evaluates, per receptor k,
//   B_k = -kT [ln sum_slots S_jk - ln sum_slots n_jk],  S = n exp(log Z),
// then dG = -kT ln((1/K) sum_k exp(-B_k / kT)) - kT ln(h^3 C mean n) as the
// full estimate does.  One CTA per replicate; rep [R][K + 1].
__global__ void __launch_bounds__(256) k_bootstrap(const double *logZ, const long long *nvalid, int J, int K, double kT,
                                                   double vscale, const double *u, int R, double *rep) {
  __shared__ double s_d[256];
  __shared__ long long s_l[256];
  const int r = blockIdx.x;
  const double *ur = u + (long long)r * J;
  double *out = rep + (long long)r * (K + 1);
  long long ntot_all = 0;
  for (int k = 0; k < K; ++k) {
    double mx = -CUDART_INF;
    long long nt = 0;
    for (int i = threadIdx.x; i < J; i += blockDim.x) {
      const int j = min(J - 1, (int)floor(ur[i] * (double)J));
      const long long n = nvalid[(long long)j * K + k];
      if (n > 0) mx = fmax(mx, logZ[(long long)j * K + k] + log((double)n));
      nt += n;
    }
    const double M = block_max(mx, s_d);
    s_l[threadIdx.x] = nt;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s_l[threadIdx.x] += s_l[threadIdx.x + o];
      __syncthreads();
    }
    const long long ntot = s_l[0];
    __syncthreads();
    double acc = 0.0;
    if (M > -CUDART_INF)
      for (int i = threadIdx.x; i < J; i += blockDim.x) {
        const int j = min(J - 1, (int)floor(ur[i] * (double)J));
        const long long n = nvalid[(long long)j * K + k];
        if (n > 0) {
          const double v = logZ[(long long)j * K + k] + log((double)n);
          if (v > -CUDART_INF) acc += exp(v - M);
        }
      }
    s_d[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0)
      out[k] = (ntot > 0 && s_d[0] > 0.0) ? -kT * (M + log(s_d[0]) - log((double)ntot)) : CUDART_INF;
    ntot_all += ntot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double mx = -CUDART_INF;
    for (int k = 0; k < K; ++k) mx = fmax(mx, -out[k] / kT);
    double s = 0.0;
    if (mx > -CUDART_INF)
      for (int k = 0; k < K; ++k) s += exp(-out[k] / kT - mx);
    const double nmean = (double)ntot_all / ((double)J * K);
    out[K] = (s > 0.0 && nmean > 0.0) ? -kT * (mx + log(s) - log((double)K)) - kT * log(vscale * nmean) : CUDART_INF;
  }
}

// Mean and sample standard deviation (ddof 1) of every column of rep.
__global__ void __launch_bounds__(256) k_bootstrap_stats(const double *rep, int R, int C, double *stats) {
  __shared__ double s_d[256];
  const int c = blockIdx.x;
  double acc = 0.0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) acc += rep[(long long)r * C + c];
  s_d[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
    __syncthreads();
  }
  const double mean = s_d[0] / R;
  __syncthreads();
  acc = 0.0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double d = rep[(long long)r * C + c] - mean;
    acc += d * d;
  }
  s_d[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[c] = mean;
    stats[C + c] = R > 1 ? sqrt(s_d[0] / (R - 1)) : 0.0;
  }
}

cudaError_t launch_bootstrap(const double *logZ, const long long *nvalid, int J, int K, double kT, double vscale,
                             const double *u, int R, double *rep, double *stats, cudaStream_t st) {
  if (R <= 0 || J <= 0) return cudaSuccess;
  k_bootstrap<<<R, 256, 0, st>>>(logZ, nvalid, J, K, kT, vscale, u, R, rep);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !stats) return e;
  k_bootstrap_stats<<<K + 1, 256, 0, st>>>(rep, R, K + 1, stats);
  return cudaGetLastError();
}

}  // namespace bpmf
