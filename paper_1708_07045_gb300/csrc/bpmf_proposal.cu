// C-ABI layer of the learned proposal: features, the MLP handle (forward,
// training step with Adam), proposal sampling and the importance-weighted
// BPMF.  Host-side orchestration only; the arithmetic runs in proposal.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/bpmf.h"
#include "proposal.cuh"

using namespace bpmf;

// Parts of the library's handles this layer reads (layouts defined in
// bpmf_api.cu, exported there through accessors).
extern "C++" {
int bpmf_internal_device(bpmf_ctx_t c);
void bpmf_internal_set_error(bpmf_ctx_t c, const std::string &msg);
int bpmf_internal_ligand_arrays(bpmf_lig_t lg, const float **coords, const float **q, const float **eps,
                                const float **R, std::vector<int> *conf_off, std::vector<int> *conf_nat,
                                std::vector<int> *conf_lig, std::vector<int> *lig_atom_off);
}

struct bpmf_mlp {
  bpmf_ctx_t ctx = nullptr;
  int n_in = 0, width = 0, depth = 0;
  long long n_params = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // packed, device
  float *norm = nullptr;                                          // x_shift[n_in] x_scale[n_in] y_shift y_scale
  long long step = 0;
  std::vector<long long> off_w, off_b;  // per layer
  std::vector<int> in, out;
};

namespace {

struct PFail {
  int code;
};

#define PCK(call)                                                             \
  do {                                                                        \
    const cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess) {                                                  \
      msg = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      throw PFail{e_ == cudaErrorMemoryAllocation ? BPMF_ERR_OOM : BPMF_ERR_CUDA}; \
    }                                                                         \
  } while (0)

thread_local std::string msg;

struct Dev {
  int prev = -1;
  explicit Dev(int d) {
    cudaGetDevice(&prev);
    if (prev != d) cudaSetDevice(d);
  }
  ~Dev() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int fail(bpmf_ctx_t c, int code) {
  if (c) bpmf_internal_set_error(c, msg);
  return code;
}

GemmArgs gemm(const float *A, long long sam, long long sak, int a_op, const float *B, long long sbk, long long sbn,
              float *C, long long scm, const float *bias, int M, int N, int K) {
  GemmArgs g{};
  g.A = A;
  g.sam = sam;
  g.sak = sak;
  g.a_op = a_op;
  g.B = B;
  g.sbk = sbk;
  g.sbn = sbn;
  g.C = C;
  g.scm = scm;
  g.bias = bias;
  g.M = M;
  g.N = N;
  g.K = K;
  return g;
}

// forward through the layers; Z[l] holds layer l's pre-activations [B][out_l]
void forward(bpmf_mlp *net, const float *Xn, int B, std::vector<float *> &Z, cudaStream_t st) {
  const int L = (int)net->in.size();
  for (int l = 0; l < L; ++l) {
    const float *A = l == 0 ? Xn : Z[l - 1];
    const int K = net->in[l], N = net->out[l];
    PCK(launch_gemm_bf16(gemm(A, K, 1, l == 0 ? 0 : 1, net->w + net->off_w[l], N, 1, Z[l], N,
                              net->w + net->off_b[l], B, N, K),
                         st));
  }
}

}  // namespace

extern "C" {

int bpmf_features(bpmf_ctx_t c, bpmf_lig_t lg, double h, float *out, void *stream) {
  if (!c || !lg || !out || !(h > 0.0)) return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  cudaStream_t st = (cudaStream_t)stream;
  int *d_tab = nullptr;
  float *d_out = nullptr;
  try {
    const float *coords, *q, *eps, *R;
    std::vector<int> off, nat, lig, aoff;
    if (bpmf_internal_ligand_arrays(lg, &coords, &q, &eps, &R, &off, &nat, &lig, &aoff) != BPMF_OK) {
      msg = "invalid ligand batch";
      throw PFail{BPMF_ERR_INVALID_ARG};
    }
    const int n = (int)off.size();
    if (n == 0) return BPMF_OK;
    std::vector<int> tab;
    tab.insert(tab.end(), off.begin(), off.end());
    tab.insert(tab.end(), nat.begin(), nat.end());
    tab.insert(tab.end(), lig.begin(), lig.end());
    tab.insert(tab.end(), aoff.begin(), aoff.end());
    PCK(cudaMallocAsync(&d_tab, sizeof(int) * tab.size(), st));
    PCK(cudaMemcpyAsync(d_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, st));
    cudaPointerAttributes at;
    const bool dev_out = cudaPointerGetAttributes(&at, out) == cudaSuccess &&
                         (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev_out) {
      d_out = out;
    } else {
      PCK(cudaMallocAsync(&d_out, sizeof(float) * kFeatures * n, st));
    }
    PCK(launch_features(coords, d_tab, d_tab + n, d_tab + 2 * n, q, eps, R, d_tab + 3 * n, n, (float)h, d_out, st));
    if (!dev_out) {
      PCK(cudaMemcpyAsync(out, d_out, sizeof(float) * kFeatures * n, cudaMemcpyDeviceToHost, st));
      PCK(cudaFreeAsync(d_out, st));
      d_out = nullptr;
    }
    PCK(cudaFreeAsync(d_tab, st));
    d_tab = nullptr;
    PCK(cudaStreamSynchronize(st));
  } catch (PFail f) {
    if (d_tab) cudaFreeAsync(d_tab, st);
    if (d_out && d_out != out) cudaFreeAsync(d_out, st);
    return fail(c, f.code);
  }
  return BPMF_OK;
}

long long bpmf_mlp_param_count(int n_in, int width, int depth) {
  if (n_in < 1 || width < 1 || depth < 1) return 0;
  return (long long)n_in * width + width + (long long)(depth - 1) * (width * (long long)width + width) + width + 1;
}

int bpmf_mlp_create(bpmf_ctx_t c, int n_in, int width, int depth, const float *params, const float *norm,
                    bpmf_mlp_t *out) {
  if (!c || !params || !norm || !out || n_in < 1 || width < 1 || depth < 1 || width > 1024)
    return BPMF_ERR_INVALID_ARG;
  *out = nullptr;
  Dev dv(bpmf_internal_device(c));
  bpmf_mlp *net = new (std::nothrow) bpmf_mlp();
  if (!net) return BPMF_ERR_OOM;
  try {
    net->ctx = c;
    net->n_in = n_in;
    net->width = width;
    net->depth = depth;
    long long o = 0;
    for (int l = 0; l <= depth; ++l) {
      const int fi = l == 0 ? n_in : width, fo = l == depth ? 1 : width;
      net->in.push_back(fi);
      net->out.push_back(fo);
      net->off_w.push_back(o);
      o += (long long)fi * fo;
      net->off_b.push_back(o);
      o += fo;
    }
    net->n_params = o;
    const size_t bytes = sizeof(float) * o;
    PCK(cudaMalloc(&net->w, bytes));
    PCK(cudaMalloc(&net->g, bytes));
    PCK(cudaMalloc(&net->m, bytes));
    PCK(cudaMalloc(&net->v, bytes));
    PCK(cudaMalloc(&net->norm, sizeof(float) * (2 * n_in + 2)));
    PCK(cudaMemcpy(net->w, params, bytes, cudaMemcpyHostToDevice));
    PCK(cudaMemset(net->m, 0, bytes));
    PCK(cudaMemset(net->v, 0, bytes));
    PCK(cudaMemcpy(net->norm, norm, sizeof(float) * (2 * n_in + 2), cudaMemcpyHostToDevice));
  } catch (PFail f) {
    bpmf_mlp_free(net);
    return fail(c, f.code);
  }
  *out = net;
  return BPMF_OK;
}

void bpmf_mlp_free(bpmf_mlp_t net) {
  if (!net) return;
  Dev dv(bpmf_internal_device(net->ctx));
  for (float *p : {net->w, net->g, net->m, net->v, net->norm})
    if (p) cudaFree(p);
  delete net;
}

int bpmf_mlp_get_params(bpmf_mlp_t net, float *params) {
  if (!net || !params) return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(net->ctx));
  if (cudaMemcpy(params, net->w, sizeof(float) * net->n_params, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return BPMF_ERR_CUDA;
  }
  return BPMF_OK;
}

int bpmf_mlp_forward(bpmf_ctx_t c, bpmf_mlp_t net, const float *X, int B, float *y, void *stream) {
  if (!c || !net || !X || !y || B < 0) return BPMF_ERR_INVALID_ARG;
  if (B == 0) return BPMF_OK;
  Dev dv(bpmf_internal_device(c));
  cudaStream_t st = (cudaStream_t)stream;
  float *buf = nullptr;
  try {
    const int L = (int)net->in.size();
    const size_t nx = (size_t)B * net->n_in, nz = (size_t)B * net->width;
    PCK(cudaMallocAsync(&buf, sizeof(float) * (nx + nz * (L - 1) + B), st));
    float *Xn = buf;
    std::vector<float *> Z(L);
    for (int l = 0; l < L - 1; ++l) Z[l] = buf + nx + nz * l;
    Z[L - 1] = buf + nx + nz * (L - 1);
    PCK(launch_affine(X, net->norm, net->norm + net->n_in, B, net->n_in, 0, Xn, st));
    forward(net, Xn, B, Z, st);
    PCK(launch_affine(Z[L - 1], net->norm + 2 * net->n_in, net->norm + 2 * net->n_in + 1, B, 1, 1, y, st));
    PCK(cudaFreeAsync(buf, st));
    buf = nullptr;
  } catch (PFail f) {
    if (buf) cudaFreeAsync(buf, st);
    return fail(c, f.code);
  }
  return BPMF_OK;
}

int bpmf_mlp_train_step(bpmf_ctx_t c, bpmf_mlp_t net, const float *X, const float *t, int B, float lr, int apply,
                        float *loss, float *grads, void *stream) {
  if (!c || !net || !X || !t || B < 1) return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  cudaStream_t st = (cudaStream_t)stream;
  float *buf = nullptr;
  try {
    const int L = (int)net->in.size();
    const int W = net->width;
    const size_t nx = (size_t)B * net->n_in, nz = (size_t)B * W;
    // Xn | Z[0..L-2] | y | tn | dy | dA (2 ping-pong) | loss
    const size_t total = nx + nz * (L - 1) + 3 * (size_t)B + 2 * nz + 1;
    PCK(cudaMallocAsync(&buf, sizeof(float) * total, st));
    float *Xn = buf, *p = buf + nx;
    std::vector<float *> Z(L);
    for (int l = 0; l < L - 1; ++l, p += nz) Z[l] = p;
    Z[L - 1] = p;
    p += B;
    float *tn = p;
    p += B;
    float *dy = p;
    p += B;
    float *dA[2] = {p, p + nz};
    p += 2 * nz;
    float *d_loss = p;
    const float *ysh = net->norm + 2 * net->n_in;
    PCK(launch_affine(X, net->norm, net->norm + net->n_in, B, net->n_in, 0, Xn, st));
    PCK(launch_affine(t, ysh, ysh + 1, B, 1, 0, tn, st));
    forward(net, Xn, B, Z, st);
    PCK(launch_mse(Z[L - 1], tn, B, dy, d_loss, st));
    // backward: dZ of the output layer is dy
    const float *dZ = dy;
    for (int l = L - 1; l >= 0; --l) {
      const int K = net->in[l], N = net->out[l];
      const float *Ain = l == 0 ? Xn : Z[l - 1];
      // dW_l = act(A_in)^T dZ   [K x N]
      PCK(launch_gemm_bf16(gemm(Ain, 1, K, l == 0 ? 0 : 1, dZ, N, 1, net->g + net->off_w[l], N, nullptr, K, N, B),
                           st));
      PCK(launch_colsum(dZ, nullptr, B, N, net->g + net->off_b[l], st));
      if (l > 0) {
        // dA_{l-1} = dZ W_l^T   [B x K], then dZ_{l-1} = dA * (Z_{l-1} > 0)
        float *dAn = dA[l & 1];
        PCK(launch_gemm_bf16(gemm(dZ, N, 1, 0, net->w + net->off_w[l], 1, N, dAn, K, nullptr, B, K, N), st));
        PCK(launch_mask_relu_grad(dAn, Z[l - 1], (long long)B * K, st));
        dZ = dAn;
      }
    }
    if (grads) PCK(cudaMemcpyAsync(grads, net->g, sizeof(float) * net->n_params, cudaMemcpyDefault, st));
    if (apply) {
      net->step += 1;
      const float b1 = 0.9f, b2 = 0.999f;
      const float bc1 = 1.f - powf(b1, (float)net->step), bc2 = 1.f - powf(b2, (float)net->step);
      PCK(launch_adam(net->w, net->g, net->m, net->v, net->n_params, lr, b1, b2, 1e-8f, bc1, bc2, st));
    }
    if (loss) PCK(cudaMemcpyAsync(loss, d_loss, sizeof(float), cudaMemcpyDefault, st));
    PCK(cudaFreeAsync(buf, st));
    buf = nullptr;
    PCK(cudaStreamSynchronize(st));
  } catch (PFail f) {
    if (buf) cudaFreeAsync(buf, st);
    return fail(c, f.code);
  }
  return BPMF_OK;
}

int bpmf_proposal_sample(bpmf_ctx_t c, const float *pred, int J, double mix, double tau, const double *u, int M,
                         int *idx, double *q_s, void *stream) {
  if (!c || !pred || !u || !idx || !q_s || J < 1 || M < 0 || !(mix >= 0.0 && mix <= 1.0) || !(tau > 0.0))
    return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  cudaStream_t st = (cudaStream_t)stream;
  double *buf = nullptr;
  try {
    PCK(cudaMallocAsync(&buf, sizeof(double) * 2 * J, st));
    PCK(launch_proposal(pred, J, mix, tau, u, M, buf, buf + J, idx, q_s, st));
    PCK(cudaFreeAsync(buf, st));
  } catch (PFail f) {
    if (buf) cudaFreeAsync(buf, st);
    return fail(c, f.code);
  }
  return BPMF_OK;
}

int bpmf_config_targets(bpmf_ctx_t c, const double *logZ, const int64_t *n_valid, int J, int K, double clip,
                        double *ls, float *t, void *stream) {
  if (!c || !logZ || !n_valid || !ls || !t || J < 1 || K < 1 || !(clip > 0.0)) return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  try {
    PCK(launch_config_targets(logZ, reinterpret_cast<const long long *>(n_valid), J, K, clip, ls, t,
                              (cudaStream_t)stream));
  } catch (PFail f) {
    return fail(c, f.code);
  }
  return BPMF_OK;
}

int bpmf_proposal_chi2(bpmf_ctx_t c, const float *pred, const double *ls, int J, double mix, double tau, double *chi2,
                       void *stream) {
  if (!c || !pred || !ls || !chi2 || J < 1 || !(mix >= 0.0 && mix <= 1.0) || !(tau > 0.0))
    return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  try {
    PCK(launch_proposal_chi2(pred, ls, J, mix, tau, chi2, (cudaStream_t)stream));
  } catch (PFail f) {
    return fail(c, f.code);
  }
  return BPMF_OK;
}

int bpmf_proposal_bpmf(bpmf_ctx_t c, const double *logZ_s, const int64_t *n_s, const double *q_s, int M, int K,
                       const int64_t *n_tot, double kT, double *bpmf, void *stream) {
  if (!c || !logZ_s || !n_s || !q_s || !n_tot || !bpmf || M < 1 || K < 1 || !(kT > 0.0)) return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  try {
    PCK(launch_is_estimate(logZ_s, reinterpret_cast<const long long *>(n_s), q_s, M, K,
                           reinterpret_cast<const long long *>(n_tot), kT, bpmf, (cudaStream_t)stream));
  } catch (PFail f) {
    return fail(c, f.code);
  }
  return BPMF_OK;
}

int bpmf_bootstrap(bpmf_ctx_t c, const double *logZ, const int64_t *n_valid, int J, int K, double kT, double h,
                   const double *u, int R, double *rep, double *stats, void *stream) {
  if (!c || !logZ || !n_valid || !u || J < 1 || K < 1 || R < 1 || !(kT > 0.0) || !(h > 0.0) || (!rep && !stats))
    return BPMF_ERR_INVALID_ARG;
  Dev dv(bpmf_internal_device(c));
  cudaStream_t st = (cudaStream_t)stream;
  double *buf = nullptr;
  try {
    double *r = rep;
    if (!r) {
      PCK(cudaMallocAsync(&buf, sizeof(double) * (size_t)R * (K + 1), st));
      r = buf;
    }
    PCK(launch_bootstrap(logZ, reinterpret_cast<const long long *>(n_valid), J, K, kT, h * h * h * kStandardConc, u, R,
                         r, stats, st));
    if (buf) PCK(cudaFreeAsync(buf, st));
  } catch (PFail f) {
    if (buf) cudaFreeAsync(buf, st);
    return fail(c, f.code);
  }
  return BPMF_OK;
}

}  // extern "C"
