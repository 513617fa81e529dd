// Learned-proposal kernels: configuration features, bf16 tensor-core GEMM,
// training helpers, proposal sampling and the importance-weighted estimator.
#pragma once
#include <cuda_runtime.h>

namespace bpmf {

constexpr int kFeatures = 24;
// Standard-state concentration (1 M = N_A / 1e27 molecules per A^3), as in kernels.cuh
#ifndef BPMF_STANDARD_CONC_DEFINED
#define BPMF_STANDARD_CONC_DEFINED
constexpr double kStandardConc = 6.02214076e23 / 1e27;
#endif

struct GemmArgs {
  const float *A;          // element (m, k) at A[m * sam + k * sak]
  long long sam, sak;
  int a_op;                // 0: as is, 1: ReLU
  const float *Zmask;      // unused (reserved)
  long long szm, szk;
  const float *B;          // element (k, n) at B[k * sbk + n * sbn]
  long long sbk, sbn;
  float *C;                // element (m, n) at C[m * scm + n]
  long long scm;
  const float *bias;       // [N] or null
  int accumulate;          // C += result
  int M, N, K;
};

cudaError_t launch_features(const float *coords, const int *conf_off, const int *conf_nat, const int *conf_lig,
                            const float *q, const float *eps, const float *R, const int *lig_atom_off, int n_conf,
                            float h, float *out, cudaStream_t st);
cudaError_t launch_gemm_bf16(const GemmArgs &g, cudaStream_t st);
cudaError_t launch_mse(const float *y, const float *t, int B, float *dy, float *loss, cudaStream_t st);
cudaError_t launch_colsum(const float *D, const float *Z, int B, int N, float *out, cudaStream_t st);
cudaError_t launch_adam(float *w, const float *gw, float *m, float *v, long long n, float lr, float b1, float b2,
                        float epsl, float bc1, float bc2, cudaStream_t st);
cudaError_t launch_mask_relu_grad(float *D, const float *Z, long long n, cudaStream_t st);
cudaError_t launch_affine(const float *x, const float *shift, const float *scale, int B, int N, int invert, float *out,
                          cudaStream_t st);
cudaError_t launch_proposal(const float *pred, int J, double mix, double tau, const double *u, int M, double *q,
                            double *cdf, int *idx, double *q_s, cudaStream_t st);
cudaError_t launch_config_targets(const double *logZ, const long long *n_valid, int J, int K, double clip, double *ls,
                                  float *t, cudaStream_t st);
cudaError_t launch_proposal_chi2(const float *pred, const double *ls, int J, double mix, double tau, double *out,
                                 cudaStream_t st);
cudaError_t launch_is_estimate(const double *logZ_s, const long long *n_s, const double *q_s, int M, int K,
                               const long long *n_tot, double kT, double *bpmf, cudaStream_t st);
cudaError_t launch_sir_configs(const double *logZ, const long long *nvalid, int J, int K, int k, const double *u,
                               int M, double *cdf, int *conf, cudaStream_t st);
cudaError_t launch_sir_translations(const double *E, int nS, double kT, const double *u, const int *conf, int j, int M,
                                    double *cdf, int *pick, cudaStream_t st);
cudaError_t launch_bootstrap(const double *logZ, const long long *nvalid, int J, int K, double kT, double vscale,
                             const double *u, int R, double *rep, double *stats, cudaStream_t st);

}  // namespace bpmf
