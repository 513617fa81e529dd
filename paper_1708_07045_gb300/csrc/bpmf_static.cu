// bpmf_export_energies_static: the per-pose energy export without any device
// allocation.  Every intermediate buffer (twiddle tables, generalised charges,
// receptor spectra and their transform passes, the ligand grid and its
// transforms, the site-window tables) lives in one file-scope __device__
// array, so a caller that is not allowed to allocate device memory -- for
// example code running inside another framework's memory pool with no free
// headroom, or a host thread that must not call cudaMalloc because the device
// allocator would synchronise or block it -- can still compute energies into
// its own buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/bpmf.h"
#include "kernels.cuh"

using namespace bpmf;

namespace {

constexpr size_t kScratchBytes = (size_t)BPMF_STATIC_SCRATCH_BYTES;

// Shared by every call on a device; held by each GPU that loads this library
// until the process exits.
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_addr[kMaxDevices] = {};  // device address of g_scratch, per device

inline size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// One-time set-up per device (the device must be current): resolve the
// array's device address.  Host code only knows a stand-in for the symbol, so
// kernels are always given this address.
int scratch_address(int dev, unsigned char **out) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    return BPMF_ERR_INVALID_ARG;
  }
  if (!g_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return BPMF_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_addr[dev]);
  return BPMF_OK;
}

// Every pointer argument must be device (or managed) memory of device `dev`.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

struct Fail {
  int code;
};

#define SCK(call)                \
  do {                           \
    if ((call) != cudaSuccess) { \
      cudaGetLastError();        \
      throw Fail{BPMF_ERR_CUDA}; \
    }                            \
  } while (0)

template <class T>
void ligand_pass(const FftPlan pl[3], const float4 *tw[3], const int P[3], int F2, long long Q, const int U[3],
                 int S[3], const float *coords, const float2 *gamma, int n_atoms, const ConfMeta *d_meta,
                 const PairInfo *d_info, const float2 *const *d_rptr, float h_hi, float h_lo, float4 *d_part,
                 double *out, float2 *box, void *lz, void *ly, void *x2, void *y2, float nsh, float nsl, float esh,
                 float esl, cudaStream_t st) {
  SpreadArgs sa{coords, gamma, n_atoms, d_meta, h_hi, h_lo, U[0], U[1], U[2], box};
  SCK(launch_spread(sa, 1, st));
  ZfwdArgs za{};
  za.in = reinterpret_cast<const float *>(box);
  za.in_pairs = 1;
  za.n_rows = 3ll * U[0] * U[1];
  za.w_in = U[2];
  za.in_stride = U[2];
  za.out = lz;
  za.out_stride = F2;
  za.plan = pl[2];
  za.tw = tw[2];
  za.L = 16;
  SCK(launch_zfwd<T>(za, st));
  AxisArgs ya{};
  ya.in = lz;
  ya.out = ly;
  ya.P = P[1];
  ya.n_in = U[1];
  ya.n_out = P[1];
  ya.n_outer = 3ll * U[0];
  ya.inner = F2;
  ya.in_os = (long long)U[1] * F2;
  ya.out_os = (long long)P[1] * F2;
  ya.w0_div = 1;
  ya.axis = 1;
  ya.plan = pl[1];
  ya.tw = tw[1];
  ya.LW = 16;
  SCK(launch_axis<T>(ya, st));
  XfusedArgs xa{};
  xa.ly = ly;
  xa.U0 = U[0];
  xa.Q = Q;
  xa.K = 1;
  xa.rhi = d_rptr;
  xa.rlo = sizeof(T) == 8 ? d_rptr + 1 : nullptr;
  xa.x2 = x2;
  xa.S0 = S[0];
  xa.info = d_info;
  xa.plan = pl[0];
  xa.tw = tw[0];
  SCK(launch_xfused<T>(xa, 1, st));
  AxisArgs yi{};
  yi.in = x2;
  yi.out = y2;
  yi.P = P[1];
  yi.n_in = P[1];
  yi.n_out = S[1];
  yi.n_outer = S[0];
  yi.inner = F2;
  yi.in_os = Q;
  yi.out_os = (long long)S[1] * F2;
  yi.info = d_info;
  yi.w0_div = S[0];
  yi.axis = 1;
  yi.inverse = 1;
  yi.plan = pl[1];
  yi.tw = tw[1];
  yi.LW = 16;
  SCK(launch_axis<T>(yi, st));
  ZinvArgs zi{};
  zi.y2 = y2;
  zi.K = 1;
  zi.S0 = S[0];
  zi.S1 = S[1];
  zi.S2 = S[2];
  zi.F2 = F2;
  zi.info = d_info;
  zi.nscale_hi = nsh;
  zi.nscale_lo = nsl;
  zi.escale_hi = esh;
  zi.escale_lo = esl;
  zi.part = d_part;
  zi.export_E = out;
  zi.plan = pl[2];
  zi.tw = tw[2];
  SCK(launch_zinv<T>(zi, 1, st));
}

}  // namespace

extern "C" int bpmf_export_energies_static(const float *grids, int nx, int ny, int nz, double h, const int site_lo[3],
                                           const int site_n[3], int n_atoms, const float *coords, const float *q,
                                           const float *eps, const float *R, int p_rep, int p_att, unsigned mode,
                                           double *out, void *stream) {
  if (!grids || !site_lo || !site_n || !coords || !q || !eps || !R || !out || nx < 2 || ny < 2 || nz < 2 ||
      !(h > 0.0) || n_atoms < 1 || p_rep < 0 || p_rep > 32 || p_att < 0 || p_att > 32 ||
      (mode != BPMF_MODE_FP32 && mode != BPMF_MODE_FF)) {
    return BPMF_ERR_INVALID_ARG;
  }
  for (int d = 0; d < 3; ++d)
    if (site_n[d] < 1) {
      return BPMF_ERR_INVALID_ARG;
    }
  if (n_atoms > BPMF_MAX_ATOMS) {
    return BPMF_ERR_SIZE_UNSUPPORTED;
  }
  const int N[3] = {nx, ny, nz};
  int P[3];
  for (int d = 0; d < 3; ++d) {
    P[d] = smooth_edge(N[d]);
    if (!P[d]) {
      return BPMF_ERR_SIZE_UNSUPPORTED;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return BPMF_ERR_CUDA;
  }
  // the arrays go straight to kernels: host memory is rejected before any work
  for (const void *p : {(const void *)grids, (const void *)coords, (const void *)q, (const void *)eps,
                        (const void *)R, (const void *)out})
    if (!on_device(p, dev)) return BPMF_ERR_INVALID_ARG;
  unsigned char *base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc != BPMF_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  try {
    const bool use_ff = mode == BPMF_MODE_FF;
    const int F2 = P[2] / 2 + 1;
    const long long Q = (long long)P[1] * F2;
    const size_t Ef = sizeof(cx<ff>), E = use_ff ? sizeof(cx<ff>) : sizeof(cx<float>);
    int S[3] = {site_n[0], site_n[1], site_n[2]};

    // ---- fixed region: tables, charges, coordinate bounds, spectra ----------
    size_t off = 0;
    auto take = [&](size_t bytes) {
      const size_t o = off;
      off += up256(bytes);
      return o;
    };
    const size_t o_tw0 = take(sizeof(float4) * P[0]), o_tw1 = take(sizeof(float4) * P[1]),
                 o_tw2 = take(sizeof(float4) * P[2]);
    const size_t o_gam = take(sizeof(float2) * 3 * n_atoms);
    const size_t o_mm = take(sizeof(float) * 6), o_off = take(sizeof(int) * 2);
    const size_t o_meta = take(sizeof(ConfMeta)), o_info = take(sizeof(PairInfo));
    const size_t o_part = take(sizeof(float4) * S[0]), o_rptr = take(sizeof(void *) * 2);
    const size_t nspec = 3ull * P[0] * Q;
    const size_t o_hi = take(sizeof(float2) * nspec), o_lo = take(sizeof(float2) * nspec);
    const size_t o_var = off;  // receptor temporaries, then the ligand buffers
    // receptor passes: z output [3][nx][ny][F2], y output [3][nx][P1][F2],
    // x output [3][P0][P1][F2] (written over the z output's region)
    const size_t rz = up256(std::max(3ull * nx * ny * F2, 3ull * P[0] * Q) * Ef), ry = up256(3ull * nx * Q * Ef);
    if (o_var + rz + ry > kScratchBytes) return BPMF_ERR_SIZE_UNSUPPORTED;  // grid too large
    float4 *tw0 = reinterpret_cast<float4 *>(base + o_tw0), *tw1 = reinterpret_cast<float4 *>(base + o_tw1),
           *tw2 = reinterpret_cast<float4 *>(base + o_tw2);
    // the three tables in one host staging vector (read by the copies until the
    // final synchronisation)
    std::vector<float4> ht((size_t)P[0] + P[1] + P[2]);
    twiddle_values(P[0], ht.data());
    twiddle_values(P[1], ht.data() + P[0]);
    twiddle_values(P[2], ht.data() + P[0] + P[1]);
    SCK(cudaMemcpyAsync(tw0, ht.data(), sizeof(float4) * P[0], cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(tw1, ht.data() + P[0], sizeof(float4) * P[1], cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(tw2, ht.data() + P[0] + P[1], sizeof(float4) * P[2], cudaMemcpyHostToDevice, st));
    const float4 *tws[3] = {tw0, tw1, tw2};
    const FftPlan pls[3] = {make_plan(P[0]), make_plan(P[1]), make_plan(P[2])};

    // generalised charges and coordinate bounds
    float2 *gam = reinterpret_cast<float2 *>(base + o_gam);
    SCK(launch_gamma(q, eps, R, n_atoms, p_rep, p_att, gam, st));
    int *d_off = reinterpret_cast<int *>(base + o_off);
    const int hoff[2] = {0, n_atoms};
    SCK(cudaMemcpyAsync(d_off, hoff, sizeof(hoff), cudaMemcpyHostToDevice, st));
    float *d_mm = reinterpret_cast<float *>(base + o_mm);
    SCK(launch_minmax(coords, d_off, d_off + 1, 1, d_mm, st));
    float mm[6];
    SCK(cudaMemcpyAsync(mm, d_mm, sizeof(mm), cudaMemcpyDeviceToHost, st));
    SCK(cudaStreamSynchronize(st));

    // placement metadata and the site window (same rules as bpmf_eval)
    ConfMeta m{};
    PairInfo pi{};
    const float hf = (float)h;
    int U[3];
    for (int d = 0; d < 3; ++d) {
      m.lo[d] = mm[d];
      m.u[d] = box_extent(mm[d], mm[3 + d], hf);
      site_window(N[d], site_lo[d], site_n[d], m.u[d], pi.w0[d], pi.sa[d], pi.sb[d]);
      pi.wc[d] = pi.w0[d];
      U[d] = std::max(1, std::min(m.u[d], P[d]));
    }
    U[1] += U[1] & 1;
    m.atom_off = 0;
    m.n_atoms = n_atoms;
    m.gamma_off = 0;
    ConfMeta *d_meta = reinterpret_cast<ConfMeta *>(base + o_meta);
    PairInfo *d_info = reinterpret_cast<PairInfo *>(base + o_info);
    SCK(cudaMemcpyAsync(d_meta, &m, sizeof(m), cudaMemcpyHostToDevice, st));
    SCK(cudaMemcpyAsync(d_info, &pi, sizeof(pi), cudaMemcpyHostToDevice, st));

    // ligand buffers (reuse the receptor temporaries' region afterwards)
    const size_t lbox = up256(3ull * U[0] * U[1] * U[2] * sizeof(float2));
    const size_t llz = up256(3ull * U[0] * U[1] * F2 * E), lly = up256(3ull * U[0] * Q * E);
    const size_t lx2 = up256((size_t)S[0] * Q * E), ly2 = up256((size_t)S[0] * S[1] * F2 * E);
    const size_t lig_need = lbox + llz + lly + lx2 + ly2;
    if (o_var + std::max(rz + ry, lig_need) > kScratchBytes) return BPMF_ERR_SIZE_UNSUPPORTED;  // box too large

    // receptor spectra FT(G_R) in float pairs
    float2 *hi = reinterpret_cast<float2 *>(base + o_hi), *lo = reinterpret_cast<float2 *>(base + o_lo);
    void *tz = base + o_var, *ty = base + o_var + rz;
    ZfwdArgs za{};
    za.in = grids;
    za.n_rows = 3ll * nx * ny;
    za.w_in = nz;
    za.in_stride = nz;
    za.out = tz;
    za.out_stride = F2;
    za.plan = pls[2];
    za.tw = tw2;
    za.L = 16;
    SCK(launch_zfwd<ff>(za, st));
    AxisArgs ya{};
    ya.in = tz;
    ya.out = ty;
    ya.P = P[1];
    ya.n_in = ny;
    ya.n_out = P[1];
    ya.n_outer = 3ll * nx;
    ya.inner = F2;
    ya.in_os = (long long)ny * F2;
    ya.out_os = Q;
    ya.w0_div = 1;
    ya.axis = 1;
    ya.plan = pls[1];
    ya.tw = tw1;
    ya.LW = 16;
    SCK(launch_axis<ff>(ya, st));
    AxisArgs xa{};
    xa.in = ty;
    xa.out = tz;
    xa.P = P[0];
    xa.n_in = nx;
    xa.n_out = P[0];
    xa.n_outer = 3;
    xa.inner = Q;
    xa.in_os = (long long)nx * Q;
    xa.out_os = (long long)P[0] * Q;
    xa.w0_div = 1;
    xa.axis = 0;
    xa.plan = pls[0];
    xa.tw = tw0;
    xa.LW = 16;
    SCK(launch_axis<ff>(xa, st));
    SCK(launch_split_ff(tz, hi, lo, (long long)nspec, st));
    const float2 **d_rptr = reinterpret_cast<const float2 **>(base + o_rptr);
    const float2 *hptr[2] = {hi, lo};
    SCK(cudaMemcpyAsync(d_rptr, hptr, sizeof(hptr), cudaMemcpyHostToDevice, st));

    // ligand side, K = 1, energies exported over the site window
    unsigned char *lb = base + o_var;
    float2 *box = reinterpret_cast<float2 *>(lb);
    void *lz = lb + lbox, *ly = lb + lbox + llz, *x2 = lb + lbox + llz + lly, *y2 = lb + lbox + llz + lly + lx2;
    const double norm = 1.0 / ((double)P[0] * P[1] * P[2]);
    const float nsh = (float)(-norm), nsl = (float)(-norm - (double)nsh);
    const float esh = (float)norm, esl = (float)(norm - (double)esh);
    const float hh = (float)h, hl = (float)(h - (double)hh);
    float4 *d_part = reinterpret_cast<float4 *>(base + o_part);
    if (use_ff)
      ligand_pass<ff>(pls, tws, P, F2, Q, U, S, coords, gam, n_atoms, d_meta, d_info, d_rptr, hh, hl, d_part, out,
                      box, lz, ly, x2, y2, nsh, nsl, esh, esl, st);
    else
      ligand_pass<float>(pls, tws, P, F2, Q, U, S, coords, gam, n_atoms, d_meta, d_info, d_rptr, hh, hl, d_part, out,
                         box, lz, ly, x2, y2, nsh, nsl, esh, esl, st);
    // the host-side tables above are stack / vector memory: finish before
    // returning so no copy reads them afterwards
    SCK(cudaStreamSynchronize(st));
  } catch (Fail f) {
    return f.code;
  }
  return BPMF_OK;
}
