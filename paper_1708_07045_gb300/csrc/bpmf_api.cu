// C-ABI layer: handles, plans, twiddle tables, workspace and the launch
// sequence of the hot path.  Host-side logic only; every arithmetic step of
// the correlation runs in the kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <array>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "../../include/bpmf.h"
#include "kernels.cuh"
#include "proposal.cuh"

using namespace bpmf;

// ------------------------------------------------ host plan helpers (shared)
namespace bpmf {

// smallest 2^a 3^b 5^c 7^d >= n with a >= 1
int smooth_edge(int n) {
  if (n < 2) n = 2;
  for (int p = n; p <= BPMF_MAX_FFT_EDGE; ++p) {
    if (p % 2) continue;
    int m = p;
    for (int r : {2, 3, 5, 7})
      while (m % r == 0) m /= r;
    if (m == 1) return p;
  }
  return 0;
}


FftPlan make_plan(int P) {
  FftPlan pl{};
  pl.n = P;
  int m = P, k = 0;
  while (m % 8 == 0) pl.r[k++] = 8, m /= 8;
  while (m % 4 == 0) pl.r[k++] = 4, m /= 4;
  while (m % 2 == 0) pl.r[k++] = 2, m /= 2;
  for (int r : {3, 5, 7})
    while (m % r == 0) pl.r[k++] = r, m /= r;
  pl.nst = k;
  return pl;
}


// exp(-2 pi i k / P), k < P, as float pairs {re hi, im hi, re lo, im lo},
// each from the exact fraction k / P in long double
void twiddle_values(int P, float4 *out) {
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int k = 0; k < P; ++k) {
    const long double a = two_pi * (long double)k / (long double)P;
    const long double re = cosl(a), im = -sinl(a);
    const float rh = (float)re, ih = (float)im;
    out[k] = make_float4(rh, ih, (float)(re - (long double)rh), (float)(im - (long double)ih));
  }
}

// ligand-box extent u = ceil((hi - lo) / h) + 4 ("two additional grid
// spacings" per side), decided in single precision exactly as the oracle does
int box_extent(float lo, float hi, float hf) {
  volatile float ext = hi - lo;
  volatile float r = ext / hf;
  return (int)std::ceil(r) + 4;
}

// Site window of one (configuration, receptor) pair along axis d: the ligand
// box centre floor(u/2) lands in [site_lo, site_lo + site_n) and the whole box
// [m, m + u] stays inside the N nodes of the grid.  Returns the valid count.
long long site_window(int N, int site_lo, int site_n, int u, int &w0, int &sa, int &sb) {
  w0 = site_lo - u / 2;
  sa = std::max(0, -w0);
  sb = std::min(site_n - 1, N - 1 - u - w0);
  return sb >= sa ? (long long)(sb - sa + 1) : 0;
}

}  // namespace bpmf

// ---------------------------------------------------------------- handles
struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
};

struct bpmf_ctx {
  int device = 0;
  bool prof = false;
  std::vector<ProfRec> pending;
  std::vector<cudaEvent_t> event_pool;
  std::vector<std::string> prof_names;
  std::vector<double> prof_ms;
  std::vector<long long> prof_n;
  std::string err;
  std::string note;            // the last evaluation's warning detail (refined-form fallbacks)
  bool refine_seeded = false;    // refined form: start each pair from the stored minimum (second pass)
  unsigned *pmin_store = nullptr;  // [total_conf][K] refined form: each pair's final running minimum
  size_t pmin_store_n = 0;
  int refine_list_cap = 0;        // refined form: list capacity per pair (0: the default rule)
  int wait_test = 0;              // testing: the x pass's first tile wait runs out (bpmf_set_wait_test)
  std::map<int, float4 *> tw;  // twiddle tables per transform length
  uint4 *tca = nullptr;        // tensor-core radix-32 fragment table (split-bf16 mode)
  const __nv_bfloat16 *tc05 = nullptr;  // the same stage's matrix in the tcgen05 layout
  void *ws = nullptr;          // grow-only device workspace
  size_t ws_bytes = 0;
  size_t ws_budget = size_t(3) << 30;  // set by bpmf_create from the device's memory
  unsigned long long next_id = 1;  // handle identities (graph cache keys)
  void *pinned = nullptr;          // pinned host staging of the eval tables
  size_t pinned_bytes = 0;
  cudaEvent_t pinned_busy = nullptr;  // recorded after the last copy / graph replay reading `pinned`
  bool graph_mode = false;         // replay bpmf_eval as a CUDA graph
  cudaGraphExec_t gexec = nullptr;
  std::vector<unsigned long long> gkey;
  // launch shapes chosen by bpmf_autotune, per (P0, P1, P2, mode); none of
  // them changes a result bit (every line transform is independent), except
  // xround, which changes the FP32 forms' x transform length (its radix plan)
  struct Tune {
    int batch_cap = 0;  // configurations per batch (0: as many as the workspace holds)
    int axis_lw = 0;    // lines per CTA of the strided passes (0: 32 for FP32 lines, 16 for float pairs)
    int zfwd_l = 16;    // complex lines per CTA of the z R2C pass
    bool xround = true; // FP32 forms: x edge rounded up to the compile-time x pass's edges
  };
  std::map<std::vector<int>, Tune> tune;
  bool warn_last = false;  // BPMF_WARN_NO_VALID of the plan behind the cached graph
  int *fail_host = nullptr;  // pinned [fail_n]: refined form, per ligand of the last call, certificate failed
  size_t fail_n = 0;
  float refine_check_scale = 1.f;  // multiplies B in the refined form's certificate check
  // library streams on which independent receptor crops are transformed
  // concurrently (forked from and joined back into the caller's stream)
  static constexpr int kSide = 4;
  cudaStream_t side[kSide] = {};
  // host-to-device copies of receptor grids given in host memory: on their
  // own stream, so that they overlap the caller's queued work
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_ev = nullptr;
  int side_next = 0;
  // device blocks of freed handles, by size, reused by later handles of the
  // same size (the free synchronises the device first, as cudaFree does)
  std::multimap<size_t, void *> blocks;
  size_t block_bytes = 0;
};

struct bpmf_rec {
  bpmf_ctx *ctx = nullptr;
  unsigned long long id = 0;
  int N[3] = {0, 0, 0}, P[3] = {0, 0, 0}, F2 = 0;
  long long Q = 0;
  double h = 0;
  double origin[3] = {0, 0, 0};
  int site_lo[3] = {0, 0, 0}, site_n[3] = {0, 0, 0};
  void *mem = nullptr;                  // one device block holding grid, sumsq, hi and lo
  size_t mem_bytes = 0;
  float2 *hi = nullptr, *lo = nullptr;  // [3][P0][Q]
  uint32_t *occ = nullptr;              // occupancy tables [kOccLevels][N0 + 32][occW][N1 + 32], or null
  int occW = 0;
  float *grid = nullptr;                // the FP32 grids [3][N0][N1][N2] (refined form)
  float *sumsq = nullptr;               // [3] their sums of squares (FP32 error bound)
  float2 *sumsq_scratch = nullptr;      // [kSumsqScratch] partial sums (launch_sumsq)
  // spectra of the grids cropped to a box of transform edges P around the
  // site, made on first use, per P (the uncropped spectrum is hi / lo)
  struct Crop {
    void *mem = nullptr;                // the device block holding hi, lo and sumsq (null: a view)
    size_t mem_bytes = 0;
    int c0[3] = {0, 0, 0};              // first node of the crop
    float2 *hi = nullptr, *lo = nullptr;  // [3][P0][P1 (P2/2+1)]
    float *sumsq = nullptr;             // [3] over the cropped nodes
    float2 *sumsq_scratch = nullptr;    // [kSumsqScratch] partial sums (launch_sumsq)
    double vol = 0;                     // cropped nodes per channel
  };
  std::map<std::array<int, 3>, Crop> crops;
  cudaEvent_t crop_ev = nullptr;        // recorded after the last crop was made (on the stream that made it)
  // Float-pair partial spectra the crops start from (a crop along one axis
  // commutes with the transforms along the others): the z spectra
  // [3][N0][N1][Pz/2+1] of the grids with z cropped to edge Pz (key Pz), and
  // their y spectra [3][N0][Py (Pz/2+1)] with y cropped to edge Py (key
  // (Py, Pz)); the uncropped ones are the load's own intermediates.  ev is
  // recorded on the stream that made the stage.
  struct Stage {
    void *mem = nullptr;
    size_t mem_bytes = 0;
    void *v = nullptr;  // cx<ff>
    cudaEvent_t ev = nullptr;
  };
  std::map<int, Stage> zst;
  std::map<std::pair<int, int>, Stage> yst;
};

struct bpmf_lig {
  bpmf_ctx *ctx = nullptr;
  unsigned long long id = 0;
  int n_lig = 0;
  std::vector<int> n_atoms, n_conf, atom_off, conf_off, coord_off;
  long long total_conf = 0, total_atoms = 0, total_coord_atoms = 0;
  float *coords = nullptr;  // device [coord_atoms][3]
  float2 *gamma = nullptr;  // device [3][total_atoms] float pairs
  float *q = nullptr, *eps = nullptr, *R = nullptr;  // device [total_atoms] (configuration features)
  std::vector<float> minmax;  // host [total_conf][6]
  std::vector<float> R_host;  // host [total_atoms] (occupancy radii)
  std::vector<float> q_host, eps_host;  // host [total_atoms] (FP32 error bound)
  void *mem = nullptr;        // one device block holding coords, gamma, q, eps and R
  size_t mem_bytes = 0;
  int p_rep = 12, p_att = 6;
};

namespace {

struct Fail {
  int code;
};

int set_err(bpmf_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                               \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      last_msg = std::string(#call) + ": " + cudaGetErrorString(e_);                            \
      throw Fail{e_ == cudaErrorMemoryAllocation ? BPMF_ERR_OOM : BPMF_ERR_CUDA};              \
    }                                                                                          \
  } while (0)

thread_local std::string last_msg;

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Fragment tables of the tensor-core radix-32 stage: the real 64 x 64 DFT-32
// matrix (rows 2r'+c', columns 2r+c), split into bf16 high, middle and low
// parts and laid out in mma.sync m16n8k16 A-fragment order, forward then
// inverse.
const uint4 *tc_table(bpmf_ctx *c);

const __nv_bfloat16 *tc05_table(bpmf_ctx *c);

// split-bf16 plan: the radix-32 factor as a final tensor-core stage when 32 | P
// (tcgen05 form; the mma.sync fragments stay as the reference form)
FftPlan make_plan_split(bpmf_ctx *c, int P) {
  if (P % 32) return make_plan(P);
  FftPlan pl = make_plan(P / 32);
  pl.n = P;
  if (P == 32) pl.nst = 0;
  pl.r[pl.nst++] = 32;
  pl.tca = tc_table(c);
  pl.tc05_f = tc05_table(c);
  return pl;
}

const float4 *twiddles(bpmf_ctx *c, int P) {
  auto it = c->tw.find(P);
  if (it != c->tw.end()) return it->second;
  std::vector<float4> h(P);
  twiddle_values(P, h.data());
  float4 *d = nullptr;
  CK(cudaMalloc(&d, sizeof(float4) * P));
  CK(cudaMemcpy(d, h.data(), sizeof(float4) * P, cudaMemcpyHostToDevice));
  c->tw[P] = d;
  return d;
}

static inline unsigned short bf16_bits(float v) {  // round to nearest even
  unsigned u;
  std::memcpy(&u, &v, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (unsigned short)(u >> 16);
}
static inline float bf16_val(unsigned short b) {
  const unsigned u = (unsigned)b << 16;
  float v;
  std::memcpy(&v, &u, 4);
  return v;
}

const uint4 *tc_table(bpmf_ctx *c) {
  if (c->tca) return c->tca;
  std::vector<uint4> h(2 * 3 * 4 * 4 * 32);
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int dir = 0; dir < 2; ++dir) {
    float A[64][64];
    for (int rp = 0; rp < 32; ++rp)
      for (int r = 0; r < 32; ++r) {
        const long double a = two_pi * (long double)((rp * r) % 32) / 32.0L;
        const float wr = (float)cosl(a), wi = (float)((dir ? 1 : -1) * sinl(a));
        A[2 * rp][2 * r] = wr;
        A[2 * rp][2 * r + 1] = -wi;
        A[2 * rp + 1][2 * r] = wi;
        A[2 * rp + 1][2 * r + 1] = wr;
      }
    for (int term = 0; term < 3; ++term)
      for (int t = 0; t < 4; ++t)
        for (int q = 0; q < 4; ++q)
          for (int lane = 0; lane < 32; ++lane) {
            const int gid = lane >> 2, tig = lane & 3;
            auto part = [&](int m, int k) {  // a = hi + mid + lo, each bf16
              const float a = A[m][k];
              const unsigned short hb = bf16_bits(a);
              const float r = a - bf16_val(hb);
              const unsigned short mb = bf16_bits(r);
              return term == 0 ? hb : (term == 1 ? mb : bf16_bits(r - bf16_val(mb)));
            };
            auto pack = [&](int m, int k) { return (unsigned)part(m, k) | ((unsigned)part(m, k + 1) << 16); };
            const int m = 16 * t + gid, k = 16 * q + 2 * tig;
            h[(((dir * 3 + term) * 4 + t) * 4 + q) * 32 + lane] =
                make_uint4(pack(m, k), pack(m + 8, k), pack(m, k + 8), pack(m + 8, k + 8));
          }
  }
  uint4 *d = nullptr;
  CK(cudaMalloc(&d, sizeof(uint4) * h.size()));
  CK(cudaMemcpy(d, h.data(), sizeof(uint4) * h.size(), cudaMemcpyHostToDevice));
  c->tca = d;
  return d;
}

// The real 64 x 64 DFT-32 matrix of the tcgen05 stage, [dir][part][64 x 64]
// bf16 (hi, mid, lo with hi + mid + lo = the FP32 coefficient), each part in
// the tensor cores' K-major core-matrix layout: element (n, k) at
// (n / 8) 512 + (k / 8) 64 + (n % 8) 8 + k % 8.
const __nv_bfloat16 *tc05_table(bpmf_ctx *c) {
  if (c->tc05) return c->tc05;
  std::vector<unsigned short> h(2 * 3 * 64 * 64);
  const long double two_pi = 6.283185307179586476925286766559L;
  for (int dir = 0; dir < 2; ++dir)
    for (int rp = 0; rp < 32; ++rp)
      for (int r = 0; r < 32; ++r) {
        const long double a = two_pi * (long double)((rp * r) % 32) / 32.0L;
        const float wr = (float)cosl(a), wi = (float)((dir ? 1 : -1) * sinl(a));
        const float F[2][2] = {{wr, -wi}, {wi, wr}};  // rows 2r' + c', columns 2r + c
        for (int cp = 0; cp < 2; ++cp)
          for (int cc = 0; cc < 2; ++cc) {
            const int n = 2 * rp + cp, k = 2 * r + cc;
            const int off = (n >> 3) * 512 + (k >> 3) * 64 + (n & 7) * 8 + (k & 7);
            float v = F[cp][cc];
            for (int part = 0; part < 3; ++part) {
              const unsigned short b = bf16_bits(v);
              h[(dir * 3 + part) * 64 * 64 + off] = b;
              v -= bf16_val(b);
            }
          }
      }
  void *d = nullptr;
  CK(cudaMalloc(&d, sizeof(unsigned short) * h.size()));
  CK(cudaMemcpy(d, h.data(), sizeof(unsigned short) * h.size(), cudaMemcpyHostToDevice));
  c->tc05 = static_cast<const __nv_bfloat16 *>(d);
  return c->tc05;
}

void *workspace(bpmf_ctx *c, size_t bytes, cudaStream_t st) {
  if (bytes <= c->ws_bytes) return c->ws;
  if (c->ws) {
    CK(cudaStreamSynchronize(st));
    CK(cudaFree(c->ws));
    c->ws = nullptr;
    c->ws_bytes = 0;
  }
  CK(cudaMalloc(&c->ws, bytes));
  c->ws_bytes = bytes;
  return c->ws;
}

inline size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

cudaEvent_t pool_event(bpmf_ctx *c) {
  if (!c->event_pool.empty()) {
    cudaEvent_t e = c->event_pool.back();
    c->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  CK(cudaEventCreate(&e));
  return e;
}

// Handle blocks: a cached block of exactly `bytes` if one is free, else a
// new allocation.  block_put returns a block to the cache (up to 2 GiB) or
// frees it; callers synchronise the device before returning a block.
constexpr size_t kBlockCacheCap = size_t(2) << 30;

void *block_get(bpmf_ctx *c, size_t bytes) {
  auto it = c->blocks.find(bytes);
  if (it != c->blocks.end()) {
    void *p = it->second;
    c->blocks.erase(it);
    c->block_bytes -= bytes;
    return p;
  }
  void *p = nullptr;
  CK(cudaMalloc(&p, bytes));
  return p;
}

void block_put(bpmf_ctx *c, void *p, size_t bytes) {
  if (!p) return;
  if (c->block_bytes + bytes <= kBlockCacheCap) {
    c->blocks.insert({bytes, p});
    c->block_bytes += bytes;
  } else {
    cudaFree(p);
  }
}

// Sub-buffers of one device allocation: add() reserves 256-byte aligned
// ranges, alloc() takes the block (block_get) and returns its base.
struct Carve {
  std::vector<std::pair<void **, size_t>> parts;
  size_t total = 0;
  template <class P>
  void add(P **ptr, size_t bytes) {
    parts.push_back({reinterpret_cast<void **>(ptr), total});
    total += align_up(std::max<size_t>(bytes, 1));
  }
  void *alloc(bpmf_ctx *c) {
    void *base = block_get(c, total);
    for (auto &pr : parts) *pr.first = static_cast<char *>(base) + pr.second;
    return base;
  }
};

// Launch `fn` (returning cudaError_t); when profiling, bracket it with events.
template <class F>
void launch(bpmf_ctx *c, const char *name, cudaStream_t st, F &&fn) {
  auto run = [&] {
    cudaError_t e = fn();
    if (e != cudaSuccess) {
      last_msg = std::string(name) + ": " + cudaGetErrorString(e);
      throw Fail{e == cudaErrorMemoryAllocation ? BPMF_ERR_OOM : BPMF_ERR_CUDA};
    }
  };
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!c->prof || (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)) {
    run();
    return;
  }
  ProfRec r{name, pool_event(c), pool_event(c)};
  CK(cudaEventRecord(r.a, st));
  run();
  CK(cudaEventRecord(r.b, st));
  c->pending.push_back(r);
}

void prof_drain(bpmf_ctx *c) {
  for (auto &r : c->pending) {
    CK(cudaEventSynchronize(r.b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, r.a, r.b));
    size_t i = 0;
    while (i < c->prof_names.size() && c->prof_names[i] != r.name) ++i;
    if (i == c->prof_names.size()) {
      c->prof_names.push_back(r.name);
      c->prof_ms.push_back(0.0);
      c->prof_n.push_back(0);
    }
    c->prof_ms[i] += ms;
    c->prof_n[i] += 1;
    c->event_pool.push_back(r.a);
    c->event_pool.push_back(r.b);
  }
  c->pending.clear();
}

void split_ff(double v, float &hi, float &lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}


// temporary device copy of a host or device input
struct DevIn {
  const void *p = nullptr;
  void *own = nullptr;
  cudaStream_t st = nullptr;
  DevIn(const void *src, size_t bytes, cudaStream_t s) : st(s) {
    if (!src) throw Fail{BPMF_ERR_INVALID_ARG};
    if (is_device_ptr(src)) {
      p = src;
    } else {
      CK(cudaMallocAsync(&own, bytes ? bytes : 1, st));
      CK(cudaMemcpyAsync(own, src, bytes, cudaMemcpyHostToDevice, st));
      p = own;
    }
  }
  ~DevIn() {
    if (own) cudaFreeAsync(own, st);
  }
};

// Runs the eval launch sequence for one batch of configurations.
struct BatchGeom {
  int U[3];
  int P[3], F2;
  long long Q;
  int S[3];
  int K;
  int occ_cap = 0;  // ligand occupancy runs per configuration (0: no clash channel)
  int occ_rb = 1;   // CTAs per configuration building the runs
  bool refine = false;  // refined form: candidate lists for k_refine
  int ref_cap = 0;      // refined form: translations per pair list
  int nmax = 0;         // atoms per configuration of the ligand
};

// Refined form: per-call inputs of run_batch
struct RefineCtx {
  const RefTab *rtabs = nullptr;  // [Kg] grids and sums of squares of the bucket's transforms
  double gnorm[3] = {0, 0, 0};    // ||gamma_t||_2 of the ligand
  double kT = 1.0;
  float4 *part_ref = nullptr;     // [batch][Kg][2] corrections (this batch's slice)
  int *fail = nullptr;            // the ligand's fallback flag
  float check_scale = 1.f;
  float bound_scale = 1.f;        // multiplies B (window and certificate)
  unsigned *store = nullptr;      // [J][K] the ligand's pair minima (RefineArgs::store)
  const int *order = nullptr;     // [batch] processing position -> configuration (this batch's slice)
  const int *kmap = nullptr;      // [Kg]
  int Kall = 0;
  bool seeded = false;            // start from the stored minima (a second pass)
};

// Translations per pair list of the refined form: every translation of the
// site window (at most kRefineMaxList), so that no list can overflow; the
// lists take memory, but only the translations a plane lists are written.
// `cap` > 0 overrides (tests).
int refine_cap(const int S[3], int cap = 0) {
  const long long nS = (long long)S[0] * S[1] * S[2];
  if (cap > 0) return (int)std::min<long long>(std::min<long long>(nS, cap), kRefineMaxList);
  return (int)std::min<long long>(nS, kRefineMaxList);
}

int clash_words(int S2) { return (S2 + 31) / 32; }

size_t batch_bytes_per_conf(const BatchGeom &g, size_t E) {
  const size_t box = 3ull * g.U[0] * g.U[1] * g.U[2] * sizeof(float2);
  const size_t lz = 3ull * g.U[0] * g.U[1] * g.F2 * E;
  const size_t ly = 3ull * g.U[0] * g.Q * E;
  const size_t x2 = (size_t)g.K * g.S[0] * g.Q * E;
  const size_t y2 = (size_t)g.K * g.S[0] * g.S[1] * g.F2 * E;
  size_t occ = 0;
  if (g.occ_cap > 0)
    occ = align_up(2 * (size_t)g.occ_cap * sizeof(OccRun)) + align_up(sizeof(int)) +
          align_up((size_t)g.K * g.S[0] * g.S[1] * clash_words(g.S[2]) * sizeof(uint32_t));
  size_t ref = 0;
  if (g.refine)  // lists, exact values, running minima, counts, levels, sums, CTA counters; window and bound
    ref = align_up((size_t)g.K * g.ref_cap * sizeof(Cand)) + align_up((size_t)g.K * g.ref_cap * sizeof(float2)) +
          3 * align_up((size_t)g.K * sizeof(int)) + 2 * align_up((size_t)g.K * sizeof(unsigned long long)) +
          2 * align_up((size_t)g.K * sizeof(float));
  return align_up(box) + align_up(lz) + align_up(ly) + align_up(x2) + align_up(y2) + occ + ref;
}

// Upper bound on the occupancy runs of one configuration: every merged
// interval of a row comes from an atom whose disk covers the row (at most
// (2 ceil(r) + 1)^2 rows per atom, r = R / h in nodes), and a long interval
// splits into pieces of at most 63 nodes over a row extent of at most
// u2 + 2 ceil(r) + 6 nodes.
int occ_run_cap(int n_atoms, float rmax_nodes, int u2) {
  const int rc = (int)std::ceil(rmax_nodes);
  const long long disk = (long long)(2 * rc + 1) * (2 * rc + 1);
  const long long nC = (long long)u2 + 2 * rc + 6;
  const long long cap = (long long)n_atoms * disk * (2 + nC / 63);
  return (int)std::min<long long>(cap, 1ll << 28);
}

template <class T>
void run_batch(bpmf_ctx *c, const bpmf_lig *lg, const BatchGeom &g, int batch, const ConfMeta *d_meta,
               const PairInfo *d_info, const float2 *const *d_rhi, const float2 *const *d_rlo, double h,
               float nscale_hi, float nscale_lo, float escale_hi, float escale_lo, float4 *d_part,
               double *export_E, char *ws, size_t ws_avail, cudaStream_t st, const bpmf_ctx::Tune &tn,
               bool split = false,
               const OccTab *d_tabs = nullptr, const RefineCtx *rf = nullptr, const float2 *const *h_rhi = nullptr,
               int *d_err = nullptr) {
  auto plan = [&](int P) {
    FftPlan pl = split ? make_plan_split(c, P) : make_plan(P);
    pl.err = d_err;  // a bounded tensor-core wait that ran out
    return pl;
  };
  const size_t E = sizeof(cx<T>);
  char *p = ws;
  float2 *box = reinterpret_cast<float2 *>(p);
  p += align_up(3ull * batch * g.U[0] * g.U[1] * g.U[2] * sizeof(float2));
  void *lz = p;
  p += align_up(3ull * batch * g.U[0] * g.U[1] * g.F2 * E);
  void *ly = p;
  p += align_up(3ull * batch * g.U[0] * g.Q * E);
  void *x2 = p;
  p += align_up((size_t)batch * g.K * g.S[0] * g.Q * E);
  void *y2 = p;
  p += align_up((size_t)batch * g.K * g.S[0] * g.S[1] * g.F2 * E);
  uint32_t *clash = nullptr;
  const int CW = clash_words(g.S[2]);
  OccRun *runs = nullptr;
  int *n_runs = nullptr;
  if (g.occ_cap > 0 && d_tabs) {
    runs = reinterpret_cast<OccRun *>(p);
    p += align_up(2 * (size_t)batch * g.occ_cap * sizeof(OccRun));
    n_runs = reinterpret_cast<int *>(p);
    p += align_up((size_t)batch * sizeof(int));
    clash = reinterpret_cast<uint32_t *>(p);
    p += align_up((size_t)batch * g.K * g.S[0] * g.S[1] * CW * sizeof(uint32_t));
  }
  RefineArgs ra{};
  if (g.refine) {
    const size_t np = (size_t)batch * g.K;
    ra.rs.cand = reinterpret_cast<Cand *>(p);
    p += align_up(np * g.ref_cap * sizeof(Cand));
    ra.rs.exact = reinterpret_cast<float2 *>(p);
    p += align_up(np * g.ref_cap * sizeof(float2));
    ra.rs.pmin = reinterpret_cast<unsigned *>(p);
    p += align_up(np * sizeof(unsigned));
    ra.rs.cnt = reinterpret_cast<int *>(p);
    p += align_up(np * sizeof(int));
    ra.rs.lvl = reinterpret_cast<unsigned long long *>(p);
    p += align_up(np * sizeof(unsigned long long));
    ra.rs.wsum = reinterpret_cast<unsigned long long *>(p);
    p += align_up(np * sizeof(unsigned long long));
    ra.rs.done = reinterpret_cast<unsigned *>(p);
    p += align_up(np * sizeof(unsigned));
    ra.win = reinterpret_cast<float *>(p);
    p += align_up((size_t)g.K * sizeof(float));
    ra.bnd = reinterpret_cast<float *>(p);
    p += align_up((size_t)g.K * sizeof(float));
  }
  // every buffer of the batch lies inside the region the plan set aside
  if ((size_t)(p - ws) > ws_avail) {
    last_msg = "internal: batch buffers exceed the planned workspace";
    throw Fail{BPMF_ERR_CUDA};
  }
  if (g.occ_cap > 0 && d_tabs) {
    OccRunsArgs ra{lg->coords, lg->R, d_meta, (float)h, g.occ_cap, runs, n_runs, g.occ_rb};
    launch(c, "k_occ_runs", st, [&] { return launch_occ_runs(ra, batch, st); });
    ClashArgs ca{};
    ca.runs = runs;
    ca.n_runs = n_runs;
    ca.cap = g.occ_cap;
    ca.tabs = d_tabs;
    ca.info = d_info;
    ca.K = g.K;
    ca.S0 = g.S[0];
    ca.S1 = g.S[1];
    ca.S2 = g.S[2];
    ca.CW = CW;
    ca.clash = clash;
    launch(c, "k_clash", st, [&] { return launch_clash(ca, batch, st); });
  }
  if (g.refine) {
    ra.rs.win = ra.win;
    ra.rs.bnd = ra.bnd;
    ra.rs.cap = g.ref_cap;
    ra.rs.fail = rf->fail;
    ra.meta = d_meta;
    ra.info = d_info;
    ra.tabs = rf->rtabs;
    for (int t = 0; t < 3; ++t) ra.gnorm[t] = (float)rf->gnorm[t];
    ra.log2P3 = (float)std::log2((double)g.P[0] * g.P[1] * g.P[2]);
    ra.check_scale = rf->check_scale;
    ra.bound_scale = rf->bound_scale;
    ra.coords = lg->coords;
    ra.gamma = lg->gamma;
    ra.gamma_stride = (int)lg->total_atoms;
    ra.kT = (float)rf->kT;
    split_ff(-1.0 / rf->kT, ra.nikT_hi, ra.nikT_lo);
    ra.K = g.K;
    ra.S0 = g.S[0];
    ra.S1 = g.S[1];
    ra.S2 = g.S[2];
    ra.part_ref = rf->part_ref;
    ra.export_E = export_E;
    ra.store = rf->store;
    ra.order = rf->order;
    ra.kmap = rf->kmap;
    ra.Kall = rf->Kall;
    ra.seeded = rf->seeded ? 1 : 0;
    launch(c, "k_refine_init", st, [&] { return launch_refine_init(ra, batch, st); });
  }

  float hh, hl;
  split_ff(h, hh, hl);
  if (sizeof(T) == 4 && !split) {
    // FP32 forms: the y-z spectra straight from the atoms (spreading + z and y passes in one)
    LigSpecArgs la{};
    la.coords = lg->coords;
    la.gamma = lg->gamma;
    la.gamma_stride = (int)lg->total_atoms;
    la.meta = d_meta;
    la.h_hi = hh;
    la.h_lo = hl;
    la.U0 = g.U[0];
    la.U1 = g.U[1];
    la.U2 = g.U[2];
    la.P1 = g.P[1];
    la.P2 = g.P[2];
    la.F2 = g.F2;
    la.Q = g.Q;
    la.tw1 = twiddles(c, g.P[1]);
    la.tw2 = twiddles(c, g.P[2]);
    la.ly = reinterpret_cast<float2 *>(ly);
    la.nmax = g.nmax;
    launch(c, "k_ligspec", st, [&] { return launch_ligspec(la, batch, st); });
  } else {
    SpreadArgs sa{lg->coords, lg->gamma, (int)lg->total_atoms, d_meta, hh, hl, g.U[0], g.U[1], g.U[2], box};
    launch(c, "k_spread", st, [&] { return launch_spread(sa, batch, st); });

    ZfwdArgs za{};
    za.in = reinterpret_cast<const float *>(box);
    za.in_pairs = 1;
    za.n_rows = 3ll * batch * g.U[0] * g.U[1];
    za.w_in = g.U[2];
    za.in_stride = g.U[2];
    za.out = lz;
    za.out_stride = g.F2;
    za.plan = plan(g.P[2]);
    za.tw = twiddles(c, g.P[2]);
    za.L = tn.zfwd_l;
    launch(c, sizeof(T) == 4 ? "k_zfwd<fp32>" : "k_zfwd<ff>", st, [&] { return launch_zfwd<T>(za, st); });

    AxisArgs ya{};
    ya.in = lz;
    ya.out = ly;
    ya.P = g.P[1];
    ya.n_in = g.U[1];
    ya.n_out = g.P[1];
    ya.n_outer = 3ll * batch * g.U[0];
    ya.inner = g.F2;
    ya.in_os = (long long)g.U[1] * g.F2;
    ya.out_os = (long long)g.P[1] * g.F2;
    ya.info = nullptr;
    ya.w0_div = 1;
    ya.axis = 1;
    ya.inverse = 0;
    ya.plan = plan(g.P[1]);
    ya.tw = twiddles(c, g.P[1]);
    ya.LW = tn.axis_lw > 0 ? tn.axis_lw : (sizeof(T) == 4 ? 32 : 16);
    launch(c, sizeof(T) == 4 ? "k_axis<fp32>(y fwd)" : "k_axis<ff>(y fwd)", st, [&] { return launch_axis<T>(ya, st); });
  }

  XfusedArgs xa{};
  xa.ly = ly;
  xa.U0 = g.U[0];
  xa.meta = d_meta;
  xa.rhi_h = h_rhi;
  xa.err = d_err;
  xa.wait_test = c->wait_test;
  xa.Q = g.Q;
  xa.K = g.K;
  xa.rhi = d_rhi;
  xa.rlo = d_rlo;
  xa.x2 = x2;
  xa.S0 = g.S[0];
  xa.info = d_info;
  xa.plan = plan(g.P[0]);
  xa.tw = twiddles(c, g.P[0]);
  if (sizeof(T) == 4 && !split && xpass_supported(g.P[0]))  // FP32 on a compile-time edge
    launch(c, "k_xpass<fp32>", st, [&] { return launch_xpass(xa, batch, st); });
  else
    launch(c, sizeof(T) == 4 ? "k_xfused<fp32>" : "k_xfused<ff>", st, [&] { return launch_xfused<T>(xa, batch, st); });

  // FP32 forms: the y and z inverses in one compile-time kernel on the edges
  // it has; else the y inverse inside the z inverse when the window fits
  const bool yz = sizeof(T) == 4 && !split &&
                  yzinv_supported(g.P[1], g.P[2], g.S[1], g.S[2], clash != nullptr, export_E != nullptr);
  const bool fuse_y =
      !yz && sizeof(T) == 4 && !split && zinv_fused_fits(g.P[1], g.P[2], g.S[1], g.S[2], g.refine);
  if (!fuse_y && !yz) {
    AxisArgs yi{};
    yi.in = x2;
    yi.out = y2;
    yi.P = g.P[1];
    yi.n_in = g.P[1];
    yi.n_out = g.S[1];
    yi.n_outer = (long long)batch * g.K * g.S[0];
    yi.inner = g.F2;
    yi.in_os = g.Q;
    yi.out_os = (long long)g.S[1] * g.F2;
    yi.info = d_info;
    yi.w0_div = g.S[0];
    yi.axis = 1;
    yi.inverse = 1;
    yi.plan = plan(g.P[1]);
    yi.tw = twiddles(c, g.P[1]);
    yi.LW = tn.axis_lw > 0 ? tn.axis_lw : (sizeof(T) == 4 ? 32 : 16);
    launch(c, sizeof(T) == 4 ? "k_axis<fp32>(y inv)" : "k_axis<ff>(y inv)", st, [&] { return launch_axis<T>(yi, st); });
  }

  ZinvArgs zi{};
  zi.y2 = y2;
  zi.K = g.K;
  zi.S0 = g.S[0];
  zi.S1 = g.S[1];
  zi.S2 = g.S[2];
  zi.F2 = g.F2;
  zi.info = d_info;
  zi.nscale_hi = nscale_hi;
  zi.nscale_lo = nscale_lo;
  zi.escale_hi = escale_hi;
  zi.escale_lo = escale_lo;
  zi.part = d_part;
  zi.export_E = export_E;  // refined form: k_refine overwrites the refined translations with exact values
  if (g.refine) zi.rs = ra.rs;
  zi.clash = clash;
  zi.CW = CW;
  zi.plan = plan(g.P[2]);
  zi.tw = twiddles(c, g.P[2]);
  if (fuse_y || yz) {
    zi.x2 = x2;
    zi.Qx = g.Q;
    zi.yplan = plan(g.P[1]);
    zi.tw1 = twiddles(c, g.P[1]);
  }
  if (yz)
    launch(c, "k_yzinv<fp32>", st, [&] { return launch_yzinv(zi, batch, st); });
  else
    launch(c, fuse_y ? "k_zinv<fp32>(+y inv)" : (sizeof(T) == 4 ? "k_zinv<fp32>" : "k_zinv<ff>"), st,
           [&] { return launch_zinv<T>(zi, batch, st); });
  if (g.refine) {
    ra.h_hi = hh;
    ra.h_lo = hl;
    launch(c, "k_refine", st, [&] { return launch_refine(ra, batch, st); });
  }
}

void check_recs(const bpmf_rec_t *recs, int K, bpmf_ctx *c) {
  for (int k = 0; k < K; ++k) {
    if (!recs[k] || recs[k]->ctx != c) throw Fail{BPMF_ERR_INVALID_ARG};
    if (recs[k]->h != recs[0]->h) {
      last_msg = "receptors in one bpmf_eval call must share the grid spacing";
      throw Fail{BPMF_ERR_SIZE_UNSUPPORTED};
    }
  }
}

// Host-side per-ligand tables: placement metadata per configuration and the
// site window / valid count per (configuration, receptor).
void ligand_tables(const bpmf_lig *lg, int li, const bpmf_rec_t *recs, int K, double h, std::vector<ConfMeta> &meta,
                   std::vector<PairInfo> &info, std::vector<long long> &nvalid) {
  const int J = lg->n_conf[li];
  const float hf = (float)h;
  meta.resize(J);
  info.resize((size_t)J * K);
  nvalid.resize((size_t)J * K);
  for (int j = 0; j < J; ++j) {
    const long long cj = lg->conf_off[li] + j;
    const float *mm = &lg->minmax[6 * cj];
    ConfMeta m{};
    for (int d = 0; d < 3; ++d) {
      m.lo[d] = mm[d];
      m.u[d] = box_extent(mm[d], mm[3 + d], hf);
    }
    m.atom_off = (int)(lg->coord_off[li] + (long long)j * lg->n_atoms[li]);
    m.n_atoms = lg->n_atoms[li];
    m.gamma_off = lg->atom_off[li];
    meta[j] = m;
    for (int k = 0; k < K; ++k) {
      PairInfo pi{};
      long long n = 1;
      for (int d = 0; d < 3; ++d) {
        n *= site_window(recs[k]->N[d], recs[k]->site_lo[d], recs[k]->site_n[d], m.u[d], pi.w0[d], pi.sa[d],
                         pi.sb[d]);
        pi.wc[d] = pi.w0[d];  // uncropped transforms
      }
      info[(size_t)j * K + k] = pi;
      nvalid[(size_t)j * K + k] = n;
    }
  }
}

}  // namespace

// ------------------------------------------- accessors for bpmf_proposal.cu
int bpmf_internal_device(bpmf_ctx_t c) { return c ? c->device : 0; }
void bpmf_internal_set_error(bpmf_ctx_t c, const std::string &m) {
  if (c) c->err = m;
}
int bpmf_internal_ligand_arrays(bpmf_lig_t lg, const float **coords, const float **q, const float **eps,
                                const float **R, std::vector<int> *conf_off, std::vector<int> *conf_nat,
                                std::vector<int> *conf_lig, std::vector<int> *lig_atom_off) {
  if (!lg) return BPMF_ERR_INVALID_ARG;
  *coords = lg->coords;
  *q = lg->q;
  *eps = lg->eps;
  *R = lg->R;
  conf_off->clear();
  conf_nat->clear();
  conf_lig->clear();
  lig_atom_off->assign(lg->atom_off.begin(), lg->atom_off.end());
  for (int i = 0; i < lg->n_lig; ++i)
    for (int j = 0; j < lg->n_conf[i]; ++j) {
      conf_off->push_back(lg->coord_off[i] + j * lg->n_atoms[i]);
      conf_nat->push_back(lg->n_atoms[i]);
      conf_lig->push_back(i);
    }
  return BPMF_OK;
}

// ===================================================================== ABI
extern "C" {

const char *bpmf_status_string(int s) {
  switch (s) {
    case BPMF_OK: return "ok";
    case BPMF_ERR_INVALID_ARG: return "invalid argument";
    case BPMF_ERR_OOM: return "out of device memory";
    case BPMF_ERR_CUDA: return "CUDA error";
    case BPMF_ERR_TIMEOUT: return "timeout";
    case BPMF_ERR_SIZE_UNSUPPORTED: return "size unsupported";
    case BPMF_WARN_NO_VALID: return "warning: some configuration has no valid translation";
    case BPMF_WARN_REFINE_FALLBACK:
      return "warning: refined-form certificate failed; the ligand was recomputed in float pairs";
    case BPMF_WARN_NO_VALID | BPMF_WARN_REFINE_FALLBACK:
      return "warnings: some configuration has no valid translation; a ligand was recomputed in float pairs";
    default: return "unknown status";
  }
}

const char *bpmf_last_error(bpmf_ctx_t ctx) { return ctx ? ctx->err.c_str() : ""; }

int bpmf_fft_edge(int n) { return n >= 1 ? smooth_edge(n) : 0; }

int bpmf_profile_enable(bpmf_ctx_t c, int on) {
  if (!c) return BPMF_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  try {
    prof_drain(c);
  } catch (Fail f) {
    return set_err(c, f.code, last_msg);
  }
  c->prof = on != 0;
  if (c->prof) {
    c->prof_names.clear();
    c->prof_ms.clear();
    c->prof_n.clear();
  }
  return BPMF_OK;
}

int bpmf_profile_count(bpmf_ctx_t c) {
  if (!c) return BPMF_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  try {
    prof_drain(c);
  } catch (Fail f) {
    return set_err(c, f.code, last_msg);
  }
  return (int)c->prof_names.size();
}

int bpmf_profile_entry(bpmf_ctx_t c, int i, char *name, int name_len, double *total_ms, int64_t *launches) {
  if (!c || i < 0 || i >= (int)c->prof_names.size()) return BPMF_ERR_INVALID_ARG;
  if (name && name_len > 0) {
    std::strncpy(name, c->prof_names[i].c_str(), (size_t)name_len - 1);
    name[name_len - 1] = '\0';
  }
  if (total_ms) *total_ms = c->prof_ms[i];
  if (launches) *launches = c->prof_n[i];
  return BPMF_OK;
}

int bpmf_valid_counts(bpmf_ctx_t c, bpmf_lig_t lg, const bpmf_rec_t *recs, int K, int64_t *n_valid) {
  if (!c || !lg || !recs || K < 1 || !n_valid || lg->ctx != c) return set_err(c, BPMF_ERR_INVALID_ARG, "null argument");
  try {
    last_msg.clear();
    check_recs(recs, K, c);
    std::vector<ConfMeta> meta;
    std::vector<PairInfo> info;
    std::vector<long long> nv;
    long long off = 0;
    for (int li = 0; li < lg->n_lig; ++li) {
      ligand_tables(lg, li, recs, K, recs[0]->h, meta, info, nv);
      for (size_t i = 0; i < (size_t)lg->n_conf[li] * K; ++i) n_valid[off + i] = nv[i];
      off += (long long)lg->n_conf[li] * K;
    }
  } catch (Fail f) {
    return set_err(c, f.code, last_msg);
  }
  return BPMF_OK;
}

int bpmf_set_graph_mode(bpmf_ctx_t c, int on) {
  if (!c) return BPMF_ERR_INVALID_ARG;
  c->graph_mode = on != 0;
  return BPMF_OK;
}

int bpmf_set_refine_check_scale(bpmf_ctx_t c, double scale) {
  if (!c || !(scale >= 0.0)) return set_err(c, BPMF_ERR_INVALID_ARG, "scale must be >= 0");
  c->refine_check_scale = (float)scale;
  return BPMF_OK;
}

int bpmf_set_refine_list_cap(bpmf_ctx_t c, int cap) {
  if (!c || cap < 0) return set_err(c, BPMF_ERR_INVALID_ARG, "cap must be >= 0");
  c->refine_list_cap = cap;
  return BPMF_OK;
}

int bpmf_set_wait_test(bpmf_ctx_t c, int on) {
  if (!c) return BPMF_ERR_INVALID_ARG;
  c->wait_test = on != 0;
  return BPMF_OK;
}

int bpmf_set_workspace_limit(bpmf_ctx_t c, size_t bytes) {
  if (!c || bytes < (size_t(1) << 20)) return set_err(c, BPMF_ERR_INVALID_ARG, "workspace limit below 1 MiB");
  c->ws_budget = bytes;
  return BPMF_OK;
}

int bpmf_create(int device, bpmf_ctx_t *out) {
  if (!out) return BPMF_ERR_INVALID_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return BPMF_ERR_CUDA;
  }
  if (device < 0 || device >= n) return BPMF_ERR_INVALID_ARG;
  bpmf_ctx *c = new (std::nothrow) bpmf_ctx();
  if (!c) return BPMF_ERR_OOM;
  c->device = device;
  DeviceGuard g(device);
  if (cudaFree(nullptr) != cudaSuccess) {  // establish the primary context
    cudaGetLastError();
    delete c;
    return BPMF_ERR_CUDA;
  }
  // workspace budget: an eighth of the device's memory, at most 16 GiB and at
  // least 1 GiB (larger batches mean fewer, fuller launches)
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
    c->ws_budget = std::min(size_t(16) << 30, std::max(size_t(1) << 30, total_b / 8));
  else
    cudaGetLastError();
  *out = c;
  return BPMF_OK;
}

void bpmf_destroy(bpmf_ctx_t c) {
  if (!c) return;
  DeviceGuard g(c->device);
  for (auto &kv : c->tw) cudaFree(kv.second);
  for (cudaStream_t &x : c->side)
    if (x) cudaStreamDestroy(x);
  if (c->copy_st) cudaStreamDestroy(c->copy_st);
  if (c->copy_ev) cudaEventDestroy(c->copy_ev);
  for (auto &kv : c->blocks) cudaFree(kv.second);
  if (c->tca) cudaFree(c->tca);
  if (c->tc05) cudaFree(const_cast<__nv_bfloat16 *>(c->tc05));
  if (c->pmin_store) cudaFree(c->pmin_store);
  if (c->ws) cudaFree(c->ws);
  for (auto &r : c->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->event_pool) cudaEventDestroy(e);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->pinned_busy) {
    cudaEventSynchronize(c->pinned_busy);
    cudaEventDestroy(c->pinned_busy);
  }
  if (c->pinned) cudaFreeHost(c->pinned);
  if (c->fail_host) cudaFreeHost(c->fail_host);
  delete c;
}

namespace {

// Float-pair receptor passes (Eq. fft_correlation_func's FT(G_R)), used by
// the loads and the crops.  z: R2C of `rows` rows of w_in floats (stride
// in_stride, zero beyond w_in) on edge Pz -> out [rows][Pz/2+1].
void rz_pass(bpmf_ctx *c, const float *in, long long rows, int w_in, long long in_stride, int Pz, void *out,
             cudaStream_t st) {
  ZfwdArgs za{};
  za.in = in;
  za.n_rows = rows;
  za.w_in = w_in;
  za.in_stride = in_stride;
  za.out = out;
  za.out_stride = Pz / 2 + 1;
  za.plan = make_plan(Pz);
  za.tw = twiddles(c, Pz);
  za.L = 16;
  launch(c, "k_zfwd<ff>(receptor)", st, [&] { return launch_zfwd<ff>(za, st); });
}

// y (axis 1) or x (axis 0): C2C on edge Pd of n_outer x inner columns whose
// n_in inputs lie `inner` apart (zero beyond n_in), outer blocks in_os apart
// -> out [n_outer][Pd][inner].
void rax_pass(bpmf_ctx *c, const void *in, int n_in, int Pd, long long n_outer, long long inner, long long in_os,
              void *out, int axis, cudaStream_t st, float2 *out_hi = nullptr, float2 *out_lo = nullptr) {
  AxisArgs ax{};
  ax.out_hi = out_hi;
  ax.out_lo = out_lo;
  ax.in = in;
  ax.out = out;
  ax.P = Pd;
  ax.n_in = n_in;
  ax.n_out = Pd;
  ax.n_outer = n_outer;
  ax.inner = inner;
  ax.in_os = in_os;
  ax.out_os = (long long)Pd * inner;
  ax.w0_div = 1;
  ax.axis = axis;
  ax.plan = make_plan(Pd);
  ax.tw = twiddles(c, Pd);
  ax.LW = 16;
  launch(c, axis == 1 ? "k_axis<ff>(receptor y)" : "k_axis<ff>(receptor x)", st,
         [&] { return launch_axis<ff>(ax, st); });
}

// The x pass of a y stage [3][N0][Q] over its rows [x0, x0 + n_in) on edge
// Px, written as the spectrum's hi / lo planes [3][Px][Q].
void rx_split(bpmf_ctx *c, const void *ystage, int N0, int x0, int n_in, int Px, long long Q, float2 *hi, float2 *lo,
              cudaStream_t st) {
  rax_pass(c, static_cast<const cx<ff> *>(ystage) + (long long)x0 * Q, n_in, Px, 3, Q, (long long)N0 * Q, nullptr, 0,
           st, hi, lo);
}

// A stage of a receptor (made on `st` and recorded there), in blocks of the
// context's cache.
bpmf_rec::Stage new_stage(bpmf_ctx *c, size_t bytes) {
  bpmf_rec::Stage sg;
  Carve cv;
  cv.add(&sg.v, bytes);
  sg.mem = cv.alloc(c);
  sg.mem_bytes = cv.total;
  return sg;
}
void record_stage(bpmf_rec::Stage &sg, cudaStream_t st) {
  if (!sg.ev) CK(cudaEventCreateWithFlags(&sg.ev, cudaEventDisableTiming));
  CK(cudaEventRecord(sg.ev, st));
}

// The z stage of receptor r for the z edge Pz (the crop along z starts at z0
// with ez nodes), made on st if new; st is ordered after it.
const bpmf_rec::Stage &z_stage(bpmf_ctx *c, bpmf_rec *r, int Pz, int z0, int ez, cudaStream_t st) {
  auto it = r->zst.find(Pz);
  if (it != r->zst.end()) {
    CK(cudaStreamWaitEvent(st, it->second.ev, 0));
    return it->second;
  }
  const long long rows = 3ll * r->N[0] * r->N[1];
  bpmf_rec::Stage sg = new_stage(c, rows * (Pz / 2 + 1) * sizeof(cx<ff>));
  try {
    rz_pass(c, r->grid + z0, rows, ez, r->N[2], Pz, sg.v, st);
    record_stage(sg, st);
  } catch (Fail) {
    cudaFree(sg.mem);
    if (sg.ev) cudaEventDestroy(sg.ev);
    throw;
  }
  return r->zst[Pz] = sg;
}

// The y stage of receptor r for the edges (Py, Pz): the y pass of its z stage
// with y cropped to [y0, y0 + ey), made on st if new; st is ordered after it.
const bpmf_rec::Stage &y_stage(bpmf_ctx *c, bpmf_rec *r, int Py, int y0, int ey, int Pz, int z0, int ez,
                               cudaStream_t st) {
  const auto key = std::make_pair(Py, Pz);
  auto it = r->yst.find(key);
  if (it != r->yst.end()) {
    CK(cudaStreamWaitEvent(st, it->second.ev, 0));
    return it->second;
  }
  const bpmf_rec::Stage &zs = z_stage(c, r, Pz, z0, ez, st);
  const long long Fz = Pz / 2 + 1;
  bpmf_rec::Stage sg = new_stage(c, 3ull * r->N[0] * Py * Fz * sizeof(cx<ff>));
  try {
    rax_pass(c, static_cast<const cx<ff> *>(zs.v) + (long long)y0 * Fz, ey, Py, 3ll * r->N[0], Fz,
             (long long)r->N[1] * Fz, sg.v, 1, st);
    record_stage(sg, st);
  } catch (Fail) {
    cudaFree(sg.mem);
    if (sg.ev) cudaEventDestroy(sg.ev);
    throw;
  }
  return r->yst[key] = sg;
}

int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// First node of a crop of edge Pc around the site [site_lo, site_lo + site_n)
// of a grid of N nodes: floor((site_n - Pc) / 2) nodes from the site, moved
// inside the grid.
int crop_start(int N, int site_lo, int site_n, int Pc) {
  const int c0 = site_lo + floor_div(site_n - Pc, 2);
  return std::max(0, std::min(c0, std::max(0, N - Pc)));
}

// Views of receptors' spectra for transform edges Pc <= P: the stored one of
// a receptor when Pc == P, else its grids cropped to Pc nodes per axis around
// the site.  Crops made on first use run on one of the library's side
// streams after the event `fork` of the caller's stream; the event recorded
// when they are done is appended to `joins` (the caller's stream waits for
// it) and the receptors made to `touched`.  A crop's spectrum is the x pass,
// over the crop's x rows, of the receptor's y stage for (Pc1, Pc2) (the y
// pass, over the crop's y rows, of its z stage for Pc2, the z pass over the
// crop's z nodes): cropping along one axis commutes with the transforms
// along the others, so crops that share edges share stages.
// Every node that a translation of the site window reaches with a ligand box
// of edge u lies in the crop when Pc >= site_n + u - 1: the crop starts
// floor((site_n - Pc) / 2) nodes from the site, moved inside the grid.
std::vector<bpmf_rec::Crop> rec_crops(bpmf_ctx *c, const std::vector<bpmf_rec *> &rs, const std::array<int, 3> &Pc,
                                      cudaEvent_t fork, std::vector<cudaEvent_t> &joins,
                                      std::vector<bpmf_rec *> &touched) {
  std::vector<bpmf_rec::Crop> out(rs.size());
  std::vector<size_t> todo;
  std::vector<std::array<int, 3>> ext;
  std::vector<int> alias(rs.size(), -1);  // a receptor passed more than once
  for (size_t m = 0; m < rs.size(); ++m) {
    bpmf_rec *r = rs[m];
    for (size_t m2 = 0; m2 < m && alias[m] < 0; ++m2)
      if (rs[m2] == r) alias[m] = (int)m2;
    if (alias[m] >= 0) continue;
    if (Pc[0] == r->P[0] && Pc[1] == r->P[1] && Pc[2] == r->P[2]) {
      out[m].hi = r->hi;
      out[m].lo = r->lo;
      out[m].sumsq = r->sumsq;
      out[m].vol = (double)r->N[0] * r->N[1] * r->N[2];
      continue;
    }
    auto it = r->crops.find(Pc);
    if (it != r->crops.end()) {
      out[m] = it->second;
      continue;
    }
    std::array<int, 3> e{};
    for (int d = 0; d < 3; ++d) {
      out[m].c0[d] = crop_start(r->N[d], r->site_lo[d], r->site_n[d], Pc[d]);
      e[d] = std::min(Pc[d], r->N[d] - out[m].c0[d]);
    }
    out[m].vol = (double)e[0] * e[1] * e[2];
    todo.push_back(m);
    ext.push_back(e);
  }
  auto resolve = [&] {
    for (size_t m = 0; m < rs.size(); ++m)
      if (alias[m] >= 0) out[m] = out[alias[m]];
  };
  if (todo.empty()) {
    resolve();
    return out;
  }
  const int n = (int)todo.size();
  const long long Q = (long long)Pc[1] * (Pc[2] / 2 + 1);
  cudaStream_t &cs_slot = c->side[c->side_next++ % bpmf_ctx::kSide];
  if (!cs_slot) CK(cudaStreamCreateWithFlags(&cs_slot, cudaStreamNonBlocking));
  const cudaStream_t st = cs_slot;
  CK(cudaStreamWaitEvent(st, fork, 0));
  try {
    for (int i = 0; i < n; ++i) {
      bpmf_rec::Crop &cr = out[todo[i]];
      Carve cv;
      cv.add(&cr.hi, 3ull * Pc[0] * Q * sizeof(float2));
      cv.add(&cr.lo, 3ull * Pc[0] * Q * sizeof(float2));
      cv.add(&cr.sumsq, 3 * sizeof(float));
      cv.add(&cr.sumsq_scratch, kSumsqScratch * sizeof(float2));
      cr.mem = cv.alloc(c);
      cr.mem_bytes = cv.total;
    }
    // per receptor: the sums of squares over the crop, then the x pass of
    // the y stage for (Pc1, Pc2) over the crop's x rows (the stages are made
    // once per receptor and edge pair and shared by the crops that use them)
    for (int i = 0; i < n; ++i) {
      bpmf_rec *r = rs[todo[i]];
      bpmf_rec::Crop &cr = out[todo[i]];
      const int e[3] = {ext[i][0], ext[i][1], ext[i][2]};
      launch(c, "k_crop", st,
             [&] { return launch_crop(r->grid, r->N, cr.c0, e, e, nullptr, cr.sumsq, cr.sumsq_scratch, st); });
      const bpmf_rec::Stage &ys = y_stage(c, r, Pc[1], cr.c0[1], e[1], Pc[2], cr.c0[2], e[2], st);
      rx_split(c, ys.v, r->N[0], cr.c0[0], e[0], Pc[0], Q, cr.hi, cr.lo, st);
    }
  } catch (Fail) {
    cudaStreamSynchronize(st);
    for (int i = 0; i < n; ++i)
      if (out[todo[i]].mem) cudaFree(out[todo[i]].mem);
    throw;
  }
  cudaEvent_t done = pool_event(c);
  CK(cudaEventRecord(done, st));
  joins.push_back(done);
  for (int i = 0; i < n; ++i) {
    bpmf_rec *r = rs[todo[i]];
    r->crops[Pc] = out[todo[i]];
    touched.push_back(r);
  }
  resolve();
  return out;
}

// Transform edge of a crop that holds a reach of W nodes: the full edge P,
// or the smooth edge near 5P/6 when W fits in it.
int crop_edge(int W, int P) {
  const int p1 = smooth_edge((5 * P + 5) / 6);
  return (p1 > 0 && p1 < P && W <= p1) ? p1 : P;
}

}  // namespace

int bpmf_crop_window(int n, int site_lo, int site_n, int u, int *edge, int *c0) {
  if (!edge || !c0 || n < 2 || site_n < 1 || u < 1) return BPMF_ERR_INVALID_ARG;
  const int P = smooth_edge(n);
  if (!P) return BPMF_ERR_SIZE_UNSUPPORTED;
  const int Pc = crop_edge(site_n + std::min(u, P) - 1, P);
  *edge = Pc;
  *c0 = Pc == P ? 0 : crop_start(n, site_lo, site_n, Pc);
  return BPMF_OK;
}

int bpmf_receptor_load(bpmf_ctx_t c, const float *grids, int nx, int ny, int nz, double h, const double origin[3],
                       const int site_lo[3], const int site_n[3], void *stream, bpmf_rec_t *out) {
  if (!c || !out || !grids || !site_lo || !site_n) return set_err(c, BPMF_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2 || !(h > 0.0))
    return set_err(c, BPMF_ERR_INVALID_ARG, "grid edges must be >= 2 and h > 0");
  for (int d = 0; d < 3; ++d)
    if (site_n[d] < 1) return set_err(c, BPMF_ERR_INVALID_ARG, "site_n must be >= 1");
  const int N[3] = {nx, ny, nz};
  int P[3];
  for (int d = 0; d < 3; ++d) {
    P[d] = smooth_edge(N[d]);
    if (!P[d]) return set_err(c, BPMF_ERR_SIZE_UNSUPPORTED, "padded FFT edge exceeds BPMF_MAX_FFT_EDGE");
  }
  DeviceGuard dg(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  bpmf_rec *r = new (std::nothrow) bpmf_rec();
  if (!r) return set_err(c, BPMF_ERR_OOM, "host allocation");
  try {
    r->ctx = c;
    r->id = c->next_id++;
    for (int d = 0; d < 3; ++d) {
      r->N[d] = N[d];
      r->P[d] = P[d];
      r->site_lo[d] = site_lo[d];
      r->site_n[d] = site_n[d];
      r->origin[d] = origin ? origin[d] : 0.0;
    }
    r->h = h;
    r->F2 = P[2] / 2 + 1;
    r->Q = (long long)P[1] * r->F2;
    const size_t vol = (size_t)nx * ny * nz;
    // host grids: copied on the context's copy stream (not behind the work
    // already queued on st), which st then waits for; the call returns once
    // the copy is done, so the caller may reuse its buffer
    struct HostIn {
      const void *p = nullptr;
      void *own = nullptr;
      cudaStream_t st = nullptr;
      ~HostIn() {
        if (own) cudaFreeAsync(own, st);
      }
    } g;
    g.st = st;
    const bool host_grids = !is_device_ptr(grids);
    if (host_grids) {
      if (!c->copy_st) CK(cudaStreamCreateWithFlags(&c->copy_st, cudaStreamNonBlocking));
      if (!c->copy_ev) CK(cudaEventCreateWithFlags(&c->copy_ev, cudaEventDisableTiming));
      CK(cudaMallocAsync(&g.own, 3 * vol * sizeof(float), c->copy_st));
      CK(cudaMemcpyAsync(g.own, grids, 3 * vol * sizeof(float), cudaMemcpyHostToDevice, c->copy_st));
      CK(cudaEventRecord(c->copy_ev, c->copy_st));
      CK(cudaStreamWaitEvent(st, c->copy_ev, 0));
      g.p = g.own;
    } else {
      g.p = grids;
    }
    Carve cv;
    cv.add(&r->grid, 3 * vol * sizeof(float));
    cv.add(&r->sumsq, 3 * sizeof(float));
    cv.add(&r->sumsq_scratch, kSumsqScratch * sizeof(float2));
    cv.add(&r->hi, 3ull * P[0] * r->Q * sizeof(float2));
    cv.add(&r->lo, 3ull * P[0] * r->Q * sizeof(float2));
    r->mem = cv.alloc(c);
    r->mem_bytes = cv.total;
    // the grids copied into the receptor's block with their sums of squares
    launch(c, "k_sumsq", st, [&] {
      return launch_sumsq(static_cast<const float *>(g.p), N, r->grid, r->sumsq, r->sumsq_scratch, st);
    });
    // the float-pair spectrum, z then y then x; the z and y stages are kept
    // for the crops (the uncropped stages of every crop with a full z, or
    // full y and z, edge)
    {
      const long long rows = 3ll * N[0] * N[1];
      bpmf_rec::Stage zs = new_stage(c, rows * r->F2 * sizeof(cx<ff>));
      r->zst[P[2]] = zs;
      rz_pass(c, static_cast<const float *>(g.p), rows, N[2], N[2], P[2], zs.v, st);
      record_stage(r->zst[P[2]], st);
      bpmf_rec::Stage ys = new_stage(c, 3ull * N[0] * r->Q * sizeof(cx<ff>));
      r->yst[std::make_pair(P[1], P[2])] = ys;
      rax_pass(c, zs.v, N[1], P[1], 3ll * N[0], r->F2, (long long)N[1] * r->F2, ys.v, 1, st);
      record_stage(r->yst[std::make_pair(P[1], P[2])], st);
      rx_split(c, ys.v, N[0], 0, N[0], P[0], r->Q, r->hi, r->lo, st);
    }
    if (host_grids) CK(cudaEventSynchronize(c->copy_ev));
  } catch (Fail f) {
    bpmf_receptor_free(r);
    return set_err(c, f.code, last_msg);
  }
  *out = r;
  c->err.clear();
  return BPMF_OK;
}

void bpmf_receptor_free(bpmf_rec_t r) {
  if (!r) return;
  if (r->ctx) {
    DeviceGuard g(r->ctx->device);
    // blocks return to the context's cache once no queued work can read them
    const bool idle = cudaDeviceSynchronize() == cudaSuccess;
    if (!idle) cudaGetLastError();
    auto put = [&](void *p, size_t bytes) {
      if (idle)
        block_put(r->ctx, p, bytes);
      else if (p)
        cudaFree(p);
    };
    put(r->mem, r->mem_bytes);
    if (r->occ) cudaFree(r->occ);
    if (r->crop_ev) cudaEventDestroy(r->crop_ev);
    for (auto &kv : r->crops) put(kv.second.mem, kv.second.mem_bytes);
    for (auto &kv : r->zst) {
      put(kv.second.mem, kv.second.mem_bytes);
      if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    }
    for (auto &kv : r->yst) {
      put(kv.second.mem, kv.second.mem_bytes);
      if (kv.second.ev) cudaEventDestroy(kv.second.ev);
    }
  }
  delete r;
}

int bpmf_receptor_set_occupancy(bpmf_ctx_t c, bpmf_rec_t r, const uint8_t *occ, void *stream) {
  if (!c || !r || r->ctx != c) return set_err(c, BPMF_ERR_INVALID_ARG, "null receptor or receptor of another context");
  DeviceGuard dg(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t *tab = nullptr;
  try {
    last_msg.clear();
    if (occ) {
      const int W = (r->N[2] + kOccZPad + 31) / 32 + 2;
      const size_t words = (size_t)kOccLevels * (r->N[0] + 2 * kOccXYPad) * W * (r->N[1] + 2 * kOccXYPad);
      DevIn o(occ, (size_t)r->N[0] * r->N[1] * r->N[2], st);
      CK(cudaMalloc(&tab, words * sizeof(uint32_t)));
      launch(c, "k_occ_table", st, [&] {
        return launch_occ_table(static_cast<const unsigned char *>(o.p), r->N[0], r->N[1], r->N[2], W, tab, st);
      });
      CK(cudaStreamSynchronize(st));
      if (r->occ) cudaFree(r->occ);
      r->occ = tab;
      r->occW = W;
      tab = nullptr;
    } else if (r->occ) {
      CK(cudaStreamSynchronize(st));
      cudaFree(r->occ);
      r->occ = nullptr;
      r->occW = 0;
    }
    r->id = c->next_id++;  // results change: a new identity for the graph cache
  } catch (Fail f) {
    if (tab) cudaFree(tab);
    return set_err(c, f.code, last_msg);
  }
  c->err.clear();
  return BPMF_OK;
}

int bpmf_ligand_batch(bpmf_ctx_t c, int n_lig, const int *n_atoms, const int *n_conf, const float *coords,
                      const float *q, const float *eps, const float *R, int p_rep, int p_att, void *stream,
                      bpmf_lig_t *out) {
  if (!c || !out || n_lig < 1 || !n_atoms || !n_conf || !q || !eps || !R)
    return set_err(c, BPMF_ERR_INVALID_ARG, "null argument or n_lig < 1");
  *out = nullptr;
  if (p_rep < 0 || p_rep > 32 || p_att < 0 || p_att > 32)
    return set_err(c, BPMF_ERR_INVALID_ARG, "exponents must lie in 0..32");
  bpmf_lig *lg = new (std::nothrow) bpmf_lig();
  if (!lg) return set_err(c, BPMF_ERR_OOM, "host allocation");
  DeviceGuard dg(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  int *d_off = nullptr, *d_nat = nullptr;
  float *d_mm = nullptr;
  try {
    lg->ctx = c;
    lg->id = c->next_id++;
    lg->n_lig = n_lig;
    lg->n_atoms.assign(n_atoms, n_atoms + n_lig);
    lg->n_conf.assign(n_conf, n_conf + n_lig);
    lg->atom_off.resize(n_lig);
    lg->conf_off.resize(n_lig);
    lg->coord_off.resize(n_lig);
    for (int i = 0; i < n_lig; ++i) {
      if (n_atoms[i] < 1 || n_conf[i] < 0) {
        last_msg = "n_atoms must be >= 1 and n_conf >= 0";
        throw Fail{BPMF_ERR_INVALID_ARG};
      }
      if (n_atoms[i] > BPMF_MAX_ATOMS) {
        last_msg = "ligand has more than BPMF_MAX_ATOMS atoms";
        throw Fail{BPMF_ERR_SIZE_UNSUPPORTED};
      }
      lg->atom_off[i] = (int)lg->total_atoms;
      lg->conf_off[i] = (int)lg->total_conf;
      lg->coord_off[i] = (int)lg->total_coord_atoms;
      lg->total_atoms += n_atoms[i];
      lg->total_conf += n_conf[i];
      lg->total_coord_atoms += (long long)n_conf[i] * n_atoms[i];
    }
    if (lg->total_coord_atoms > 0 && !coords) {
      last_msg = "coords is null";
      throw Fail{BPMF_ERR_INVALID_ARG};
    }
    const size_t na = lg->total_atoms;
    Carve cv;
    cv.add(&lg->gamma, 3 * na * sizeof(float2));
    cv.add(&lg->q, na * sizeof(float));
    cv.add(&lg->eps, na * sizeof(float));
    cv.add(&lg->R, na * sizeof(float));
    cv.add(&lg->coords, std::max<size_t>(1, 3 * lg->total_coord_atoms) * sizeof(float));
    lg->mem = cv.alloc(c);
    lg->mem_bytes = cv.total;
    CK(cudaMemcpyAsync(lg->q, q, na * sizeof(float), cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(lg->eps, eps, na * sizeof(float), cudaMemcpyDefault, st));
    CK(cudaMemcpyAsync(lg->R, R, na * sizeof(float), cudaMemcpyDefault, st));
    lg->R_host.resize(na);
    CK(cudaMemcpyAsync(lg->R_host.data(), lg->R, na * sizeof(float), cudaMemcpyDeviceToHost, st));
    lg->q_host.resize(na);
    lg->eps_host.resize(na);
    CK(cudaMemcpyAsync(lg->q_host.data(), lg->q, na * sizeof(float), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(lg->eps_host.data(), lg->eps, na * sizeof(float), cudaMemcpyDeviceToHost, st));
    lg->p_rep = p_rep;
    lg->p_att = p_att;
    {
      DevIn dq(q, na * sizeof(float), st), de(eps, na * sizeof(float), st), dr(R, na * sizeof(float), st);
      launch(c, "k_gamma", st, [&] {
        return launch_gamma((const float *)dq.p, (const float *)de.p, (const float *)dr.p, (int)na, p_rep, p_att,
                            lg->gamma, st);
      });
    }
    if (lg->total_coord_atoms > 0)
      CK(cudaMemcpyAsync(lg->coords, coords, 3 * lg->total_coord_atoms * sizeof(float), cudaMemcpyDefault, st));
    const long long TC = lg->total_conf;
    std::vector<int> off(std::max<long long>(TC, 1)), nat(std::max<long long>(TC, 1));
    for (int i = 0; i < n_lig; ++i)
      for (int j = 0; j < n_conf[i]; ++j) {
        off[lg->conf_off[i] + j] = lg->coord_off[i] + j * n_atoms[i];
        nat[lg->conf_off[i] + j] = n_atoms[i];
      }
    lg->minmax.assign(6 * std::max<long long>(TC, 1), 0.f);
    if (TC > 0) {
      CK(cudaMallocAsync(&d_off, TC * sizeof(int), st));
      CK(cudaMallocAsync(&d_nat, TC * sizeof(int), st));
      CK(cudaMallocAsync(&d_mm, 6 * TC * sizeof(float), st));
      CK(cudaMemcpyAsync(d_off, off.data(), TC * sizeof(int), cudaMemcpyHostToDevice, st));
      CK(cudaMemcpyAsync(d_nat, nat.data(), TC * sizeof(int), cudaMemcpyHostToDevice, st));
      launch(c, "k_minmax", st, [&] { return launch_minmax(lg->coords, d_off, d_nat, (int)TC, d_mm, st); });
      CK(cudaMemcpyAsync(lg->minmax.data(), d_mm, 6 * TC * sizeof(float), cudaMemcpyDeviceToHost, st));
      CK(cudaFreeAsync(d_off, st));
      d_off = nullptr;
      CK(cudaFreeAsync(d_nat, st));
      d_nat = nullptr;
      CK(cudaFreeAsync(d_mm, st));
      d_mm = nullptr;
    }
    CK(cudaStreamSynchronize(st));
  } catch (Fail f) {
    if (d_off) cudaFreeAsync(d_off, st);
    if (d_nat) cudaFreeAsync(d_nat, st);
    if (d_mm) cudaFreeAsync(d_mm, st);
    bpmf_ligand_free(lg);
    return set_err(c, f.code, last_msg);
  }
  *out = lg;
  c->err.clear();
  return BPMF_OK;
}

void bpmf_ligand_free(bpmf_lig_t lg) {
  if (!lg) return;
  if (lg->ctx) {
    DeviceGuard g(lg->ctx->device);
    if (lg->mem) {
      // the block returns to the context's cache once no queued work can read it
      if (cudaDeviceSynchronize() == cudaSuccess) {
        block_put(lg->ctx, lg->mem, lg->mem_bytes);
      } else {
        cudaGetLastError();
        cudaFree(lg->mem);
      }
    }
  }
  delete lg;
}

namespace {

// Shared driver of bpmf_eval and bpmf_export_energies.
bool lg_warn_cached(const bpmf_ctx *c) { return c->warn_last; }

// Receptors that share padded FFT edges share the ligand's forward transforms.
struct RecGroup {
  int P[3] = {0, 0, 0};
  int S[3] = {0, 0, 0};  // max site edges over the group
  int F2 = 0;
  long long Q = 0;
  std::vector<int> ks;   // receptor indices (call order)
};

std::vector<RecGroup> group_receptors(const bpmf_rec_t *recs, int K) {
  std::vector<RecGroup> gs;
  for (int k = 0; k < K; ++k) {
    const bpmf_rec *r = recs[k];
    size_t i = 0;
    while (i < gs.size() && !(gs[i].P[0] == r->P[0] && gs[i].P[1] == r->P[1] && gs[i].P[2] == r->P[2])) ++i;
    if (i == gs.size()) {
      RecGroup g;
      for (int d = 0; d < 3; ++d) g.P[d] = r->P[d];
      g.F2 = r->F2;
      g.Q = r->Q;
      gs.push_back(g);
    }
    gs[i].ks.push_back(k);
    for (int d = 0; d < 3; ++d) gs[i].S[d] = std::max(gs[i].S[d], r->site_n[d]);
  }
  return gs;
}

// Transform edges of each of J configurations against a receptor group:
// the crop edge that holds every receptor node the site windows of the group
// reach with the configuration's ligand box (the split-bf16 form keeps the
// full edges), and a crop is kept only where its configurations save at least
// 24 configurations' worth of spectrum volume (a crop costs one transform of
// the group's grids).
// x-axis edge of the FP32 forms: the smallest edge of the compile-time x
// pass (k_xpass) that holds P, when it is at most 5/4 of P (its transforms
// cost fewer instructions per point than the generic engine's), else P.
// Padding with zeros past the grid, like any larger edge, changes no energy
// of the site window (no kept translation wraps).
int xpass_edge(int P) {
  for (int e = P; 4 * e <= 5 * P && e <= BPMF_MAX_FFT_EDGE; ++e)
    if (xpass_supported(e)) return e;
  return P;
}

std::vector<std::array<int, 3>> transform_edges(const ConfMeta *mj, int J, const RecGroup &g, const bpmf_rec_t *recs,
                                                bool split, bool fp32_x) {
  const int Kg = (int)g.ks.size();
  std::vector<std::array<int, 3>> pc(std::max(J, 1));
  for (int i = 0; i < J; ++i) {
    for (int d = 0; d < 3; ++d) {
      int W = 0;
      for (int kg = 0; kg < Kg; ++kg) W = std::max(W, recs[g.ks[kg]]->site_n[d] + std::min(mj[i].u[d], g.P[d]) - 1);
      pc[i][d] = split ? g.P[d] : crop_edge(W, g.P[d]);
    }
    if (fp32_x) pc[i][0] = xpass_edge(pc[i][0]);
  }
  const std::array<int, 3> Pf{fp32_x ? xpass_edge(g.P[0]) : g.P[0], g.P[1], g.P[2]};
  auto vol = [](const std::array<int, 3> &p) { return (double)p[0] * p[1] * (p[2] / 2 + 1); };
  std::map<std::array<int, 3>, int> count;
  for (int i = 0; i < J; ++i) ++count[pc[i]];
  for (int i = 0; i < J; ++i)
    if (pc[i] != Pf && count[pc[i]] * (1.0 - vol(pc[i]) / vol(Pf)) < 24.0) pc[i] = Pf;
  return pc;
}

bpmf_ctx::Tune tune_for(bpmf_ctx *c, const int P[3], unsigned mode) {
  auto it = c->tune.find(std::vector<int>{P[0], P[1], P[2], (int)mode});
  return it == c->tune.end() ? bpmf_ctx::Tune{} : it->second;
}

// Host plan of one bpmf_eval call: every table of every ligand and receptor
// group lives in one pinned blob uploaded with a single copy, so the execute
// phase issues no host-synchronising call and can be captured as a graph.
// Configurations of one group that share a crop of every receptor grid of the
// group (transform edges P): contiguous processing positions [j0, j1).
struct BucketPlan {
  int P[3] = {0, 0, 0}, F2 = 0;
  long long Q = 0;
  int j0 = 0, j1 = 0;
  int B = 1;                           // configurations per batch
  size_t off_rptr = 0, off_ref = 0;    // blob: [2 Kg] spectrum pointers (hi, then lo), [Kg] RefTab
  std::vector<std::array<int, 3>> Ub;  // ligand box per batch
  cudaEvent_t join = nullptr;          // crops made for this bucket by this call are done
};

struct GroupPlan {
  size_t off_meta = 0, off_order = 0;  // blob: [J] ConfMeta and caller's index, processing order
  size_t off_info = 0;                 // blob: [J][Kg] PairInfo, processing order
  size_t off_kmap = 0, off_occ = 0;    // blob: [Kg] receptor index, [Kg] OccTab
  int occ_cap = 0;                     // occupancy runs per configuration, 0 without occupancy
  int occ_rb = 1;                      // CTAs per configuration building runs
  std::vector<BucketPlan> buckets;
};

struct LigPlan {
  int li = 0, J = 0, j_first = 0;
  size_t off_nv = 0;                   // blob: [J][K] valid counts, caller's order
  double gnorm[3] = {0, 0, 0};         // ||gamma_t||_2 of the ligand
  std::vector<GroupPlan> gp;           // per receptor group
  size_t fixed = 0, batch_bytes = 0;
};

// A kernel whose bounded wait ran out set the last flag the call copied out
// (read after the stream has synchronised).
void check_timeout(bpmf_ctx *c, int n_plan_ligs) {
  if (c->fail_host && c->fail_n > (size_t)n_plan_ligs && c->fail_host[n_plan_ligs]) {
    last_msg = "a kernel's bounded wait for its tensor copies ran out";
    throw Fail{BPMF_ERR_TIMEOUT};
  }
}

int eval_impl(bpmf_ctx *c, const bpmf_lig *lg, const bpmf_rec_t *recs, int K, double kT, unsigned mode,
              double *logZ, int64_t *n_valid, double *bpmf_out, double *dG, cudaStream_t st, int only_lig,
              int only_conf, double *export_E, double *Emin = nullptr, double *Dom = nullptr,
              std::vector<std::pair<int, int>> *fail_ligs = nullptr) {
  check_recs(recs, K, c);
  const double h = recs[0]->h;
  const bool use_ff = (mode == BPMF_MODE_FF);
  const bool split = (mode == BPMF_MODE_SPLIT_BF16 || mode == BPMF_MODE_SPLIT_REFINE);
  const bool refine = (mode == BPMF_MODE_REFINE || mode == BPMF_MODE_SPLIT_REFINE);
  const size_t E = use_ff ? sizeof(cx<ff>) : sizeof(cx<float>);
  const std::vector<RecGroup> groups = group_receptors(recs, K);
  if (split) tc_table(c);
  const int lig_begin = only_lig >= 0 ? only_lig : 0;
  const int lig_end = only_lig >= 0 ? only_lig + 1 : lg->n_lig;
  const bool host_out = !export_E && ((logZ && !is_device_ptr(logZ)) || (n_valid && !is_device_ptr(n_valid)) ||
                                      (bpmf_out && !is_device_ptr(bpmf_out)) || (dG && !is_device_ptr(dG)) ||
                                      (Emin && !is_device_ptr(Emin)) || (Dom && !is_device_ptr(Dom)));
  // graph replay: same handles, mode, kT and output buffers as the cached graph
  const bool use_graph =
      c->graph_mode && !export_E && !host_out && st != nullptr && !c->prof && only_lig < 0 && only_conf < 0 &&
      !c->wait_test;
  std::vector<unsigned long long> key;
  if (use_graph) {
    key = {lg->id, (unsigned long long)K, mode, (unsigned long long)c->ws_budget};
    for (int k = 0; k < K; ++k) key.push_back(recs[k]->id);
    unsigned long long kb;
    std::memcpy(&kb, &kT, sizeof(kb));
    key.push_back(kb);
    unsigned cs;  // the refined form's test settings enter the captured launches
    std::memcpy(&cs, &c->refine_check_scale, sizeof(cs));
    key.insert(key.end(), {(unsigned long long)cs, (unsigned long long)c->refine_list_cap});
    // device buffers the captured launches address: a call that grew them
    // since (outside graph mode) leaves the cached graph stale
    key.insert(key.end(), {(unsigned long long)(uintptr_t)c->ws, (unsigned long long)(uintptr_t)c->pmin_store});
    for (const void *q : {(const void *)logZ, (const void *)n_valid, (const void *)bpmf_out, (const void *)dG,
                          (const void *)Emin, (const void *)Dom})
      key.push_back((unsigned long long)(uintptr_t)q);
    for (const auto &g : groups) {
      const bpmf_ctx::Tune t = tune_for(c, g.P, mode);
      key.insert(key.end(), {(unsigned long long)t.batch_cap, (unsigned long long)t.axis_lw,
                             (unsigned long long)t.zfwd_l, (unsigned long long)t.xround});
    }
    if (c->gexec && key == c->gkey) {
      CK(cudaGraphLaunch(c->gexec, st));
      CK(cudaEventRecord(c->pinned_busy, st));
      if (refine) {  // the certificate flags the graph copied out
        CK(cudaStreamSynchronize(st));
        check_timeout(c, lig_end - lig_begin);
        for (int li = lig_begin; li < lig_end; ++li)
          if (c->fail_host[li - lig_begin] && fail_ligs) fail_ligs->push_back({li, c->fail_host[li - lig_begin]});
      }
      return lg_warn_cached(c) ? BPMF_WARN_NO_VALID : BPMF_OK;
    }
  }

  // ---------------------------------------------------------------- plan
  std::vector<char> blob;
  auto put = [&](const void *src, size_t bytes) {
    const size_t o = blob.size();
    blob.resize(o + align_up(bytes));
    if (bytes) std::memcpy(blob.data() + o, src, bytes);
    return o;
  };
  bool warn = false;
  std::vector<LigPlan> plans;
  std::vector<ConfMeta> meta;
  std::vector<PairInfo> info;
  std::vector<long long> nv;
  size_t ws_need = 0;
  // receptor crops made by this call: forked from this point of the stream
  cudaEvent_t fork = pool_event(c);
  CK(cudaEventRecord(fork, st));
  std::vector<cudaEvent_t> joins;
  std::vector<bpmf_rec *> touched;
  for (int li = lig_begin; li < lig_end; ++li) {
    ligand_tables(lg, li, recs, K, h, meta, info, nv);
    LigPlan pl;
    pl.li = li;
    for (int i = 0; i < lg->n_atoms[li]; ++i) {
      const int ai = lg->atom_off[li] + i;
      const double q = lg->q_host[ai], se = std::sqrt((double)lg->eps_host[ai]), R = lg->R_host[ai];
      const double gr = se * std::pow(R, lg->p_rep), ga = se * std::pow(R, lg->p_att);
      pl.gnorm[0] += q * q;
      pl.gnorm[1] += gr * gr;
      pl.gnorm[2] += ga * ga;
    }
    for (int t = 0; t < 3; ++t) pl.gnorm[t] = std::sqrt(pl.gnorm[t]);
    pl.J = lg->n_conf[li];
    if (only_conf >= 0) {
      if (only_conf >= pl.J) throw Fail{BPMF_ERR_INVALID_ARG};
      pl.j_first = only_conf;
      pl.J = 1;
    }
    const int J = pl.J;
    std::vector<long long> nv_c((size_t)std::max(J, 1) * K);
    for (int i = 0; i < J; ++i)
      for (int k = 0; k < K; ++k) {
        nv_c[(size_t)i * K + k] = nv[(size_t)(pl.j_first + i) * K + k];
        if (nv_c[(size_t)i * K + k] == 0) warn = true;
      }
    pl.off_nv = put(nv_c.data(), sizeof(long long) * J * K);
    const size_t JK = (size_t)std::max(J, 1) * K;
    size_t fixed = align_up(sizeof(long long) * JK) + align_up(sizeof(double) * JK) * 3 +
                   align_up(sizeof(double) * (2 * K + 3));
    size_t batch_bytes = 0;
    for (const auto &g : groups) {
      const int Kg = (int)g.ks.size();
      GroupPlan gpn;
      const ConfMeta *mj = meta.data() + pl.j_first;
      std::vector<std::array<int, 3>> pc = transform_edges(
          mj, J, g, recs, split, (mode == BPMF_MODE_FP32 || mode == BPMF_MODE_REFINE) && tune_for(c, g.P, mode).xround);
      const std::array<int, 3> Pf{g.P[0], g.P[1], g.P[2]};
      // processing order: by crop, then by ligand-box extent, so each batch's
      // box (the maximum over its members) stays tight; the merge scatters
      // results back to the caller's order
      std::vector<int> order(std::max(J, 1), 0);
      for (int i = 0; i < J; ++i) order[i] = i;
      std::stable_sort(order.begin(), order.begin() + J, [&](int a, int b) {
        // the uncropped bucket first: its work starts while the crops are made
        const bool fa = pc[a] == Pf, fb = pc[b] == Pf;
        if (fa != fb) return fa;
        if (pc[a] != pc[b]) return pc[a] < pc[b];
        for (int d = 0; d < 3; ++d)
          if (mj[a].u[d] != mj[b].u[d]) return mj[a].u[d] < mj[b].u[d];
        return false;
      });
      std::vector<ConfMeta> meta_s(std::max(J, 1));
      for (int i = 0; i < J; ++i) meta_s[i] = mj[order[i]];
      gpn.off_meta = put(meta_s.data(), sizeof(ConfMeta) * J);
      gpn.off_order = put(order.data(), sizeof(int) * J);
      gpn.off_kmap = put(g.ks.data(), sizeof(int) * Kg);
      std::vector<OccTab> ot(Kg);
      bool any_occ = false;
      for (int kg = 0; kg < Kg; ++kg) {
        const bpmf_rec *r = recs[g.ks[kg]];
        ot[kg] = OccTab{r->occ, r->N[0], r->N[1], r->N[2], r->occW};
        any_occ = any_occ || r->occ;
      }
      gpn.off_occ = put(ot.data(), sizeof(OccTab) * Kg);
      std::array<int, 3> Um{1, 1, 1};
      for (int i = 0; i < J; ++i)
        // each box clamped by its own bucket's edges, which may exceed the
        // padded ones (the FP32 forms' rounded x edge)
        for (int d = 0; d < 3; ++d)
          Um[d] = std::max(Um[d], std::min(meta_s[i].u[d], std::max(g.P[d], pc[order[i]][d])));
      Um[1] += Um[1] & 1;
      BatchGeom bg{};
      for (int d = 0; d < 3; ++d) bg.S[d] = g.S[d];
      bg.K = Kg;
      if (any_occ && J > 0) {
        float rmax = 0.f;
        const float hf = (float)h;
        for (int i = 0; i < lg->n_atoms[li]; ++i)
          rmax = std::max(rmax, std::fabs(lg->R_host[lg->atom_off[li] + i] / hf));
        if (g.S[2] > 256) {
          last_msg = "site boxes above 256 translations along z with an occupancy grid";
          throw Fail{BPMF_ERR_SIZE_UNSUPPORTED};
        }
        if (!(rmax <= 60.f)) {
          last_msg = "occupancy radius above 60 grid spacings";
          throw Fail{BPMF_ERR_SIZE_UNSUPPORTED};
        }
        bg.occ_cap = occ_run_cap(lg->n_atoms[li], rmax, Um[2]);
        // (a, b) rows of a configuration: about (u0 + 2 r + 4)(u1 + 2 r + 4), 256 per CTA
        const long long rows = (long long)(Um[0] + 2 * (int)std::ceil(rmax) + 4) * (Um[1] + 2 * (int)std::ceil(rmax) + 4);
        bg.occ_rb = (int)std::max<long long>(1, std::min<long long>(32, (rows + 255) / 256));
      }
      gpn.occ_cap = bg.occ_cap;
      gpn.occ_rb = bg.occ_rb;
      bg.refine = refine;
      bg.ref_cap = refine ? refine_cap(g.S, c->refine_seeded ? 0 : c->refine_list_cap) : 0;
      bg.nmax = lg->n_atoms[li];
      const size_t part = align_up(sizeof(float4) * (size_t)std::max(J, 1) * Kg * g.S[0]) +
                          (refine ? align_up(sizeof(float4) * 2 * (size_t)std::max(J, 1) * Kg) : 0);
      const bpmf_ctx::Tune tn = tune_for(c, g.P, mode);
      std::vector<PairInfo> info_g((size_t)std::max(J, 1) * Kg);
      for (int j0 = 0; j0 < J;) {
        int j1 = j0;
        while (j1 < J && pc[order[j1]] == pc[order[j0]]) ++j1;
        BucketPlan bk;
        const std::array<int, 3> Pc = pc[order[j0]];
        for (int d = 0; d < 3; ++d) bk.P[d] = Pc[d];
        bk.F2 = Pc[2] / 2 + 1;
        bk.Q = (long long)Pc[1] * bk.F2;
        bk.j0 = j0;
        bk.j1 = j1;
        std::vector<const float2 *> rp(2 * Kg);
        std::vector<RefTab> rt(Kg);
        std::vector<bpmf_rec *> rg(Kg);
        for (int kg = 0; kg < Kg; ++kg) rg[kg] = recs[g.ks[kg]];
        const size_t nj = joins.size();
        const std::vector<bpmf_rec::Crop> crs = rec_crops(c, rg, Pc, fork, joins, touched);
        if (joins.size() > nj) bk.join = joins.back();
        for (int kg = 0; kg < Kg; ++kg) {
          bpmf_rec *r = rg[kg];
          const bpmf_rec::Crop &cr = crs[kg];
          rp[kg] = cr.hi;
          rp[Kg + kg] = cr.lo;
          rt[kg] = RefTab{r->grid, cr.sumsq, r->N[0], r->N[1], r->N[2], (float)cr.vol};
          for (int i = j0; i < j1; ++i) {
            PairInfo pi = info[(size_t)(pl.j_first + order[i]) * K + g.ks[kg]];
            for (int d = 0; d < 3; ++d) pi.wc[d] = pi.w0[d] - cr.c0[d];
            info_g[(size_t)i * Kg + kg] = pi;
          }
        }
        bk.off_rptr = put(rp.data(), sizeof(void *) * 2 * Kg);
        bk.off_ref = put(rt.data(), sizeof(RefTab) * Kg);
        for (int d = 0; d < 3; ++d) twiddles(c, Pc[d]);
        BatchGeom bb = bg;
        for (int d = 0; d < 3; ++d) {
          bb.U[d] = std::min(Um[d], Pc[d]);
          bb.P[d] = Pc[d];
        }
        bb.F2 = bk.F2;
        bb.Q = bk.Q;
        const size_t per_conf = batch_bytes_per_conf(bb, E);
        int B = (int)std::max<size_t>(1, (c->ws_budget > fixed + part ? c->ws_budget - fixed - part : 0) / per_conf);
        if (tn.batch_cap > 0) B = std::min(B, tn.batch_cap);
        B = std::min(B, j1 - j0);
        bk.B = B;
        for (int b0 = j0; b0 < j1; b0 += B) {
          std::array<int, 3> U{1, 1, 1};
          for (int i = b0; i < std::min(j1, b0 + B); ++i)
            for (int d = 0; d < 3; ++d) U[d] = std::max(U[d], std::min(meta_s[i].u[d], Pc[d]));
          // z rows are transformed in (y, y+1) pairs: an even y extent keeps each
          // pair inside one plane, so results do not depend on the batching
          U[1] += U[1] & 1;
          bk.Ub.push_back(U);
        }
        batch_bytes = std::max(batch_bytes, part + per_conf * B);
        gpn.buckets.push_back(std::move(bk));
        j0 = j1;
      }
      gpn.off_info = put(info_g.data(), sizeof(PairInfo) * J * Kg);
      pl.gp.push_back(std::move(gpn));
    }
    pl.fixed = fixed;
    pl.batch_bytes = batch_bytes;
    ws_need = std::max(ws_need, fixed + batch_bytes);
    plans.push_back(std::move(pl));
  }
  const size_t blob_bytes = align_up(blob.size());
  const int n_plan_ligs = lig_end - lig_begin;
  // per ligand: the refined form's certificate flag; then one flag for a
  // bounded wait that ran out in a kernel
  const size_t fail_bytes = align_up(sizeof(int) * (n_plan_ligs + 1));
  // device resources are made ready before any work is queued (and so before
  // a capture begins): workspace, pinned staging, twiddle tables, the pinned
  // certificate flags
  char *ws = static_cast<char *>(workspace(c, blob_bytes + fail_bytes + ws_need, st));
  if (refine && (size_t)lg->total_conf * K > c->pmin_store_n) {
    if (c->pmin_store) {
      CK(cudaStreamSynchronize(st));
      CK(cudaFree(c->pmin_store));
      c->pmin_store = nullptr;
      c->pmin_store_n = 0;
    }
    CK(cudaMalloc(&c->pmin_store, sizeof(unsigned) * (size_t)lg->total_conf * K));
    c->pmin_store_n = (size_t)lg->total_conf * K;
  }
  if (c->fail_n < (size_t)n_plan_ligs + 1) {
    if (c->fail_host) {
      CK(cudaStreamSynchronize(st));
      CK(cudaFreeHost(c->fail_host));
      c->fail_host = nullptr;
      c->fail_n = 0;
    }
    CK(cudaMallocHost(&c->fail_host, sizeof(int) * (n_plan_ligs + 1)));
    c->fail_n = n_plan_ligs + 1;
  }
  // the pinned staging is rewritten: wait for the last copy or graph replay
  // that reads it, and drop the cached graph, whose copy node points at it
  if (!c->pinned_busy) CK(cudaEventCreateWithFlags(&c->pinned_busy, cudaEventDisableTiming));
  CK(cudaEventSynchronize(c->pinned_busy));
  if (c->gexec) {
    CK(cudaGraphExecDestroy(c->gexec));
    c->gexec = nullptr;
    c->gkey.clear();
  }
  if (blob_bytes > c->pinned_bytes) {
    if (c->pinned) {
      CK(cudaFreeHost(c->pinned));
      c->pinned = nullptr;
      c->pinned_bytes = 0;
    }
    CK(cudaMallocHost(&c->pinned, blob_bytes));
    c->pinned_bytes = blob_bytes;
  }
  if (!blob.empty()) std::memcpy(c->pinned, blob.data(), blob.size());
  for (const auto &g : groups)
    for (int d = 0; d < 3; ++d) twiddles(c, g.P[d]);
  // crops made earlier (perhaps on another stream) are ordered by their
  // receptor's event.  Crops made here: a graph capture waits for all of them
  // first; otherwise each bucket waits for its own before its first batch, so
  // the work of the buckets before it overlaps them.  Their receptors' events
  // complete with the last of them (recorded on a side stream that joins them).
  for (int k = 0; k < K; ++k)
    if (recs[k]->crop_ev) CK(cudaStreamWaitEvent(st, recs[k]->crop_ev, 0));
  if (use_graph)
    for (cudaEvent_t e : joins) CK(cudaStreamWaitEvent(st, e, 0));
  if (!touched.empty()) {
    cudaStream_t &sj = c->side[0];
    if (!sj) CK(cudaStreamCreateWithFlags(&sj, cudaStreamNonBlocking));
    for (cudaEvent_t e : joins) CK(cudaStreamWaitEvent(sj, e, 0));
    for (bpmf_rec *r : touched) {
      if (!r->crop_ev) CK(cudaEventCreateWithFlags(&r->crop_ev, cudaEventDisableTiming));
      CK(cudaEventRecord(r->crop_ev, sj));
    }
  }
  c->warn_last = warn;

  // -------------------------------------------------------------- execute
  if (use_graph) CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  try {
    char *tab = ws;
    // refined form: one certificate flag per ligand of the call, then the
    // per-ligand region
    int *d_fail = reinterpret_cast<int *>(ws + blob_bytes);
    char *lw = ws + blob_bytes + fail_bytes;
    if (blob_bytes) {
      CK(cudaMemcpyAsync(tab, c->pinned, blob.size(), cudaMemcpyHostToDevice, st));
      if (!use_graph) CK(cudaEventRecord(c->pinned_busy, st));
    }
    CK(cudaMemsetAsync(d_fail, 0, sizeof(int) * (n_plan_ligs + 1), st));
    long long conf_base = 0;
    for (int li = 0; li < lig_begin; ++li) conf_base += lg->n_conf[li];
    for (const LigPlan &pl : plans) {
      const int J = pl.J;
      const size_t JK = (size_t)std::max(J, 1) * K;
      char *p = lw;
      long long *d_nvout = reinterpret_cast<long long *>(p);
      p += align_up(sizeof(long long) * JK);
      double *d_logZ = reinterpret_cast<double *>(p);
      p += align_up(sizeof(double) * JK);
      double *d_logS = reinterpret_cast<double *>(p);
      p += align_up(sizeof(double) * JK);
      double *d_emin = reinterpret_cast<double *>(p);
      p += align_up(sizeof(double) * JK);
      double *d_B = reinterpret_cast<double *>(p);
      p += align_up(sizeof(double) * (2 * K + 3));  // bpmf [K], dG, dominant-state [K + 2]
      char *d_grp = p;  // partials + batch buffers, reused group by group
      const long long *d_nv = reinterpret_cast<const long long *>(tab + pl.off_nv);
      for (size_t gi = 0; gi < groups.size(); ++gi) {
        const RecGroup &g = groups[gi];
        const GroupPlan &gp = pl.gp[gi];
        const int Kg = (int)g.ks.size();
        const ConfMeta *d_meta = reinterpret_cast<const ConfMeta *>(tab + gp.off_meta);
        const PairInfo *d_info = reinterpret_cast<const PairInfo *>(tab + gp.off_info);
        const OccTab *d_tabs = reinterpret_cast<const OccTab *>(tab + gp.off_occ);
        float4 *d_part = reinterpret_cast<float4 *>(d_grp);
        char *d_batch = d_grp + align_up(sizeof(float4) * (size_t)std::max(J, 1) * Kg * g.S[0]);
        float4 *d_part_ref = nullptr;  // refined form: [J][Kg][2] corrections
        if (refine) {
          d_part_ref = reinterpret_cast<float4 *>(d_batch);
          d_batch += align_up(sizeof(float4) * 2 * (size_t)std::max(J, 1) * Kg);
        }
        const bpmf_ctx::Tune tn = tune_for(c, g.P, mode);
        for (const BucketPlan &bk : gp.buckets) {
          if (!use_graph && bk.join) CK(cudaStreamWaitEvent(st, bk.join, 0));
          const double norm = 1.0 / ((double)bk.P[0] * bk.P[1] * bk.P[2]);
          float nsh, nsl, esh, esl;
          split_ff(-norm / kT, nsh, nsl);
          split_ff(norm, esh, esl);
          const float2 *const *d_rptr = reinterpret_cast<const float2 *const *>(tab + bk.off_rptr);
          const RefTab *d_rtabs = reinterpret_cast<const RefTab *>(tab + bk.off_ref);
          for (int b0 = bk.j0, bi = 0; b0 < bk.j1; b0 += bk.B, ++bi) {
            const int nb = std::min(bk.B, bk.j1 - b0);
            BatchGeom gb{};
            for (int d = 0; d < 3; ++d) {
              gb.U[d] = bk.Ub[bi][d];
              gb.P[d] = bk.P[d];
              gb.S[d] = g.S[d];
            }
            gb.F2 = bk.F2;
            gb.Q = bk.Q;
            gb.K = Kg;
            gb.occ_cap = gp.occ_cap;
            gb.occ_rb = gp.occ_rb;
            gb.refine = refine;
            gb.ref_cap = refine ? refine_cap(g.S, c->refine_seeded ? 0 : c->refine_list_cap) : 0;
            gb.nmax = lg->n_atoms[pl.li];
            RefineCtx rf;
            if (refine) {
              rf.rtabs = d_rtabs;
              for (int t = 0; t < 3; ++t) rf.gnorm[t] = pl.gnorm[t];
              rf.kT = kT;
              rf.part_ref = d_part_ref + 2 * (size_t)b0 * Kg;
              rf.fail = d_fail + (pl.li - lig_begin);
              rf.check_scale = c->refine_check_scale;
              // the split locator's error: measured up to ~8x the FP32 form's (the
              // tensor cores' FP32 accumulation is not IEEE-rounded)
              rf.bound_scale = split ? 8.f : 1.f;
              rf.store = c->pmin_store + ((size_t)lg->conf_off[pl.li] + pl.j_first) * K;
              rf.order = reinterpret_cast<const int *>(tab + gp.off_order) + b0;
              rf.kmap = reinterpret_cast<const int *>(tab + gp.off_kmap);
              rf.Kall = K;
              rf.seeded = c->refine_seeded;
            }
            // the batch buffers end inside the workspace allocation
            const size_t avail = c->ws_bytes - (size_t)(d_batch - static_cast<char *>(c->ws));
            if (use_ff)
              run_batch<ff>(c, lg, gb, nb, d_meta + b0, d_info + (size_t)b0 * Kg, d_rptr, d_rptr + Kg, h, nsh, nsl,
                            esh, esl, d_part + (size_t)b0 * Kg * g.S[0], export_E, d_batch, avail, st, tn, false,
                            d_tabs);
            else
              run_batch<float>(c, lg, gb, nb, d_meta + b0, d_info + (size_t)b0 * Kg, d_rptr, nullptr, h, nsh, nsl,
                               esh, esl, d_part + (size_t)b0 * Kg * g.S[0], export_E, d_batch, avail, st, tn, split,
                               d_tabs,
                               refine ? &rf : nullptr,
                               reinterpret_cast<const float2 *const *>(blob.data() + bk.off_rptr),
                               d_fail + n_plan_ligs);
          }
        }
        if (export_E) continue;
        MergeArgs ma{};
        ma.part = d_part;
        ma.part_ref = d_part_ref;
        ma.nvalid = d_nv;
        ma.order = reinterpret_cast<const int *>(tab + gp.off_order);
        ma.kmap = reinterpret_cast<const int *>(tab + gp.off_kmap);
        ma.Kg = Kg;
        ma.J = J;
        ma.K = K;
        ma.S0 = g.S[0];
        ma.logS = d_logS;
        ma.logZ = d_logZ;
        ma.nvalid_out = d_nvout;
        ma.kT = kT;
        ma.emin = d_emin;
        launch(c, "k_merge", st, [&] { return launch_merge_pairs(ma, st); });
      }
      if (export_E) break;
      MergeArgs mf{};
      mf.nvalid = d_nv;
      mf.J = J;
      mf.K = K;
      mf.kT = kT;
      mf.vsite_scale = h * h * h * kStandardConc;
      mf.logS = d_logS;
      mf.logZ = d_logZ;
      mf.bpmf = d_B;
      mf.dG = d_B + K;
      mf.emin = d_emin;
      mf.dom = Dom ? d_B + K + 1 : nullptr;
      launch(c, "k_merge", st, [&] { return launch_merge(mf, st); });
      if (J > 0) {
        CK(cudaMemcpyAsync(logZ + conf_base * K, d_logZ, sizeof(double) * J * K, cudaMemcpyDefault, st));
        if (n_valid)
          CK(cudaMemcpyAsync(n_valid + conf_base * K, d_nvout, sizeof(int64_t) * J * K, cudaMemcpyDefault, st));
        if (Emin) CK(cudaMemcpyAsync(Emin + conf_base * K, d_emin, sizeof(double) * J * K, cudaMemcpyDefault, st));
      }
      if (bpmf_out)
        CK(cudaMemcpyAsync(bpmf_out + (size_t)pl.li * K, d_B, sizeof(double) * K, cudaMemcpyDefault, st));
      if (dG) CK(cudaMemcpyAsync(dG + pl.li, d_B + K, sizeof(double), cudaMemcpyDefault, st));
      if (Dom)
        CK(cudaMemcpyAsync(Dom + (size_t)pl.li * (K + 2), d_B + K + 1, sizeof(double) * (K + 2), cudaMemcpyDefault,
                           st));
      // the next ligand reuses the workspace; stream order keeps these copies first
      conf_base += lg->n_conf[pl.li];
    }
    CK(cudaMemcpyAsync(c->fail_host, d_fail, sizeof(int) * (n_plan_ligs + 1), cudaMemcpyDeviceToHost, st));
  } catch (Fail f) {
    if (use_graph) {
      cudaGraph_t gr = nullptr;
      cudaStreamEndCapture(st, &gr);
      if (gr) cudaGraphDestroy(gr);
      cudaGetLastError();
    }
    throw;
  }
  if (use_graph) {
    cudaGraph_t gr = nullptr;
    CK(cudaStreamEndCapture(st, &gr));
    const cudaError_t ie = cudaGraphInstantiate(&c->gexec, gr, 0);
    cudaGraphDestroy(gr);
    CK(ie);
    c->gkey = key;
    CK(cudaGraphLaunch(c->gexec, st));
    CK(cudaEventRecord(c->pinned_busy, st));
  }
  // the fork and join events are queued in every wait that uses them: reusable
  for (cudaEvent_t e : joins) c->event_pool.push_back(e);
  c->event_pool.push_back(fork);
  if (refine || host_out || export_E) {
    CK(cudaStreamSynchronize(st));
    check_timeout(c, n_plan_ligs);
  }
  if (refine)  // the certificate flags: the ligands to recompute in float pairs
    for (int li = lig_begin; li < lig_end; ++li)
      if (c->fail_host[li - lig_begin] && fail_ligs) fail_ligs->push_back({li, c->fail_host[li - lig_begin]});
  return warn ? BPMF_WARN_NO_VALID : BPMF_OK;
}

}  // namespace

namespace {
// eval_impl plus the refined form's fallbacks.  A ligand whose candidate list
// overflowed (and whose certificate held) is evaluated again in the refined
// form, each pair's running minimum starting from the first pass's final
// minimum; a ligand whose
// certificate failed, or whose list overflowed again, is evaluated again in
// float pairs over the same outputs, and the result carries
// BPMF_WARN_REFINE_FALLBACK.  The context's note (bpmf_last_error) counts both,
// the fallbacks by the reasons of the ligand's last refined pass (a first
// pass with a capped list may check no translation of the final window, so
// only its re-run can tell whether the certificate holds).
int eval_checked(bpmf_ctx *c, const bpmf_lig *lg, const bpmf_rec_t *recs, int K, double kT, unsigned mode,
                 double *logZ, int64_t *n_valid, double *bpmf_out, double *dG, cudaStream_t st, int only_lig,
                 int only_conf, double *export_E, double *Emin = nullptr, double *Dom = nullptr) {
  std::vector<std::pair<int, int>> fails;  // (ligand, reasons: bit 0 certificate, bit 1 list overflow)
  int rc = eval_impl(c, lg, recs, K, kT, mode, logZ, n_valid, bpmf_out, dG, st, only_lig, only_conf, export_E, Emin,
                     Dom, &fails);
  int n_cert = 0, n_over = 0, n_rerun = 0;
  for (const auto &f : fails) {
    int reasons = f.second;  // of the last refined pass of this ligand
    if (f.second == 2) {
      // only the list overflowed (the certificate held where it was checked):
      // the ligand again in the same form, every pair starting from its
      // first-pass minimum, so that the lists hold about the final window
      struct Seeded {
        bpmf_ctx *c;
        ~Seeded() { c->refine_seeded = false; }
      } guard{c};
      c->refine_seeded = true;
      std::vector<std::pair<int, int>> again;
      eval_impl(c, lg, recs, K, kT, mode, logZ, n_valid, bpmf_out, dG, st, f.first, only_conf, export_E, Emin, Dom,
                &again);
      if (again.empty()) {
        ++n_rerun;
        continue;
      }
      reasons = again.front().second;  // why the re-run failed
    }
    eval_impl(c, lg, recs, K, kT, BPMF_MODE_FF, logZ, n_valid, bpmf_out, dG, st, f.first, only_conf, export_E, Emin,
              Dom);
    n_cert += (reasons & 1) != 0;
    n_over += (reasons & 2) != 0;
  }
  c->note.clear();
  if (n_rerun)
    c->note = "refined form: " + std::to_string(n_rerun) + " ligand(s) re-run from the first pass's minima";
  if (n_cert + n_over) {
    rc |= BPMF_WARN_REFINE_FALLBACK;
    c->note += std::string(c->note.empty() ? "" : "; ") + "refined form: " + std::to_string(n_cert + n_over) +
               " ligand(s) recomputed in float pairs (certificate failed: " + std::to_string(n_cert) +
               ", candidate list overflowed: " + std::to_string(n_over) + ")";
  }
  return rc;
}

int eval_entry(bpmf_ctx_t c, bpmf_lig_t lg, const bpmf_rec_t *recs, int K, double kT, unsigned mode, double *logZ,
               int64_t *n_valid, double *bpmf_out, double *dG, double *psi_min, double *psi_dom, void *stream) {
  if (!c || !lg || !recs || K < 1 || !(kT > 0.0) || (!logZ && lg && lg->total_conf > 0))
    return set_err(c, BPMF_ERR_INVALID_ARG, "null argument, K < 1 or kT <= 0");
  if (mode != BPMF_MODE_FP32 && mode != BPMF_MODE_FF && mode != BPMF_MODE_SPLIT_BF16 && mode != BPMF_MODE_REFINE &&
      mode != BPMF_MODE_SPLIT_REFINE)
    return set_err(c, BPMF_ERR_INVALID_ARG, "unknown mode");
  if (lg->ctx != c) return set_err(c, BPMF_ERR_INVALID_ARG, "ligand batch from another context");
  DeviceGuard dg(c->device);
  try {
    last_msg.clear();
    int rc = eval_checked(c, lg, recs, K, kT, mode, logZ, n_valid, bpmf_out, dG, (cudaStream_t)stream, -1, -1,
                          nullptr, psi_min, psi_dom);
    c->err = c->note;  // empty unless a warning has a detail to report
    return rc;
  } catch (Fail f) {
    return set_err(c, f.code, last_msg.empty() ? bpmf_status_string(f.code) : last_msg);
  } catch (std::bad_alloc &) {
    return set_err(c, BPMF_ERR_OOM, "host allocation");
  }
}
}  // namespace

int bpmf_transform_edges(bpmf_ctx_t c, bpmf_lig_t lg, const bpmf_rec_t *recs, int K, unsigned mode, int *edges) {
  if (!c || !lg || !recs || K < 1 || (!edges && lg->total_conf > 0))
    return set_err(c, BPMF_ERR_INVALID_ARG, "null argument or K < 1");
  if (mode != BPMF_MODE_FP32 && mode != BPMF_MODE_FF && mode != BPMF_MODE_SPLIT_BF16 && mode != BPMF_MODE_REFINE &&
      mode != BPMF_MODE_SPLIT_REFINE)
    return set_err(c, BPMF_ERR_INVALID_ARG, "unknown mode");
  try {
    last_msg.clear();
    check_recs(recs, K, c);
    const std::vector<RecGroup> groups = group_receptors(recs, K);
    std::vector<ConfMeta> meta;
    std::vector<PairInfo> info;
    std::vector<long long> nv;
    for (int li = 0; li < lg->n_lig; ++li) {
      ligand_tables(lg, li, recs, K, recs[0]->h, meta, info, nv);
      const int J = lg->n_conf[li];
      for (const RecGroup &g : groups) {
        const std::vector<std::array<int, 3>> pc =
            transform_edges(meta.data(), J, g, recs, mode == BPMF_MODE_SPLIT_BF16 || mode == BPMF_MODE_SPLIT_REFINE,
                            (mode == BPMF_MODE_FP32 || mode == BPMF_MODE_REFINE) && tune_for(c, g.P, mode).xround);
        for (int i = 0; i < J; ++i)
          for (int k : g.ks)
            for (int d = 0; d < 3; ++d) edges[((lg->conf_off[li] + i) * K + k) * 3 + d] = pc[i][d];
      }
    }
    return BPMF_OK;
  } catch (Fail f) {
    return set_err(c, f.code, last_msg.empty() ? bpmf_status_string(f.code) : last_msg);
  } catch (std::bad_alloc &) {
    return set_err(c, BPMF_ERR_OOM, "host allocation");
  }
}

int bpmf_eval(bpmf_ctx_t c, bpmf_lig_t lg, const bpmf_rec_t *recs, int K, double kT, unsigned mode, double *logZ,
              int64_t *n_valid, double *bpmf_out, double *dG, void *stream) {
  return eval_entry(c, lg, recs, K, kT, mode, logZ, n_valid, bpmf_out, dG, nullptr, nullptr, stream);
}

int bpmf_eval_dominant(bpmf_ctx_t c, bpmf_lig_t lg, const bpmf_rec_t *recs, int K, double kT, unsigned mode,
                       double *logZ, int64_t *n_valid, double *bpmf_out, double *dG, double *psi_min,
                       double *psi_dom, void *stream) {
  if (!psi_min && !psi_dom) return set_err(c, BPMF_ERR_INVALID_ARG, "psi_min and psi_dom both null");
  return eval_entry(c, lg, recs, K, kT, mode, logZ, n_valid, bpmf_out, dG, psi_min, psi_dom, stream);
}

int bpmf_autotune(bpmf_ctx_t c, bpmf_lig_t lg, const bpmf_rec_t *recs, int K, unsigned mode, void *stream) {
  if (!c || !lg || !recs || K < 1 || lg->ctx != c) return set_err(c, BPMF_ERR_INVALID_ARG, "null argument or K < 1");
  if (mode != BPMF_MODE_FP32 && mode != BPMF_MODE_FF && mode != BPMF_MODE_SPLIT_BF16 && mode != BPMF_MODE_REFINE &&
      mode != BPMF_MODE_SPLIT_REFINE)
    return set_err(c, BPMF_ERR_INVALID_ARG, "unknown mode");
  DeviceGuard dg(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const long long JK = std::max<long long>(1, lg->total_conf) * K;
  double *d_logZ = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool prof = c->prof, graph = c->graph_mode;
  try {
    last_msg.clear();
    check_recs(recs, K, c);
    c->prof = false;
    c->graph_mode = false;
    CK(cudaMallocAsync(&d_logZ, sizeof(double) * JK, st));
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<std::vector<int>> keys;
    for (const auto &g : group_receptors(recs, K)) keys.push_back({g.P[0], g.P[1], g.P[2], (int)mode});
    auto apply = [&](const bpmf_ctx::Tune &t) {
      for (const auto &k : keys) c->tune[k] = t;
    };
    auto timeit = [&](const bpmf_ctx::Tune &t) {
      apply(t);
      eval_impl(c, lg, recs, K, 1.0, mode, d_logZ, nullptr, nullptr, nullptr, st, -1, -1, nullptr);
      CK(cudaEventRecord(e0, st));
      eval_impl(c, lg, recs, K, 1.0, mode, d_logZ, nullptr, nullptr, nullptr, st, -1, -1, nullptr);
      CK(cudaEventRecord(e1, st));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      return ms;
    };
    // coordinate descent over launch shapes that leave every result bit unchanged
    bpmf_ctx::Tune best;
    float tbest = timeit(best);
    for (int cap : {256, 128, 64, 32}) {
      bpmf_ctx::Tune t = best;
      t.batch_cap = cap;
      const float tt = timeit(t);
      if (tt < tbest) tbest = tt, best = t;
    }
    for (int lw : {8, 16}) {
      bpmf_ctx::Tune t = best;
      t.axis_lw = lw;
      const float tt = timeit(t);
      if (tt < tbest) tbest = tt, best = t;
    }
    for (int l : {8}) {
      bpmf_ctx::Tune t = best;
      t.zfwd_l = l;
      const float tt = timeit(t);
      if (tt < tbest) tbest = tt, best = t;
    }
    // the FP32 forms' x transform: rounded up to the compile-time x pass, or
    // on the padded / crop edge with the generic engine (a different radix
    // plan: results agree within rounding, not bit for bit)
    if (mode == BPMF_MODE_FP32 || mode == BPMF_MODE_REFINE) {
      bpmf_ctx::Tune t = best;
      t.xround = false;
      const float tt = timeit(t);
      if (tt < tbest) tbest = tt, best = t;
    }
    apply(best);
    CK(cudaFreeAsync(d_logZ, st));
    d_logZ = nullptr;
    CK(cudaStreamSynchronize(st));
  } catch (Fail f) {
    if (d_logZ) cudaFreeAsync(d_logZ, st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->prof = prof;
    c->graph_mode = graph;
    return set_err(c, f.code, last_msg.empty() ? bpmf_status_string(f.code) : last_msg);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->prof = prof;
  c->graph_mode = graph;
  c->err.clear();
  return BPMF_OK;
}

int bpmf_export_energies(bpmf_ctx_t c, bpmf_lig_t lg, bpmf_rec_t rec, int lig_index, int conf_index, unsigned mode,
                         double *out, void *stream) {
  if (!c || !lg || !rec || !out || lig_index < 0 || lig_index >= lg->n_lig || conf_index < 0 ||
      conf_index >= lg->n_conf[lig_index])
    return set_err(c, BPMF_ERR_INVALID_ARG, "null argument or index out of range");
  if (mode != BPMF_MODE_FP32 && mode != BPMF_MODE_FF && mode != BPMF_MODE_SPLIT_BF16 && mode != BPMF_MODE_REFINE &&
      mode != BPMF_MODE_SPLIT_REFINE)
    return set_err(c, BPMF_ERR_INVALID_ARG, "unknown mode");
  DeviceGuard dg(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  double *d_out = nullptr;
  const size_t n = (size_t)rec->site_n[0] * rec->site_n[1] * rec->site_n[2];
  try {
    last_msg.clear();
    const bool dev = is_device_ptr(out);
    if (dev) {
      d_out = out;
    } else {
      CK(cudaMallocAsync(&d_out, n * sizeof(double), st));
    }
    bpmf_rec_t recs[1] = {rec};
    eval_checked(c, lg, recs, 1, 1.0, mode, nullptr, nullptr, nullptr, nullptr, st, lig_index, conf_index, d_out);
    if (!dev) {
      CK(cudaMemcpyAsync(out, d_out, n * sizeof(double), cudaMemcpyDeviceToHost, st));
      CK(cudaFreeAsync(d_out, st));
      d_out = nullptr;
      CK(cudaStreamSynchronize(st));
    }
  } catch (Fail f) {
    if (d_out && d_out != out) cudaFreeAsync(d_out, st);
    return set_err(c, f.code, last_msg.empty() ? bpmf_status_string(f.code) : last_msg);
  }
  c->err.clear();
  return BPMF_OK;
}

int bpmf_sir_poses(bpmf_ctx_t c, bpmf_lig_t lg, int lig_index, bpmf_rec_t rec, int K, int k, double kT, unsigned mode,
                   const double *logZ, const int64_t *n_valid, const double *u1, const double *u2, int M, int *conf,
                   int *pose, void *stream) {
  if (!c || !lg || !rec || !logZ || !n_valid || !u1 || !u2 || !conf || !pose || lig_index < 0 ||
      lig_index >= lg->n_lig || K < 1 || k < 0 || k >= K || !(kT > 0.0) || M < 0)
    return set_err(c, BPMF_ERR_INVALID_ARG, "null argument or index out of range");
  if (mode != BPMF_MODE_FP32 && mode != BPMF_MODE_FF && mode != BPMF_MODE_SPLIT_BF16 && mode != BPMF_MODE_REFINE &&
      mode != BPMF_MODE_SPLIT_REFINE)
    return set_err(c, BPMF_ERR_INVALID_ARG, "unknown mode");
  if (lg->ctx != c || rec->ctx != c) return set_err(c, BPMF_ERR_INVALID_ARG, "handle from another context");
  for (const void *q : {(const void *)logZ, (const void *)n_valid, (const void *)u1, (const void *)u2,
                        (const void *)conf, (const void *)pose})
    if (!is_device_ptr(q)) return set_err(c, BPMF_ERR_INVALID_ARG, "bpmf_sir_poses takes device memory");
  const int J = lg->n_conf[lig_index];
  if (M == 0 || J == 0) {
    c->err.clear();
    return BPMF_OK;
  }
  DeviceGuard dg(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int nS = rec->site_n[0] * rec->site_n[1] * rec->site_n[2];
  double *d_cdf = nullptr, *d_E = nullptr;
  try {
    last_msg.clear();
    CK(cudaMallocAsync(&d_cdf, sizeof(double) * std::max(J, nS), st));
    CK(cudaMallocAsync(&d_E, sizeof(double) * std::max(nS, 1), st));
    CK(cudaMemsetAsync(pose, 0xff, sizeof(int) * M, st));  // -1 until a translation is drawn
    launch(c, "k_sir_configs", st, [&] {
      return launch_sir_configs(logZ, reinterpret_cast<const long long *>(n_valid), J, K, k, u1, M, d_cdf, conf, st);
    });
    std::vector<int> h_conf(M);
    CK(cudaMemcpyAsync(h_conf.data(), conf, sizeof(int) * M, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    std::vector<int> js;
    for (int v : h_conf)
      if (v >= 0) js.push_back(v);
    std::sort(js.begin(), js.end());
    js.erase(std::unique(js.begin(), js.end()), js.end());
    bpmf_rec_t recs[1] = {rec};
    for (int j : js) {
      eval_checked(c, lg, recs, 1, 1.0, mode, nullptr, nullptr, nullptr, nullptr, st, lig_index, j, d_E);
      launch(c, "k_sir_translations", st,
             [&] { return launch_sir_translations(d_E, nS, kT, u2, conf, j, M, d_cdf, pose, st); });
    }
    CK(cudaFreeAsync(d_E, st));
    d_E = nullptr;
    CK(cudaFreeAsync(d_cdf, st));
    d_cdf = nullptr;
    CK(cudaStreamSynchronize(st));
  } catch (Fail f) {
    if (d_E) cudaFreeAsync(d_E, st);
    if (d_cdf) cudaFreeAsync(d_cdf, st);
    return set_err(c, f.code, last_msg.empty() ? bpmf_status_string(f.code) : last_msg);
  } catch (std::bad_alloc &) {
    if (d_E) cudaFreeAsync(d_E, st);
    if (d_cdf) cudaFreeAsync(d_cdf, st);
    return set_err(c, BPMF_ERR_OOM, "host allocation");
  }
  c->err.clear();
  return BPMF_OK;
}

}  // extern "C"
