// Kernel argument blocks and launch wrappers shared by the C-ABI layer and
// the kernel translation units.
#pragma once
#include <cuda.h>

#include <cstdint>

#include "fft.cuh"

namespace bpmf {

// Standard-state concentration of Eq. standard_binding_fe: 1 mol/L, i.e.
// N_A molecules per litre = N_A / 1e27 molecules per A^3.
#ifndef BPMF_STANDARD_CONC_DEFINED
#define BPMF_STANDARD_CONC_DEFINED
constexpr double kStandardConc = 6.02214076e23 / 1e27;
#endif

// Per-configuration placement metadata (computed from the FP32 coordinates).
struct ConfMeta {
  float lo[3];   // minimum coordinate per axis (A)
  int u[3];      // ligand-box extent in nodes for the receptor spacing in use
  int atom_off;  // first atom of this configuration in the coordinate array
  int n_atoms;
  int gamma_off; // first atom of this ligand in the gamma arrays
  int pad;
};

// Per (configuration, receptor) site window: output s_d in [0, S_d) maps to
// translation m_d = w0_d + s_d; s_d is valid when sa_d <= s_d <= sb_d.  The
// transforms run on the receptor grid cropped at node c0 (0 when uncropped):
// translation m_d sits at index wc_d + s_d = m_d - c0_d of the correlation.
struct PairInfo {
  int w0[3];
  int sa[3];
  int sb[3];
  int wc[3];
};

struct SpreadArgs {
  const float *coords;     // [atoms][3]
  const float2 *gamma;     // [3][total_atoms] float pairs
  int gamma_stride;        // total atoms (channel stride)
  const ConfMeta *meta;    // [batch]
  float h_hi, h_lo;        // grid spacing as a float pair
  int U0, U1, U2;          // ligand-box array dims (max over the batch)
  float2 *box;             // [batch][3][U0][U1][U2] float pairs
  int chunk_rows;          // y rows accumulated per shared-memory pass (set by launch_spread)
};

struct LigSpecArgs {        // ligand y-z spectra straight from the atoms (FP32 forms)
  const float *coords;     // [atoms][3]
  const float2 *gamma;     // [3][total_atoms] float pairs (hi parts used)
  int gamma_stride;
  const ConfMeta *meta;    // [batch]
  float h_hi, h_lo;
  int U0, U1, U2;          // ligand-box array dims (max over the batch)
  int P1, P2, F2;          // transform sizes, F2 = P2 / 2 + 1
  long long Q;             // P1 * F2
  const float4 *tw1, *tw2; // exp(-2 pi i k / P) tables for P1, P2
  float2 *ly;              // [batch][3][U0][Q]
  int nmax;                // atoms per configuration (bounds the atoms on one plane)
  int chunk;               // atoms per shared-memory pass (set by launch_ligspec)
};

struct ZfwdArgs {          // real rows -> half spectra along the contiguous axis
  const float *in;         // rows of floats, or of float pairs when in_pairs
  int in_pairs;
  long long n_rows;
  int w_in;                // stored width; zero beyond
  long long in_stride;     // elements (floats or pairs) between rows
  void *out;               // cx<T> rows of F = P/2+1
  long long out_stride;    // cx<T> elements between rows
  FftPlan plan;
  const float4 *tw;
  int L;                   // complex lines per CTA (2L real rows)
};

struct AxisArgs {          // C2C along a strided axis, pruned input / output
  const void *in;
  void *out;
  int P, n_in, n_out;
  long long n_outer, inner;
  long long in_os, out_os; // cx<T> elements between consecutive outer indices
  const PairInfo *info;    // output window start info[o / w0_div].wc[axis]
  int w0_div, axis;
  int inverse;
  FftPlan plan;
  const float4 *tw;
  int LW;
  // float pairs: when set, the outputs go to these hi / lo planes (indexed
  // like out) instead of out
  float2 *out_hi, *out_lo;
};

struct XfusedArgs {        // x: forward ligand DFT, product with each receptor, inverse, window
  const void *ly;          // [batch][3][U0][Q] cx<T>
  int U0;
  const ConfMeta *meta;    // [batch] or null: rows x >= u[0] of configuration j are zero (and need not be read)
  long long Q;
  int K;
  const float2 *const *rhi;  // [K] -> [3][P0][Q]
  const float2 *const *rlo;  // [K] (ff only)
  void *x2;                // [batch][K][S0][Q] cx<T>
  int S0;
  const PairInfo *info;    // [batch][K]
  FftPlan plan;
  const float4 *tw;
  const float2 *const *rhi_h;  // host copy of rhi (tensor maps of the FP32 x pass), or null
  int *err;                // device flag set when a bounded wait of the x pass runs out, or null
  int wait_test;           // testing: the first receptor tile is not requested, so its (short) wait runs out
};

// ---- steric clashes (Eq. occupancy_grid) -----------------------------------
// Receptor occupancy as bit rows along z with one dilation per run length:
// level v holds D_v(z) = OR_{t <= v} occ(z + t) (runs of v + 1 nodes), bit
// (z + kOccZPad) of the row, for z outside [0, N2) occ = 0.  Layout
// [v][X + kOccXYPad][w][Y + kOccXYPad] (u32 words w, Y fastest), with
// kOccXYPad zero rows on both sides of x and y.
constexpr int kOccLevels = 32;
constexpr int kOccZPad = 64;
constexpr int kOccXYPad = 16;

struct OccTab {            // one receptor's tables (tab null: no occupancy grid)
  const uint32_t *tab;
  int N0, N1, N2, W;       // grid edges and words per row (padded rows: N + 2 kOccXYPad)
};

// One run of occupied ligand nodes along z in the ligand-box frame: nodes
// (a, b, c0 .. c0 + lv), read as the single level-lv window at c0.
struct OccRun {
  short a, b, c0;
  unsigned char dc, lv;    // dc unused (0)
};

struct OccRunsArgs {
  const float *coords;     // [atoms][3]
  const float *R;          // [total_atoms] LJ size parameter (occupancy radius 2^(-1/6) R)
  const ConfMeta *meta;    // [batch]
  float h;
  int cap;                 // runs per configuration
  OccRun *runs;            // [batch][2][cap]: as found, then sorted by length (longest first)
  int *n_runs;             // [batch]
  int rb;                  // CTAs per configuration
};

struct ClashArgs {
  const OccRun *runs;      // [batch][2][cap] (k_occ_runs)
  const int *n_runs;       // [batch]
  int cap;
  const OccTab *tabs;      // [K]
  const PairInfo *info;    // [batch][K]
  int K, S0, S1, S2, CW;   // CW = 32-bit words per (s0, s1) row of flags
  int T0, T1;              // translations (s0, s1) per CTA (set by launch_clash)
  uint32_t *clash;         // [batch][K][S0][S1][CW], bit s2: translation clashes
};

// ---- refined form (refine.cu) -----------------------------------------------
struct RefTab {            // one receptor's grids, FP32 [3][N0][N1][N2]
  const float *grid;
  const float *sumsq;      // [3] sum of squares of each grid over the transformed (cropped) nodes
  int N0, N1, N2;
  float vol;               // transformed nodes per channel (FP32 error bound: rms = sqrt(sumsq / vol))
};

// A translation kept for the exact re-evaluation: window index
// t = (s0 S1 + s1) S2 + s2 and its FP32 energy e.
struct Cand {
  unsigned t;
  float e;
};

// Running per-pair state of one batch of the refined form.  k_refine_init
// resets it; every k_zinv CTA lowers the pair's running FP32 minimum and
// appends the translations of its plane that lie within the window of that
// running minimum (a superset of those within the window of the final
// minimum), and leaves them out of its LSE partial; k_refine reads the final
// minimum and the lists and writes each pair's partial over its list.
struct RefineState {
  const float *win;        // [K] W + 2B per receptor (kcal/mol)
  const float *bnd;        // [K] B per receptor times the check scale (certificate threshold)
  unsigned *pmin;          // [batch][K] running minimum energy, order-preserving unsigned encoding
  int *cnt;                // [batch][K] translations appended (may exceed cap: overflow)
  Cand *cand;              // [batch][K][cap]
  float2 *exact;           // [batch][K][cap] k_refine: exact -E/kT (float pair) of the refined entries
  unsigned long long *lvl; // [batch][K] largest exact -E/kT, as an ordered key of its float pair
  unsigned long long *wsum;  // [batch][K] fixed-point sum of the weights relative to lvl
  unsigned *done;          // [batch][K] CTAs of k_refine_sum finished
  int cap;
  int *fail;               // set to 1 when a list overflows or a certificate check fails
};

// Order-preserving encoding of a float as an unsigned (larger float, larger
// code), so that atomicMin on the code keeps the minimum float.
__device__ __forceinline__ unsigned f2ord(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
constexpr int kRefineMaxList = 1 << 23;  // translations per pair list (fixed-point sum range)

struct RefineArgs {
  RefineState rs;
  float *win, *bnd;        // writable views of rs.win / rs.bnd (k_refine_init)
  const ConfMeta *meta;    // [batch]
  const PairInfo *info;    // [batch][K]
  const RefTab *tabs;      // [K]
  float gnorm[3];          // ||gamma_t||_2 of the ligand (FP32 error bound)
  float log2P3;            // log2(P0 P1 P2) of the transforms
  float check_scale;       // multiplies B in the certificate check (1 in normal use)
  float bound_scale;       // multiplies B in both the window and the check (the locator's error scale)
  const float *coords;     // [atoms][3]
  const float2 *gamma;     // [3][gamma_stride] generalised charges as float pairs
  int gamma_stride;
  float h_hi, h_lo;        // grid spacing as a float pair
  float kT;                // kcal/mol
  float nikT_hi, nikT_lo;  // -1 / kT as a float pair
  int K, S0, S1, S2;
  float4 *part_ref;        // [batch][K][2] per pair: {level M hi, lo, sum of weights hi, lo} over the
                           // re-evaluated translations, then {max exact -E/kT hi, lo, 0, 0}
  double *export_E;        // optional, batch entry 0, receptor 0: [S0][S1][S2] (exact where refined)
  // each pair's final running minimum, kept per (configuration, receptor) of
  // the ligand so that a second pass can start from it: store[order[j] Kall +
  // kmap[k]] (k_refine writes it; k_refine_init reads it when seeded)
  unsigned *store;
  const int *order;        // [batch] processing position -> the ligand's configuration index
  const int *kmap;         // [K] group-local receptor -> receptor index of the call
  int Kall;
  int seeded;
};

struct ZinvArgs {          // z: C2R + scale + mask + max-shifted log-sum-exp partials
  const void *y2;          // [batch][K][S0][S1][F2] cx<T>
  int K, S0, S1, S2, F2;
  const PairInfo *info;    // [batch][K]
  float nscale_hi, nscale_lo;   // -1 / (kT P0 P1 P2)
  float escale_hi, escale_lo;   // 1 / (P0 P1 P2) (energy export)
  float4 *part;            // [batch][K][S0] {M_hi, M_lo, s, 0}
  double *export_E;        // optional [S0][S1][S2] energies (+inf masked), batch entry 0, receptor 0
  const uint32_t *clash;   // optional [batch][K][S0][S1][CW] clash flags (excluded, +inf when exported)
  int CW;
  int Lc;                  // row pairs per shared-memory chunk (set by launch_zinv)
  RefineState rs;          // refined form (FP32 only): candidate lists; rs.cand null otherwise
  FftPlan plan;
  const float4 *tw;
  // FP32 forms: the y inverse fused in front (y2 unused) when x2 is set: each
  // CTA transforms its plane x2[(j K + k) S0 + s0] ([P1][F2], Qx = P1 F2)
  // along y, keeps the site window rows in shared memory and goes on with z
  const void *x2;
  long long Qx;
  FftPlan yplan;
  const float4 *tw1;
};

struct MergeArgs {
  const float4 *part;      // [J][Kg][S0] of one receptor group, processing order
  const float4 *part_ref;  // [J][Kg][2] refined form: each pair's re-evaluated weight (RefineArgs::part_ref), or null
  const long long *nvalid; // [J][K], caller's order, all receptors
  const int *order;        // [J] processing position -> caller's configuration index (null: identity)
  const int *kmap;         // [Kg] group-local receptor -> receptor index in the call (null: identity)
  int Kg;                  // receptors in the group (k_merge_pairs)
  double *logS;            // [J][K] scratch, caller's order
  int J, K, S0;
  double kT;
  double vsite_scale;      // h^3 * C_standard
  double *logZ;            // [J][K], caller's order
  double *bpmf;            // [K]
  double *dG;              // [1]
  long long *nvalid_out;   // [J][K], caller's order (may be null)
  double *emin;            // [J][K], caller's order: minimum energy over valid translations (may be null)
  double *dom;             // [K + 2] (k_merge, with emin): min over configurations per receptor, the min over
                           // receptors, and -kT ln mean_k exp(-min_k / kT) (may be null)
};

int sm_count();                      // streaming multiprocessors of the current device (kernels.cu)

// ---- host plan helpers (bpmf_api.cu), shared by every entry point ----------
int smooth_edge(int n);              // smallest even 2^a 3^b 5^c 7^d >= n (<= BPMF_MAX_FFT_EDGE), else 0
FftPlan make_plan(int P);            // radix stages 8, 4, 2, then 3, 5, 7
void twiddle_values(int P, float4 *out);  // exp(-2 pi i k / P), k < P, as float pairs
int box_extent(float lo, float hi, float hf);  // ligand-box edge in nodes (single precision rule)
// site window of a (configuration, receptor) pair along one axis; returns its valid count
long long site_window(int N, int site_lo, int site_n, int u, int &w0, int &sa, int &sb);

// ---- launch wrappers (kernels.cu, ligspec.cu, occupancy.cu, refine.cu) ---------
cudaError_t launch_refine_init(const RefineArgs &a, int batch, cudaStream_t st);  // before k_zinv
cudaError_t launch_refine(const RefineArgs &a, int batch, cudaStream_t st);       // after k_zinv (two kernels)
// sums of squares of the three grids [3][N0][N1][N2] into sumsq[3]
// (deterministic; scratch: kSumsqScratch float2 of device memory), copying
// the grids to out when it is not null
constexpr int kSumsqScratch = 3 * 256;
cudaError_t launch_sumsq(const float *g, const int N[3], float *out, float *sumsq, float2 *scratch, cudaStream_t st);
cudaError_t launch_crop(const float *grid, const int N[3], const int c0[3], const int e[3], const int E[3],
                        float *out, float *sumsq, float2 *scratch, cudaStream_t st);
cudaError_t launch_occ_table(const unsigned char *occ, int N0, int N1, int N2, int W, uint32_t *tab,
                             cudaStream_t st);
cudaError_t launch_occ_runs(const OccRunsArgs &a, int batch, cudaStream_t st);
cudaError_t launch_clash(ClashArgs a, int batch, cudaStream_t st);
cudaError_t launch_spread(const SpreadArgs &a, int batch, cudaStream_t st);
cudaError_t launch_ligspec(const LigSpecArgs &a, int batch, cudaStream_t st);
template <class T> cudaError_t launch_zfwd(const ZfwdArgs &a, cudaStream_t st);
template <class T> cudaError_t launch_axis(const AxisArgs &a, cudaStream_t st);
template <class T> cudaError_t launch_xfused(const XfusedArgs &a, int batch, cudaStream_t st);
// FP32 x pass on compile-time edges (xpass.cu): P in {64, 72, 80, 96}, no tensor-core stage.
// Receptor tiles arrive by TMA for up to kXpMaxMaps receptors per launch.
constexpr int kXpMaxMaps = 8;
struct alignas(64) XpassMaps {
  CUtensorMap m[kXpMaxMaps];
  // the ligand's y-z spectra [batch][3][U0][Q] float2 as FP32 with the
  // dimensions (2Q, batch, 3, U0): a box of 8 columns x 2 configurations x 3
  // channels x U0 rows lands in the x pass's forward buffer in its own row
  // layout [row][channel][configuration][column]; lig_ok = 0 when not encoded
  CUtensorMap lig;
  int lig_ok;
};
bool xpass_supported(int P);
// FP32 y + z inverse on compile-time edges P1 = P2 in {64, 72, 80, 96} (yzinv.cu)
bool yzinv_supported(int P1, int P2, int S1, int S2, bool clash, bool export_E);
cudaError_t launch_yzinv(const ZinvArgs &a, int batch, cudaStream_t st);
cudaError_t launch_xpass(const XfusedArgs &a, int batch, cudaStream_t st);
template <class T> cudaError_t launch_zinv(const ZinvArgs &a, int batch, cudaStream_t st);
// whether the FP32 z inverse can take the y inverse in front (whole site
// window in one shared-memory chunk at 3 CTAs per SM)
bool zinv_fused_fits(int P1, int P2, int S1, int S2, bool refine);
cudaError_t launch_merge_pairs(const MergeArgs &a, cudaStream_t st);  // per receptor group
cudaError_t launch_merge(const MergeArgs &a, cudaStream_t st);        // B_k and dG over all receptors
cudaError_t launch_split_ff(const void *spec, float2 *hi, float2 *lo, long long n, cudaStream_t st);
cudaError_t launch_gamma(const float *q, const float *eps, const float *R, int n, int p_rep, int p_att, float2 *gamma,
                         cudaStream_t st);
cudaError_t launch_minmax(const float *coords, const int *conf_atom_off, const int *conf_natoms, int n_conf,
                          float *out_minmax, cudaStream_t st);

}  // namespace bpmf
