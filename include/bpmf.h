/*
 * bpmf.h -- C ABI of the GB300 FFT-correlation BPMF library (libbpmf.so).
 *
 * Method: Nguyen, Zhou & Minh, "Using the Fast Fourier Transform in Binding
 * Free Energy Calculations" (FFTdG).  For every rigid ligand configuration and
 * every rigid receptor conformation, the receptor-ligand interaction energy of
 * every grid translation is the cross-correlation of the receptor potential
 * grids with the ligand's spread generalised charges (Eqs. general_form,
 * receptor_grid, correlation_func), evaluated with FFTs (Eq.
 * fft_correlation_func); the energies of the valid translations are reduced
 * by exponential averaging to the binding potential of mean force (Eq.
 * sample_mean_BPMF) and the BPMFs of the receptor conformations to the
 * standard binding free energy (Eqs. standard_binding_fe, binding_FE_estimate).
 *
 * Conventions shared by every call
 *  - Status: every int-returning call returns BPMF_OK (0), a negative
 *    BPMF_ERR_* code, or a positive value: the OR of the warning bits
 *    BPMF_WARN_*.  No C++ exception crosses the ABI.  bpmf_last_error() gives
 *    a one-line reason.
 *  - Pointers: array arguments may be host memory or device memory of the
 *    context's GPU (detected per pointer with cudaPointerGetAttributes), except
 *    the small per-ligand count arrays, which must be host memory.  Inputs are
 *    borrowed for the duration of the call only; outputs belong to the caller.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Work
 *    is stream ordered.  When every output is device memory the call returns
 *    without waiting for the GPU; when any output is host memory the call
 *    synchronises the stream before returning.
 *  - Handles (bpmf_ctx_t, bpmf_rec_t, bpmf_lig_t) are library-owned until
 *    their *_free / bpmf_destroy call.  A context is not thread safe.
 *  - Units: lengths in Angstrom, energies in kcal/mol, charges in e.
 */
#ifndef BPMF_H
#define BPMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BPMF_OK 0
#define BPMF_ERR_INVALID_ARG (-1)
#define BPMF_ERR_OOM (-2)
#define BPMF_ERR_CUDA (-3)
/* A kernel's bounded wait (for its tensor-memory copies or tensor-core
 * operations) ran out: it set a flag, waited once more (bounded) for what it
 * had in flight and returned, so the context stays usable.  Reported by the
 * calls that synchronise the stream (the refined forms, host outputs,
 * exports). */
#define BPMF_ERR_TIMEOUT (-4)
#define BPMF_ERR_SIZE_UNSUPPORTED (-5)
/* warning: at least one (configuration, receptor) pair has no valid
 * translation; its log Z is -inf (and a BPMF with no valid pose is +inf). */
#define BPMF_WARN_NO_VALID 1
/* warning (BPMF_MODE_REFINE): for at least one ligand the certificate check
 * failed (an FP32 energy further than B from its exact value) or a candidate
 * list overflowed again in a second pass from the first pass's minima; that
 * ligand's results were recomputed in float pairs (BPMF_MODE_FF) and are
 * exact to the float-pair form's precision. */
#define BPMF_WARN_REFINE_FALLBACK 2

/* Arithmetic of the correlation (forward transforms, spectral product,
 * inverse transforms).  Spreading is FP32 in both; the merge is FP64.
 *   BPMF_MODE_FP32 -- plain single precision.
 *   BPMF_MODE_FF   -- compensated float pairs (hi + lo, ~44-48 bits) built
 *                     from FP32 instructions; the form that meets a 1e-3
 *                     kcal/mol energy tolerance on grids whose repulsive
 *                     values reach 1e4. */
#define BPMF_MODE_FP32 0u
#define BPMF_MODE_FF 1u
/*   BPMF_MODE_SPLIT_BF16 -- the FP32 form with every radix-32 stage (padded
 *                     edges divisible by 32) run as a dense tensor-core
 *                     contraction: the 64 x 64 real DFT-32 matrix times the
 *                     twiddled data, each split into three bf16 parts
 *                     (hi, mid, lo), the six products of order up to 2^-16
 *                     accumulated by the tensor cores (FP32 without IEEE
 *                     rounding): errors up to several times the FP32 form's,
 *                     reported against the oracle per result.
 *                     Other edges fall back to the FP32 stages. */
#define BPMF_MODE_SPLIT_BF16 2u
/*   BPMF_MODE_REFINE -- the FP32 correlation for every translation, then an
 *     exact re-evaluation, in float-pair arithmetic (FP32 instructions,
 *     about 2^-44 relative), of the translations that can matter.  The FP32
 *     correlation error is expected below B = 8 eps32 sqrt(log2 P0 P1 P2)
 *     sum_t rms(G_t) ||gamma_t||_2 (the typical roundoff growth of an FFT
 *     correlation).  Every translation whose FP32 energy lies within W + 2B
 *     of the configuration's FP32 minimum (W = kT max(20, ln(1e5 n)), n the
 *     site-window size) is re-evaluated as the direct sum the correlation
 *     equals: sum_i sum_t gamma_t,i trilinear(G_t, g_i + m).  While the bound
 *     holds, every translation within W of the true minimum is among them;
 *     the others together weigh less than 1e-5 of S (6e-6 kcal/mol on
 *     kT log Z) and are left out.  The bound is checked as a certificate on
 *     every re-evaluated translation (|E_fp32 - E_exact| <= B).  A candidate
 *     list that
 *     overflows (flat landscapes: small ligands in wide sites) makes the call
 *     evaluate that ligand again in this form, each pair's running minimum
 *     starting at the first pass's; a failed check, or a second overflow,
 *     makes it recompute the ligand in float pairs and return
 *     BPMF_WARN_REFINE_FALLBACK (bpmf_last_error counts both).  In this form
 *     bpmf_eval synchronises `stream` before returning (it reads the
 *     certificate flags).  The energies that can carry weight are exact, and
 *     so are log Z, BPMF and dG up to that 1e-5, at about the FP32 form's
 *     cost; results are the same on every run.  Exported energies
 *     outside the window are the FP32 values.  The energy volume never
 *     reaches device memory: each site plane appends only its candidates to a
 *     per-pair list.  The receptor handle keeps a device copy of its FP32
 *     grids for this form. */
#define BPMF_MODE_REFINE 3u
/*   BPMF_MODE_SPLIT_REFINE -- the refined form with the split-bf16
 *     tensor-core correlation (BPMF_MODE_SPLIT_BF16) as its locator: the
 *     same window, certificate and float-pair fallback, with the bound B taken
 *     eight times as wide (the six-term split carries FP32's significand, but
 *     the tensor cores accumulate without IEEE rounding: measured errors reach
 *     several times the FP32 form's).  Runs on the full padded edges (the
 *     tensor-core stage needs edges divisible by 32). */
#define BPMF_MODE_SPLIT_REFINE 4u

/* Largest supported ligand (atoms) and padded FFT edge. */
#define BPMF_MAX_ATOMS 256
#define BPMF_MAX_FFT_EDGE 256

typedef struct bpmf_ctx *bpmf_ctx_t;
typedef struct bpmf_rec *bpmf_rec_t;
typedef struct bpmf_lig *bpmf_lig_t;

/* Create a context bound to CUDA device `device`.  Errors: INVALID_ARG (no
 * such device), CUDA.  bpmf_destroy releases the context's device memory,
 * including the blocks that freed receptors and ligand batches left in its
 * cache (see bpmf_receptor_free); free every handle of the context first. */
int bpmf_create(int device, bpmf_ctx_t *out);
void bpmf_destroy(bpmf_ctx_t ctx);

/* One-line description of a status code (static storage). */
const char *bpmf_status_string(int status);
/* Reason for the last failing call on this context ("" if none); after a
 * bpmf_eval that returned BPMF_WARN_REFINE_FALLBACK, how many ligands were
 * recomputed and why (certificate failed, candidate list overflowed), by
 * the reasons of each ligand's last refined pass (its re-run, when the first
 * pass only overflowed). */
const char *bpmf_last_error(bpmf_ctx_t ctx);

/*
 * bpmf_receptor_load -- take one rigid receptor conformation's potential
 * grids (Eq. receptor_grid: one grid per term of Eq. general_form) and compute
 * and cache their forward 3D real-to-complex spectra FT(G_R) (Eq.
 * fft_correlation_func) on the GPU, in float-pair precision.
 *
 *  grids    [3][nx][ny][nz] float32, C order, terms in the order
 *           electrostatic, LJ-repulsive, LJ-attractive (the -2 of the
 *           attractive term and the Coulomb factor included).  Node (i,j,k)
 *           sits at origin + (i,j,k) h.  Host or device.  Host grids are
 *           copied on a stream of the context's own (so the copy overlaps
 *           the work already queued on `stream`, which waits for it) and
 *           the call returns once that copy is done, not the transforms.
 *  h        grid spacing (> 0).
 *  origin   [3] position of node (0,0,0) (informational; energies depend on
 *           grid indices only).
 *  site_lo, site_n
 *           the site box in nodes: a translation m is sampled when the
 *           ligand-box centre c = floor(u/2) lands at m + c in
 *           [site_lo, site_lo + site_n) (Methodology, FFT-based BPMF
 *           Estimation; translations whose ligand box leaves the grid are
 *           discarded).  site_n >= 1 per axis.
 *  out      receives the handle.  The spectra are zero padded to the
 *           smallest 2^a 3^b 5^c 7^d edge >= n (exact for every kept
 *           translation, which never wraps).
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED (padded edge > BPMF_MAX_FFT_EDGE),
 * OOM, CUDA.
 */
int bpmf_receptor_load(bpmf_ctx_t ctx, const float *grids, int nx, int ny, int nz, double h,
                       const double origin[3], const int site_lo[3], const int site_n[3], void *stream,
                       bpmf_rec_t *out);
/* Frees a receptor.  It synchronises the device (as cudaFree does) and
 * keeps the receptor's device blocks (its spectra, and the spectra of its
 * site crops made by bpmf_eval) in the context's cache, up to 2 GiB, for the
 * next receptor or crop of the same size; the rest is freed. */
void bpmf_receptor_free(bpmf_rec_t rec);

/*
 * bpmf_receptor_set_occupancy -- attach the receptor occupancy grid of the
 * steric-clash treatment (Eq. occupancy_grid; methodology, "FFT-based BPMF
 * Estimation": receptor grids built with V(r) = 0 inside 2^(-1/6) sigma, clashes
 * detected by correlating the receptor and ligand occupancy grids).
 *   occ  [nx][ny][nz] uint8 (0 = free, nonzero = occupied), the receptor's
 *        own grid dimensions; host or device; NULL detaches the grid.
 * With a grid attached, every evaluation against this receptor treats a
 * valid translation as clashing when some occupied ligand node lands on an
 * occupied receptor node (nodes outside the grid are free); a clashing pose
 * keeps its place in the sample (it counts in n_valid) with infinite energy:
 * it adds nothing to S, is +inf in bpmf_export_energies and is never drawn
 * by bpmf_sir_poses.  The ligand occupancy grid marks node n when
 * |p_i - n|^2 < 2^(-1/3) (R_i / h)^2 for some atom i, with p_i the atom's
 * position in grid units after placement and R the size parameter given to
 * bpmf_ligand_batch, each step rounded to IEEE single precision in the order
 * p = (x - min x) / h + 2, r = R / h, threshold = (r r) 2^(-1/3),
 * distance = ((dx dx + dy dy) + dz dz).  The library copies the grid into
 * bit tables (32 run-length dilations with 16 zero rows on each side of x
 * and y: about 32 (nx + 32)(ny + 32)(nz + 128) / 8 bytes of device memory).
 * Synchronises `stream`.  Errors: INVALID_ARG, OOM, CUDA; bpmf_eval returns
 * SIZE_UNSUPPORTED when an occupancy radius exceeds 60 grid spacings.
 */
int bpmf_receptor_set_occupancy(bpmf_ctx_t ctx, bpmf_rec_t rec, const uint8_t *occ, void *stream);

/*
 * bpmf_ligand_batch -- upload a batch of ligands and their rigid
 * configurations (the randomly rotated apo-ensemble snapshots of Methodology,
 * Ligand Sampling) and compute the generalised charges of Eq. general_form:
 * gamma = (q, sqrt(eps) R^p_rep, sqrt(eps) R^p_att) per atom.
 *
 *  n_lig            number of ligands (>= 1).
 *  n_atoms, n_conf  [n_lig] HOST arrays: atoms per ligand (1..BPMF_MAX_ATOMS)
 *                   and configurations per ligand (>= 0).
 *  coords           float32 concatenated [lig][conf][atom][3] (A), already
 *                   rotated; host or device.
 *  q, eps, R        float32 concatenated [lig][atom]; host or device.
 *  p_rep, p_att     integer exponents of R in the repulsive / attractive
 *                   factors (12 and 6 for the R-form of the synthetic
 *                   recipe; 6 and 3 give the paper's sigma form), 0..32.
 * The call synchronises `stream` once (it reads back each configuration's
 * coordinate bounds, which fix the ligand-box sizes).
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED (too many atoms), OOM, CUDA.
 */
int bpmf_ligand_batch(bpmf_ctx_t ctx, int n_lig, const int *n_atoms, const int *n_conf, const float *coords,
                      const float *q, const float *eps, const float *R, int p_rep, int p_att, void *stream,
                      bpmf_lig_t *out);
/* Frees a ligand batch; synchronises the device and keeps its device block in
 * the context's cache, as bpmf_receptor_free. */
void bpmf_ligand_free(bpmf_lig_t lig);

/*
 * bpmf_eval -- the hot path.  For every ligand, configuration j and receptor
 * k: spread the ligand (trilinear weights x gamma), forward 3D FFT, spectral
 * conj-multiply-sum over the three terms against the cached receptor spectra,
 * inverse FFT restricted to the site box, translation mask, and a
 * max-shifted log-sum-exp, then an FP64 merge:
 *    log S_jk = ln sum_{m valid} exp(-E_jk(m) / kT)
 *    logZ_jk  = log S_jk - ln n_jk                (mean over translations)
 *    B_k      = -kT [ ln sum_j S_jk - ln sum_j n_jk ]   (Eq. sample_mean_BPMF
 *                                                      over all valid poses)
 *    dG       = -kT ln[(1/K) sum_k exp(-B_k/kT)] - kT ln(V_site C)
 * with C = N_A / 1e27 = 6.02214076e-4 A^-3 (1 M) and V_site = h^3 * mean_jk n_jk (Eqs.
 * standard_binding_fe and binding_FE_estimate with uniform receptor weights).
 *
 *  recs, K   receptor handles; all must share the grid spacing (else
 *            SIZE_UNSUPPORTED).  Receptors with different grid sizes are
 *            processed in groups of equal padded FFT edges; the ligand's
 *            forward transforms are shared within a group.
 * Cropped transforms: a configuration's energies over the site window read
 * only the receptor nodes within site_n + u - 1 of the site (u its ligand-box
 * edge).  Where that reach fits a smaller smooth edge (about 5/6 of the
 * padded edge) on an axis, and enough configurations share the crop to pay
 * for its transform, the configuration runs on the receptor grids cropped to
 * that edge around the site: the same energies, up to rounding, from smaller
 * transforms.  A receptor's crop spectra are made on first use (on library
 * streams forked from and joined back into `stream`) and kept until
 * bpmf_receptor_free.  The split-BF16 form always uses the full edges.
 *  kT        > 0 (kcal/mol).
 *  mode      BPMF_MODE_FP32, BPMF_MODE_FF, BPMF_MODE_SPLIT_BF16, BPMF_MODE_REFINE or
 *            BPMF_MODE_SPLIT_REFINE.
 *  logZ      [total_conf][K] float64, total_conf = sum n_conf, ligand-major.
 *  n_valid   [total_conf][K] int64 (may be NULL).
 *  bpmf      [n_lig][K] float64 (may be NULL).
 *  dG        [n_lig] float64 (may be NULL).
 * Returns BPMF_WARN_NO_VALID when some n_jk = 0 (results still written).
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED, OOM, CUDA.
 */
int bpmf_eval(bpmf_ctx_t ctx, bpmf_lig_t lig, const bpmf_rec_t *recs, int K, double kT, unsigned mode, double *logZ,
              int64_t *n_valid, double *bpmf, double *dG, void *stream);

/*
 * bpmf_eval_dominant -- bpmf_eval plus the dominant-state quantities
 * (Section "Dominant state approximation": the minimum interaction energy used
 * in place of the exponential average, per receptor snapshot, then combined
 * over snapshots by the minimum or by an exponential average).  They come out
 * of the same pass: the minimum is the maximum -E/kT that the inverse pass
 * already keeps for its shifted log-sum-exp.
 *   psi_min  [total_conf][K] float64 (may be null): min over the valid
 *            translations of E (kcal/mol) for each (configuration, receptor);
 *            +inf where n_jk = 0.
 *   psi_dom  [n_lig][K + 2] float64 (may be null): per ligand, entries 0..K-1
 *            are min_j psi_min[j][k]; entry K the minimum over receptors;
 *            entry K + 1 is -kT ln( (1/K) sum_k exp(-psi_dom[k] / kT) ).
 * At least one of psi_min, psi_dom must be non-null; host or device memory.
 * The other arguments, results and errors are those of bpmf_eval.
 */
int bpmf_eval_dominant(bpmf_ctx_t ctx, bpmf_lig_t lig, const bpmf_rec_t *recs, int K, double kT, unsigned mode,
                       double *logZ, int64_t *n_valid, double *bpmf, double *dG, double *psi_min, double *psi_dom,
                       void *stream);

/*
 * bpmf_export_energies -- debug export of one configuration's interaction
 * energies E(m) over receptor `rec`'s site window, computed by the same
 * kernels as bpmf_eval.  out: [S0][S1][S2] float64 (S = the receptor's
 * site_n), entry s is translation m = site_lo + s - floor(u/2); +inf where
 * the translation is discarded.  Host or device.
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED, OOM, CUDA.
 */
int bpmf_export_energies(bpmf_ctx_t ctx, bpmf_lig_t lig, bpmf_rec_t rec, int lig_index, int conf_index,
                         unsigned mode, double *out, void *stream);

/* Padded FFT edge the library uses for a grid edge n (0 if unsupported). */
int bpmf_fft_edge(int n);

/*
 * bpmf_crop_window -- the cropped transform (see bpmf_eval) along one axis of
 * a receptor grid of n nodes with site box [site_lo, site_lo + site_n), for a
 * configuration whose ligand box has edge u nodes.  Host only; no device work.
 *  edge  receives the transform edge: bpmf_fft_edge(n), or the smooth edge
 *        near 5/6 of it when site_n + min(u, bpmf_fft_edge(n)) - 1 nodes fit
 *        in it.  (bpmf_eval may still use the full edge for the crop when too
 *        few configurations share it.)
 *  c0    receives the crop's first receptor node: 0 for the full edge, else
 *        floor((site_n - edge) / 2) nodes from site_lo, moved into [0, n - edge].
 * Every receptor node that a kept translation of the site window reads lies
 * in [c0, c0 + edge).
 * Errors: INVALID_ARG (null output, n < 2, site_n < 1 or u < 1),
 * SIZE_UNSUPPORTED (bpmf_fft_edge(n) == 0).
 */
int bpmf_crop_window(int n, int site_lo, int site_n, int u, int *edge, int *c0);

/* bpmf_transform_edges -- the transform edges (P0, P1, P2) on which
 * bpmf_eval runs each configuration against each receptor in `mode`: the
 * receptor's padded edges, or the edges of the site crop it is given (the
 * per-axis rule of bpmf_crop_window, kept only where the crop's
 * configurations save at least 24 configurations' worth of spectrum volume).
 * Host only; no device work.  edges: HOST int [total_conf][K][3].
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED (receptors of different spacings). */
int bpmf_transform_edges(bpmf_ctx_t ctx, bpmf_lig_t lig, const bpmf_rec_t *recs, int K, unsigned mode, int *edges);

/* bpmf_set_refine_check_scale -- multiply B in the refined form's
 * certificate check (not in its window) by `scale` (default 1).  A scale
 * below the observed error ratio makes the check fail, which exercises the
 * float-pair fallback; it exists for testing.  Errors: INVALID_ARG
 * (scale < 0). */
int bpmf_set_refine_check_scale(bpmf_ctx_t ctx, double scale);

/* bpmf_set_refine_list_cap -- candidate-list capacity per (configuration,
 * receptor) pair in the refined form (0, the default: every translation of
 * the site window, up to 2^23).  A small cap makes the first pass's lists
 * overflow, which exercises the second pass from the first pass's minima
 * (that pass uses the default lists); it exists for testing.  Errors:
 * INVALID_ARG (cap < 0). */
int bpmf_set_refine_list_cap(bpmf_ctx_t ctx, int cap);

/* bpmf_set_wait_test -- when on, the FP32 x pass does not request its first
 * receptor tile and waits for it about 2^20 cycles only, so every CTA's
 * bounded wait runs out and the next synchronising bpmf_eval returns
 * BPMF_ERR_TIMEOUT (no fault, no hang; CUDA graphs are not used meanwhile).
 * It exists for testing the timeout path.  Errors: INVALID_ARG. */
int bpmf_set_wait_test(bpmf_ctx_t ctx, int on);

/* Upper bound on the device workspace bpmf_eval may hold (bytes, default
 * an eighth of the device's memory, at most 16 GiB and at least 1 GiB);
 * configurations are processed in batches that fit, and fewer, larger
 * batches run faster.  Results do not depend on the batch size (every step
 * is deterministic).  Errors: INVALID_ARG (bytes < 1 MiB). */
int bpmf_set_workspace_limit(bpmf_ctx_t ctx, size_t bytes);

/*
 * bpmf_set_graph_mode -- when on, bpmf_eval records its whole device-side
 * launch sequence (table upload, every batch of every receptor group, the
 * merges, the result copies) into a CUDA graph on first use and replays the
 * graph on later calls with the same ligand handle, receptor handles, mode,
 * kT, output pointers and launch shapes.  Requires a non-default stream and
 * device-memory outputs (otherwise the call runs without a graph).  Results
 * are bit-identical with and without graphs.  Errors: INVALID_ARG.
 */
int bpmf_set_graph_mode(bpmf_ctx_t ctx, int on);

/*
 * bpmf_autotune -- time bpmf_eval on (lig, recs) under candidate launch
 * shapes (configurations per batch, lines per CTA of the strided passes, rows
 * per CTA of the z pass) and, in the FP32 and refined forms, the x transform's
 * plan (the x edge rounded up to the compile-time x pass, or the padded or crop
 * edge on the generic engine), and keep the fastest for every padded grid size
 * of `recs` and this mode.  The launch shapes give bit-identical results; the
 * x plan changes FP32 rounding only (the refined form's results stay within
 * its tolerance).  Runs ~12 evaluations and synchronises `stream`.
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED, OOM, CUDA.
 */
int bpmf_autotune(bpmf_ctx_t ctx, bpmf_lig_t lig, const bpmf_rec_t *recs, int K, unsigned mode, void *stream);

/* bpmf_valid_counts -- number of valid translations n_jk of every
 * configuration against every receptor (the ligand-box filter of bpmf_eval),
 * computed on the host from the configurations' coordinate bounds.
 * n_valid: HOST int64 [total_conf][K].  Errors: INVALID_ARG, SIZE_UNSUPPORTED. */
int bpmf_valid_counts(bpmf_ctx_t ctx, bpmf_lig_t lig, const bpmf_rec_t *recs, int K, int64_t *n_valid);

/* ------------------------------------------------------------------------
 * Learned proposal over configurations.  A small MLP predicts, from a
 * configuration's features, log sum_k S_jk (its weight in the sample mean of
 * Eq. sample_mean_BPMF) relative to its ligand's largest, clipped below
 * (bpmf_config_targets).  Configurations are then drawn from
 * q_j = mix * softmax(pred / tau)_j + (1 - mix) / J, and the BPMF is estimated by
 * importance weighting, which stays unbiased for Z_k = sum_j S_jk thanks to
 * the uniform component.  The full enumeration (bpmf_eval) is the fallback and
 * the reference for its error.
 * ------------------------------------------------------------------------ */
#define BPMF_N_FEATURES 24

/* bpmf_features -- per configuration, 24 float32 features:
 *  [0..3]   unit quaternion (w >= 0) of the rotation from the principal frame
 *           of the gyration tensor (axes by ascending moment, first two signed
 *           by a positive third moment, right-handed) to the lab frame;
 *  [4..6]   ligand-box extents u_d = ceil((max - min) / h) + 4 (nodes);
 *  [7..9]   principal moments of the gyration tensor (A^2), ascending;
 *  [10]     radius of gyration (A);  [11] end-to-end (first-last atom) distance;
 *  [12..15] sin, cos of the torsions of atoms (0,1,2,3) and (1,2,3,4);
 *  [16..23] atom counts in the 8 classes (R > 1.75) x (eps > 0.125) x (q > 0).
 * out: [total_conf][24], host or device.  Synchronises `stream`.
 * Errors: INVALID_ARG, OOM, CUDA. */
int bpmf_features(bpmf_ctx_t ctx, bpmf_lig_t lig, double h, float *out, void *stream);

typedef struct bpmf_mlp *bpmf_mlp_t;

/* Number of parameters of an MLP with n_in inputs, `depth` hidden ReLU layers
 * of `width` units and one output (0 for invalid sizes). */
long long bpmf_mlp_param_count(int n_in, int width, int depth);

/* bpmf_mlp_create -- an MLP n_in -> width (ReLU) -> ... -> width (ReLU) -> 1.
 *  params  HOST float32, packed layer by layer: W_l [in_l][out_l] row-major,
 *          then b_l [out_l]; bpmf_mlp_param_count() values.
 *  norm    HOST float32 [2 n_in + 2]: input shift[n_in], input scale[n_in],
 *          target shift, target scale (inputs are (x - shift) / scale; the
 *          network predicts (y - shift) / scale).
 * Weights are kept in FP32 (master copy for Adam); every GEMM rounds its
 * operands to bf16 and runs on the tensor cores with FP32 accumulation.
 * Errors: INVALID_ARG, OOM, CUDA. */
int bpmf_mlp_create(bpmf_ctx_t ctx, int n_in, int width, int depth, const float *params, const float *norm,
                    bpmf_mlp_t *out);
void bpmf_mlp_free(bpmf_mlp_t mlp);
/* Copy the current FP32 parameters (packed as in bpmf_mlp_create) to HOST params. */
int bpmf_mlp_get_params(bpmf_mlp_t mlp, float *params);
/* y[B] = prediction for features X[B][n_in]; both DEVICE memory. Stream ordered. */
int bpmf_mlp_forward(bpmf_ctx_t ctx, bpmf_mlp_t mlp, const float *X, int B, float *y, void *stream);
/* One training step on (X[B][n_in], t[B]) (DEVICE): mean squared error in
 * normalised units, backward pass, and (apply != 0) one Adam step with
 * learning rate lr (beta 0.9 / 0.999, eps 1e-8).  loss (host or device,
 * optional) receives the loss before the step; grads (device, optional) the
 * packed parameter gradients.  Synchronises `stream`. */
int bpmf_mlp_train_step(bpmf_ctx_t ctx, bpmf_mlp_t mlp, const float *X, const float *t, int B, float lr, int apply,
                        float *loss, float *grads, void *stream);

/* bpmf_proposal_sample -- q = mix softmax(pred / tau) + (1 - mix)/J over J
 * configurations (FP64); for each caller-supplied uniform u_s in [0,1) the
 * index of the first configuration whose cumulative q exceeds u_s, and q of
 * that configuration.  tau > 0 tempers the prediction (large tau: closer to
 * uniform).  pred [J] float32, u [M] float64, idx [M] int32, q_s [M]
 * float64: DEVICE memory.  Stream ordered.  Errors: INVALID_ARG, OOM, CUDA. */
int bpmf_proposal_sample(bpmf_ctx_t ctx, const float *pred, int J, double mix, double tau, const double *u, int M,
                         int *idx, double *q_s, void *stream);

/* bpmf_config_targets -- training targets of the proposal for ONE ligand's J
 * configurations (FP64): ls_j = ln sum_k n_jk exp(logZ_jk) (the
 * configuration's weight in the sample mean of Eq. sample_mean_BPMF, -inf
 * without a valid translation) and t_j = max(ls_j - max_j' ls_j', -clip)
 * (float32; the proposal needs only the ranking within a ligand).
 * logZ, n_valid [J][K] as bpmf_eval returns them; ls [J] float64, t [J]
 * float32: DEVICE memory.  Errors: INVALID_ARG (clip <= 0), CUDA. */
int bpmf_config_targets(bpmf_ctx_t ctx, const double *logZ, const int64_t *n_valid, int J, int K, double clip,
                        double *ls, float *t, void *stream);

/* bpmf_proposal_chi2 -- exact relative variance of the importance-sampling
 * estimate of Z = sum_j exp(ls_j) from ONE draw of the proposal q of
 * bpmf_proposal_sample (mix, tau): chi2 = sum_j exp(2 ls_j) / (q_j Z^2) - 1
 * (M independent draws: chi2 / M).  Used to choose tau on fully enumerated
 * ligands and to report a proposal's quality without sampling noise.
 * pred [J] float32, ls [J] float64, chi2 [1] float64: DEVICE memory.
 * Errors: INVALID_ARG, CUDA. */
int bpmf_proposal_chi2(bpmf_ctx_t ctx, const float *pred, const double *ls, int J, double mix, double tau, double *chi2,
                       void *stream);

/* bpmf_proposal_bpmf -- importance-weighted BPMF per receptor from M sampled
 * configurations: Z_k = (1/M) sum_s S_{j_s k} / q_s with S = exp(logZ) n,
 * B_k = -kT [ln Z_k - ln n_tot_k].  logZ_s [M][K], n_s [M][K] (as returned by
 * bpmf_eval for the sampled configurations), q_s [M], n_tot [K] (valid
 * translations summed over all J configurations), bpmf [K]: DEVICE memory,
 * FP64 arithmetic.  Errors: INVALID_ARG, CUDA. */
int bpmf_proposal_bpmf(bpmf_ctx_t ctx, const double *logZ_s, const int64_t *n_s, const double *q_s, int M, int K,
                       const int64_t *n_tot, double kT, double *bpmf, void *stream);

/*
 * bpmf_sir_poses -- sampling importance resampling of M poses of ligand
 * `lig_index` against receptor `rec`, with weight exp(-E/kT) over all its
 * (configuration, translation) poses (Section "Implicit solvent": poses drawn
 * from the bound state by sampling importance resampling before the
 * single-step perturbation).  Exact two-stage draw in FP64:
 *   conf[s] = first j with sum_{i<=j} S_i > u1[s] sum_i S_i, where
 *             S_j = n_valid[j][k] exp(logZ[j][k]) (inverse CDF over configurations);
 *   pose[s] = first window index t with sum_{i<=t} exp(-E_i/kT) >
 *             u2[s] sum_i exp(-E_i/kT), E = the energies of configuration
 *             conf[s] as bpmf_export_energies returns them (same mode).
 * The window index t = (s0 S1 + s1) S2 + s2 is translation
 * m_d = site_lo_d + s_d - floor(u_d/2) (u = the configuration's ligand box).
 *  logZ, n_valid  [J][K] float64 / int64 for this ligand's J configurations,
 *                 as bpmf_eval returns them (column k = this receptor);
 *  u1, u2         [M] float64 uniforms in [0, 1);  conf, pose [M] int32 out
 *                 (-1 where no pose has finite weight).
 * All arrays DEVICE memory.  Runs one energy export per distinct drawn
 * configuration and synchronises `stream`.
 * Errors: INVALID_ARG, SIZE_UNSUPPORTED, OOM, CUDA.
 */
int bpmf_sir_poses(bpmf_ctx_t ctx, bpmf_lig_t lig, int lig_index, bpmf_rec_t rec, int K, int k, double kT,
                   unsigned mode, const double *logZ, const int64_t *n_valid, const double *u1, const double *u2,
                   int M, int *conf, int *pose, void *stream);

/*
 * bpmf_bootstrap -- bootstrap uncertainty of the pooled BPMF and of the
 * standard binding free energy (results, "BPMF uncertainty": configurations
 * resampled with replacement), FP64.  Replicate r fills J slots with
 * configurations j = min(J - 1, floor(u[r][i] J)) and evaluates, per
 * receptor k, B_k = -kT [ln sum_slots n_jk exp(logZ_jk) - ln sum_slots n_jk],
 * then dG = -kT ln((1/K) sum_k exp(-B_k/kT)) - kT ln(h^3 C mean n) exactly as
 * bpmf_eval does for the full set (C = 6.02214076e-4 A^-3, 1 M).
 *   logZ, n_valid  [J][K] as bpmf_eval returns them for one ligand;
 *   u              [R][J] float64 uniforms in [0, 1);
 *   rep            [R][K + 1] out (B_k, then dG per replicate), may be null;
 *   stats          [2][K + 1] out: mean, then sample standard deviation
 *                  (ddof 1) over replicates, may be null (not both).
 * All arrays DEVICE memory; stream ordered.  Errors: INVALID_ARG, OOM, CUDA.
 */
int bpmf_bootstrap(bpmf_ctx_t ctx, const double *logZ, const int64_t *n_valid, int J, int K, double kT, double h,
                   const double *u, int R, double *rep, double *stats, void *stream);

/*
 * Kernel timing (tracing).  While enabled, every kernel the library launches
 * is bracketed by CUDA events recorded on the stream it runs on.
 * bpmf_profile_enable(ctx, 1) clears the counters and starts recording,
 * (ctx, 0) stops.  bpmf_profile_count waits for the recorded events and
 * returns the number of distinct kernels seen; bpmf_profile_entry(i) gives
 * kernel i's name (NUL-terminated, truncated to name_len), total device time
 * in milliseconds and number of launches.  Errors: INVALID_ARG, CUDA.
 */
int bpmf_profile_enable(bpmf_ctx_t ctx, int on);
int bpmf_profile_count(bpmf_ctx_t ctx);
int bpmf_profile_entry(bpmf_ctx_t ctx, int i, char *name, int name_len, double *total_ms, int64_t *launches);

/*
 * bpmf_export_energies_static -- the energy export of bpmf_export_energies
 * for callers that cannot allocate device memory.  The paper has no
 * counterpart; it exists for callers such as code running inside another
 * framework's pre-reserved memory pool, or threads that must not call
 * cudaMalloc/cudaFree because those synchronise the device.  It allocates
 * nothing: every intermediate (twiddle tables, generalised charges, the
 * receptor spectra, the ligand grid and all transform passes) lives in one
 * library-owned static device array of BPMF_STATIC_SCRATCH_BYTES, which every
 * GPU that loads this library holds until the process exits.
 *
 *  grids      [3][nx][ny][nz] float32 receptor grids (as bpmf_receptor_load),
 *             DEVICE memory of the current device.
 *  h, site_lo, site_n   as bpmf_receptor_load (site_lo / site_n host arrays).
 *  n_atoms, coords [n_atoms][3], q, eps, R [n_atoms]: one ligand
 *             configuration, DEVICE memory; p_rep, p_att as bpmf_ligand_batch.
 *  mode       BPMF_MODE_FP32 or BPMF_MODE_FF.
 *  out        [S0][S1][S2] float64 DEVICE memory (S = site_n): energy of
 *             translation m = site_lo + s - floor(u/2), +inf where discarded;
 *             the same values bpmf_export_energies returns.
 * Every array argument must be DEVICE memory of the current device (checked
 * per pointer with cudaPointerGetAttributes; host memory returns INVALID_ARG
 * before any work is queued).
 * Runs on the current device and on `stream`.  Each call reads the ligand's
 * coordinate bounds back to the host and synchronises `stream` before
 * returning, so no call can be captured into a CUDA graph.  The first call on
 * a device also resolves the array's device address (cudaGetSymbolAddress).
 * Every call shares the one array and
 * leaves its contents behind: calls whose GPU work overlaps (other threads,
 * other streams) race and must be serialised by the caller.
 * Errors: INVALID_ARG; SIZE_UNSUPPORTED when the grid or the ligand box needs
 * more scratch than BPMF_STATIC_SCRATCH_BYTES (a 96^3 grid with a ligand box
 * up to ~60 nodes per edge fits) or exceeds the other limits; CUDA.
 */
#define BPMF_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int bpmf_export_energies_static(const float *grids, int nx, int ny, int nz, double h, const int site_lo[3],
                                const int site_n[3], int n_atoms, const float *coords, const float *q,
                                const float *eps, const float *R, int p_rep, int p_att, unsigned mode, double *out,
                                void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BPMF_H */
