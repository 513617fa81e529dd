/*
 * FP64 reference ("oracle") for the FFT-correlation BPMF hot path.
 *
 * TEST INFRASTRUCTURE ONLY: the parity tests, the smoke check and the
 * benchmark's CPU-baseline leg call this; the product path never does.  It
 * shares no code, header or table with the CUDA library.
 *
 * What it computes is the plain definition that the FFT method reaches
 * exactly for every valid translation: the ligand's generalised charges
 * gamma_{t,i} (Eq. general_form, Eqs. electrostatic / repulsive_LJ /
 * attractive_LJ) spread to the 8 trilinear corners, correlated with the
 * receptor grids G_t (Eq. receptor_grid, Eq. correlation_func).  Spreading by
 * trilinear weights and then correlating equals trilinear interpolation of
 * each G_t at each atom, so for each translation m the oracle evaluates
 *     E(m) = sum_i sum_t gamma_{t,i} * trilinear(G_t, g_i + m)
 * directly, in FP64, one pose at a time.  g_i is the atom's position in grid
 * units after placement (Methodology, "FFT-based BPMF Estimation": lowest
 * x, y, z two grid spacings above the planes i, j, k = 0).
 *
 * Translation filter (same section): the ligand box spans nodes 0..u_d per
 * axis with u_d = ceil(extent_d / h) + 4; translation m is kept when the box
 * stays inside the receptor grid (m_d >= 0 and m_d + u_d <= N_d - 1) and the
 * box centre c_d = floor(u_d / 2) lands in the site box
 * (lo_d <= m_d + c_d < lo_d + S_d).  u_d is an integer decided by floating
 * point, so it is decided in IEEE single precision exactly as the CUDA path
 * decides it (correctly rounded subtract and divide, then ceil).
 *
 * Sample mean (Eq. sample_mean_BPMF) for one configuration j and receptor k:
 *     log S_jk = log sum_{m valid} exp(-E(m) / kT),   n_jk = #valid.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* Placement of one configuration: g[n][3] grid-unit coordinates of each atom
 * relative to the ligand-box corner, u[3] the ligand-box extents (nodes).
 * Returns ORACLE_OK or ORACLE_EINVAL (n_atoms < 1, h <= 0). */
int oracle_place(int n_atoms, const float *xyz, double h, double *g, int *u)
{
    if (n_atoms < 1 || !(h > 0.0)) return ORACLE_EINVAL;
    for (int d = 0; d < 3; ++d) {
        float lo = xyz[d], hi = xyz[d];
        for (int i = 1; i < n_atoms; ++i) {
            const float v = xyz[3 * i + d];
            if (v < lo) lo = v;
            if (v > hi) hi = v;
        }
        /* integer box extent, decided in single precision */
        volatile float ext = hi - lo;
        volatile float hf = (float)h;
        volatile float ratio = ext / hf;
        u[d] = (int)ceilf(ratio) + 4;
        for (int i = 0; i < n_atoms; ++i)
            g[3 * i + d] = ((double)xyz[3 * i + d] - (double)lo) / h + 2.0;
    }
    return ORACLE_OK;
}

/* Number of valid translations along one axis and the first valid m. */
static int axis_range(int N, int u, int lo, int S, int *m0)
{
    const int c = u / 2;
    int a = lo - c;            /* site condition: lo <= m + c */
    int b = lo + S - 1 - c;    /*                 m + c < lo + S */
    if (a < 0) a = 0;          /* box inside the grid */
    if (b > N - 1 - u) b = N - 1 - u;
    *m0 = a;
    return b >= a ? b - a + 1 : 0;
}

static double trilinear(const float *G, const int dims[3], const double p[3])
{
    int c[3];
    double f[3];
    for (int d = 0; d < 3; ++d) {
        double fl = floor(p[d]);
        int ci = (int)fl;
        /* a position exactly on the last node uses the cell below it */
        if (ci > dims[d] - 2) ci = dims[d] - 2;
        if (ci < 0) ci = 0;
        c[d] = ci;
        f[d] = p[d] - (double)ci;
    }
    const size_t sy = (size_t)dims[2], sx = (size_t)dims[1] * dims[2];
    double v = 0.0;
    for (int dx = 0; dx < 2; ++dx)
        for (int dy = 0; dy < 2; ++dy)
            for (int dz = 0; dz < 2; ++dz) {
                const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) *
                                 (dz ? f[2] : 1.0 - f[2]);
                const size_t idx = (size_t)(c[0] + dx) * sx + (size_t)(c[1] + dy) * sy + (size_t)(c[2] + dz);
                v += w * (double)G[idx];
            }
    return v;
}

/* Interaction energy of every translation in the site window, one
 * configuration against one receptor.
 * grids: [3][nx][ny][nz] FP32 (elec, LJr, LJa); gamma: [3][n_atoms] FP64.
 * E: [S0][S1][S2], entry s holds translation m = lo + s - c, +INFINITY when
 * m is not valid.  *n_valid receives the number of finite entries. */
int oracle_pose_energies(const float *grids, const int dims[3], double h, const int site_lo[3],
                         const int site_n[3], int n_atoms, const float *xyz, const double *gamma,
                         double *E, int64_t *n_valid)
{
    if (n_atoms < 1 || !(h > 0.0)) return ORACLE_EINVAL;
    double *g = (double *)malloc(sizeof(double) * 3 * (size_t)n_atoms);
    if (!g) return ORACLE_EINVAL;
    int u[3];
    oracle_place(n_atoms, xyz, h, g, u);
    const size_t vol = (size_t)dims[0] * dims[1] * dims[2];
    int64_t cnt = 0;
    for (int s0 = 0; s0 < site_n[0]; ++s0)
        for (int s1 = 0; s1 < site_n[1]; ++s1)
            for (int s2 = 0; s2 < site_n[2]; ++s2) {
                const int s[3] = {s0, s1, s2};
                int m[3], ok = 1;
                for (int d = 0; d < 3; ++d) {
                    m[d] = site_lo[d] + s[d] - u[d] / 2;
                    if (m[d] < 0 || m[d] + u[d] > dims[d] - 1) ok = 0;
                }
                const size_t o = ((size_t)s0 * site_n[1] + s1) * site_n[2] + s2;
                if (!ok) {
                    E[o] = INFINITY;
                    continue;
                }
                double e = 0.0;
                for (int i = 0; i < n_atoms; ++i) {
                    const double p[3] = {g[3 * i] + m[0], g[3 * i + 1] + m[1], g[3 * i + 2] + m[2]};
                    for (int t = 0; t < 3; ++t)
                        e += gamma[(size_t)t * n_atoms + i] * trilinear(grids + t * vol, dims, p);
                }
                E[o] = e;
                ++cnt;
            }
    free(g);
    *n_valid = cnt;
    return ORACLE_OK;
}

/* log S_jk, n_jk and min E for J configurations against one receptor, OpenMP
 * over configurations.  xyz: [J][n_atoms][3].  logS = -INFINITY when no
 * translation is valid (then Emin = +INFINITY). */
int oracle_logS_batch(const float *grids, const int dims[3], double h, const int site_lo[3],
                      const int site_n[3], int n_conf, int n_atoms, const float *xyz,
                      const double *gamma, double kT, double *logS, int64_t *n_valid, double *Emin)
{
    if (n_atoms < 1 || !(h > 0.0) || !(kT > 0.0) || n_conf < 0) return ORACLE_EINVAL;
    const size_t nS = (size_t)site_n[0] * site_n[1] * site_n[2];
    int err = 0;
#pragma omp parallel
    {
        double *E = (double *)malloc(sizeof(double) * (nS ? nS : 1));
        if (!E) {
#pragma omp atomic write
            err = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int j = 0; j < n_conf; ++j) {
            if (!E) continue;
            int64_t cnt = 0;
            oracle_pose_energies(grids, dims, h, site_lo, site_n, n_atoms, xyz + (size_t)j * n_atoms * 3,
                                 gamma, E, &cnt);
            double mx = -INFINITY, emin = INFINITY;
            for (size_t s = 0; s < nS; ++s)
                if (isfinite(E[s])) {
                    if (-E[s] / kT > mx) mx = -E[s] / kT;
                    if (E[s] < emin) emin = E[s];
                }
            double acc = 0.0;
            for (size_t s = 0; s < nS; ++s)
                if (isfinite(E[s])) acc += exp(-E[s] / kT - mx);
            logS[j] = cnt ? mx + log(acc) : -INFINITY;
            n_valid[j] = cnt;
            Emin[j] = emin;
        }
        free(E);
    }
    return err ? ORACLE_EINVAL : ORACLE_OK;
}

/* Closed-form count of valid translations (product of per-axis counts). */
int64_t oracle_count_valid(const int dims[3], const int u[3], const int site_lo[3], const int site_n[3])
{
    int64_t n = 1;
    for (int d = 0; d < 3; ++d) {
        int m0;
        n *= axis_range(dims[d], u[d], site_lo[d], site_n[d], &m0);
    }
    return n;
}
