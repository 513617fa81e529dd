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
 * Steric clashes (Eq. occupancy_grid), when a receptor occupancy grid is
 * given: the ligand occupancy grid marks every node n with |g_i - n| <
 * 2^(-1/6) R_i / h for some atom i (R is the ligand's LJ size parameter, in
 * the role of sigma_ii); a valid translation m clashes when some occupied
 * ligand node n lands on an occupied receptor node m + n (nodes outside the
 * receptor grid are unoccupied).  A clashing translation keeps its place in
 * the sample (it counts in n_jk) with E = +infinity.  The occupancy of a
 * node is an integer decided by floating point, so it is decided in IEEE
 * single precision, in the fixed order written in ligand_occupancy().
 *
 * Sample mean (Eq. sample_mean_BPMF) for one configuration j and receptor k:
 *     log S_jk = log sum_{m valid} exp(-E(m) / kT),   n_jk = #valid
 * (clashing translations add nothing to the sum).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)

/* 2^(-1/3): the squared ratio of the occupancy radius to R */
#define OCC_R2_SCALE 0.79370052598409973737585281963615f

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

/* Occupied ligand nodes in the ligand-box frame (Eq. occupancy_grid).
 * Positions p_i = (x_i - min x) / h + 2 and thresholds (R_i / h)^2 2^(-1/3)
 * in single precision; node n is occupied when
 *     ((n_x - p_x)^2 + (n_y - p_y)^2) + (n_z - p_z)^2 < threshold_i
 * for some atom i, each operation rounded to single precision in this order.
 * Returns the number of occupied nodes written to nodes[3 * count] (NULL on
 * allocation failure, count = -1). */
static int *ligand_occupancy(int n_atoms, const float *xyz, const float *R, double h, int *count)
{
    const float hf = (float)h;
    float *p = (float *)malloc(sizeof(float) * 3 * (size_t)n_atoms);
    float *thr = (float *)malloc(sizeof(float) * (size_t)n_atoms);
    if (!p || !thr) {
        free(p);
        free(thr);
        *count = -1;
        return NULL;
    }
    float rmax = 0.0f;
    for (int d = 0; d < 3; ++d) {
        float lo = xyz[d];
        for (int i = 1; i < n_atoms; ++i)
            if (xyz[3 * i + d] < lo) lo = xyz[3 * i + d];
        for (int i = 0; i < n_atoms; ++i) {
            volatile float e = xyz[3 * i + d] - lo;
            volatile float q = e / hf;
            p[3 * i + d] = q + 2.0f;
        }
    }
    for (int i = 0; i < n_atoms; ++i) {
        volatile float r = R[i] / hf;
        volatile float r2 = r * r;
        thr[i] = r2 * OCC_R2_SCALE;
        if (r > rmax) rmax = r;
    }
    int lo[3], hi[3];
    for (int d = 0; d < 3; ++d) {
        float a = p[d], b = p[d];
        for (int i = 1; i < n_atoms; ++i) {
            if (p[3 * i + d] < a) a = p[3 * i + d];
            if (p[3 * i + d] > b) b = p[3 * i + d];
        }
        lo[d] = (int)floorf(a - rmax) - 1;
        hi[d] = (int)ceilf(b + rmax) + 1;
    }
    const size_t cap = (size_t)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
    int *nodes = (int *)malloc(sizeof(int) * 3 * cap);
    int cnt = 0;
    if (nodes) {
        for (int a = lo[0]; a <= hi[0]; ++a)
            for (int b = lo[1]; b <= hi[1]; ++b)
                for (int c = lo[2]; c <= hi[2]; ++c) {
                    int occ = 0;
                    for (int i = 0; i < n_atoms && !occ; ++i) {
                        volatile float dx = (float)a - p[3 * i];
                        volatile float dy = (float)b - p[3 * i + 1];
                        volatile float dz = (float)c - p[3 * i + 2];
                        volatile float xx = dx * dx, yy = dy * dy, zz = dz * dz;
                        volatile float s2 = xx + yy;
                        volatile float d2 = s2 + zz;
                        occ = d2 < thr[i];
                    }
                    if (occ) {
                        nodes[3 * cnt] = a;
                        nodes[3 * cnt + 1] = b;
                        nodes[3 * cnt + 2] = c;
                        ++cnt;
                    }
                }
    }
    free(p);
    free(thr);
    *count = nodes ? cnt : -1;
    return nodes;
}

/* Interaction energy of every translation in the site window, one
 * configuration against one receptor.
 * grids: [3][nx][ny][nz] FP32 (elec, LJr, LJa); gamma: [3][n_atoms] FP64.
 * occ: NULL, or the receptor occupancy grid [nx][ny][nz] (0 / 1), with R
 * [n_atoms] the ligand's LJ size parameters.
 * E: [S0][S1][S2], entry s holds translation m = lo + s - c, +INFINITY when
 * m is not valid or clashes.  *n_valid receives the number of valid
 * translations (clashing ones included). */
int oracle_pose_energies(const float *grids, const int dims[3], double h, const int site_lo[3],
                         const int site_n[3], int n_atoms, const float *xyz, const double *gamma,
                         const float *R, const unsigned char *occ, double *E, int64_t *n_valid)
{
    if (n_atoms < 1 || !(h > 0.0) || (occ && !R)) return ORACLE_EINVAL;
    double *g = (double *)malloc(sizeof(double) * 3 * (size_t)n_atoms);
    if (!g) return ORACLE_EINVAL;
    int u[3];
    oracle_place(n_atoms, xyz, h, g, u);
    int n_occ = 0;
    int *lnodes = NULL;
    if (occ) {
        lnodes = ligand_occupancy(n_atoms, xyz, R, h, &n_occ);
        if (!lnodes) {
            free(g);
            return ORACLE_EINVAL;
        }
    }
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
                ++cnt;
                int clash = 0;
                for (int t = 0; t < n_occ && !clash; ++t) {
                    const int x = m[0] + lnodes[3 * t], y = m[1] + lnodes[3 * t + 1], z = m[2] + lnodes[3 * t + 2];
                    if (x >= 0 && x < dims[0] && y >= 0 && y < dims[1] && z >= 0 && z < dims[2])
                        clash = occ[((size_t)x * dims[1] + y) * dims[2] + z] != 0;
                }
                if (clash) {
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
            }
    free(g);
    free(lnodes);
    *n_valid = cnt;
    return ORACLE_OK;
}

/* Occupied ligand nodes of one configuration (box frame), for the tests:
 * writes min(count, cap) nodes to nodes[3 * .] and returns count (-1 on
 * error). */
int oracle_ligand_occupancy(int n_atoms, const float *xyz, const float *R, double h, int *nodes, int cap)
{
    if (n_atoms < 1 || !(h > 0.0)) return -1;
    int n = 0;
    int *v = ligand_occupancy(n_atoms, xyz, R, h, &n);
    if (!v) return -1;
    for (int t = 0; t < n && t < cap; ++t)
        for (int d = 0; d < 3; ++d) nodes[3 * t + d] = v[3 * t + d];
    free(v);
    return n;
}

/* log S_jk, n_jk and min E for J configurations against one receptor, OpenMP
 * over configurations.  xyz: [J][n_atoms][3].  logS = -INFINITY when no
 * translation is valid (then Emin = +INFINITY). */
int oracle_logS_batch(const float *grids, const int dims[3], double h, const int site_lo[3],
                      const int site_n[3], int n_conf, int n_atoms, const float *xyz,
                      const double *gamma, const float *R, const unsigned char *occ, double kT,
                      double *logS, int64_t *n_valid, double *Emin)
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
            if (oracle_pose_energies(grids, dims, h, site_lo, site_n, n_atoms, xyz + (size_t)j * n_atoms * 3,
                                     gamma, R, occ, E, &cnt) != ORACLE_OK) {
#pragma omp atomic write
                err = 1;
                continue;
            }
            double mx = -INFINITY, emin = INFINITY;
            for (size_t s = 0; s < nS; ++s)
                if (isfinite(E[s])) {
                    if (-E[s] / kT > mx) mx = -E[s] / kT;
                    if (E[s] < emin) emin = E[s];
                }
            double acc = 0.0;
            for (size_t s = 0; s < nS; ++s)
                if (isfinite(E[s])) acc += exp(-E[s] / kT - mx);
            logS[j] = (cnt && acc > 0.0) ? mx + log(acc) : -INFINITY;
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
