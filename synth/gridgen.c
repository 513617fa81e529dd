/*
 * Seeded synthetic input support: receptor potential grids.
 *
 * This file builds the INPUTS of the hot path, not the hot path itself: the
 * three receptor grids of Eq. (receptor_grid), one value per grid node,
 *     G_t(n) = sum_j gamma_{t,j} V_t(|r_j - n|)
 * for t = electrostatic, LJ-repulsive, LJ-attractive, with the synthetic
 * recipe's constants (Coulomb factor, pair distance clamp, repulsive clip).
 * Both the FP64 oracle and the CUDA path read the grids this writes; neither
 * links this file.  FP64 accumulation, written out as FP32 (the grids are
 * FP32 inputs by contract).
 *
 * Node n = (i, j, k) sits at origin + (i, j, k) * h.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>

/* out: [3][nx][ny][nz] C order (elec, LJr, LJa).
 * atoms: [n_atoms][3] positions (A), q [n_atoms] (e), eps (kcal/mol), R (A).
 * p_rep / p_att: exponents of R in the receptor factors (12 and 6 in the
 * synthetic recipe), and 1/r^12, 1/r^6 distance laws.
 * clamp: r is clamped to >= clamp.  clip: LJr sum is clipped to <= clip
 * (clip <= 0 disables).  cutoff > 0: every term of atom j is zero for
 * r < cutoff * R_j (the overflow guard of the methodology, V(r) = 0 inside
 * 2^(-1/6) sigma; clash translations are then flagged by the occupancy
 * grids).  Returns 0, or -1 if scratch allocation fails. */
int gridgen_build(float *out, int nx, int ny, int nz, double h,
                  const double origin[3], int n_atoms, const double *xyz,
                  const double *q, const double *eps, const double *R,
                  double p_rep, double p_att, double coulomb, double clamp,
                  double clip, double cutoff)
{
    const size_t plane = (size_t)ny * nz, vol = (size_t)nx * plane;
    double *fr = (double *)malloc(sizeof(double) * (size_t)(n_atoms > 0 ? n_atoms : 1));
    double *fa = (double *)malloc(sizeof(double) * (size_t)(n_atoms > 0 ? n_atoms : 1));
    if (!fr || !fa) { free(fr); free(fa); return -1; }
    for (int a = 0; a < n_atoms; ++a) {
        fr[a] = sqrt(eps[a]) * pow(R[a], p_rep);
        fa[a] = sqrt(eps[a]) * pow(R[a], p_att);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < nx; ++i) {
        for (int j = 0; j < ny; ++j) {
            for (int k = 0; k < nz; ++k) {
                const double px = origin[0] + i * h;
                const double py = origin[1] + j * h;
                const double pz = origin[2] + k * h;
                double se = 0.0, sr = 0.0, sa = 0.0;
                for (int a = 0; a < n_atoms; ++a) {
                    const double dx = px - xyz[3 * a + 0];
                    const double dy = py - xyz[3 * a + 1];
                    const double dz = pz - xyz[3 * a + 2];
                    double r = sqrt(dx * dx + dy * dy + dz * dz);
                    if (cutoff > 0.0 && r < cutoff * R[a]) continue;
                    if (r < clamp) r = clamp;
                    const double ir = 1.0 / r;
                    const double ir2 = ir * ir;
                    const double ir6 = ir2 * ir2 * ir2;
                    se += q[a] * ir;
                    sr += fr[a] * ir6 * ir6;
                    sa += fa[a] * ir6;
                }
                se *= coulomb;
                if (clip > 0.0 && sr > clip) sr = clip;
                sa *= -2.0;
                const size_t idx = (size_t)i * plane + (size_t)j * nz + k;
                out[idx] = (float)se;
                out[vol + idx] = (float)sr;
                out[2 * vol + idx] = (float)sa;
            }
        }
    }
    free(fr);
    free(fa);
    return 0;
}

/* Receptor occupancy grid (Eq. occupancy_grid): out[i][j][k] = 1 when some
 * atom a has |r_a - n| < scale * R_a, else 0.  Decided in FP64 (the grid is
 * an input of both the oracle and the CUDA path). */
void gridgen_occupancy(unsigned char *out, int nx, int ny, int nz, double h, const double origin[3],
                       int n_atoms, const double *xyz, const double *R, double scale)
{
    const size_t plane = (size_t)ny * nz;
    for (size_t i = 0; i < (size_t)nx * plane; ++i) out[i] = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < n_atoms; ++a) {
        const double rad = scale * R[a];
        int lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            const int n = d == 0 ? nx : d == 1 ? ny : nz;
            lo[d] = (int)floor((xyz[3 * a + d] - rad - origin[d]) / h);
            hi[d] = (int)ceil((xyz[3 * a + d] + rad - origin[d]) / h);
            if (lo[d] < 0) lo[d] = 0;
            if (hi[d] > n - 1) hi[d] = n - 1;
        }
        for (int i = lo[0]; i <= hi[0]; ++i)
            for (int j = lo[1]; j <= hi[1]; ++j)
                for (int k = lo[2]; k <= hi[2]; ++k) {
                    const double dx = origin[0] + i * h - xyz[3 * a + 0];
                    const double dy = origin[1] + j * h - xyz[3 * a + 1];
                    const double dz = origin[2] + k * h - xyz[3 * a + 2];
                    if (dx * dx + dy * dy + dz * dz < rad * rad) out[(size_t)i * plane + (size_t)j * nz + k] = 1;
                }
    }
}
