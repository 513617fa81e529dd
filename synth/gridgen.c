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
 * (clip <= 0 disables).  Returns 0, or -1 if scratch allocation fails. */
int gridgen_build(float *out, int nx, int ny, int nz, double h,
                  const double origin[3], int n_atoms, const double *xyz,
                  const double *q, const double *eps, const double *R,
                  double p_rep, double p_att, double coulomb, double clamp,
                  double clip)
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
