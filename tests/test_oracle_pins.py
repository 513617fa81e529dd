"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics,
independent of the oracle's own code (CPU only).

The paper prints no worked numeric example, so each pin is a closed form, an
exact identity, an invariance or a brute-force computation on a tiny case,
chosen so that a dropped term, a wrong sign or exponent, a transposed axis or
an off-by-one in placement / the translation filter fails at least one test.
"""
import itertools

import numpy as np
import pytest
from scipy.special import logsumexp

import oracle
import synth

KT = 0.5925


def _site(shape, S):
    return synth.central_site(shape, S)


# ---------------------------------------------------------------- placement

def test_placement_min_at_two_spacings_and_box():
    """Lowest x, y, z of the ligand sit exactly 2 spacings above planes 0
    ("FFT-based BPMF Estimation"); all trilinear corners fit in the box."""
    rng = np.random.default_rng(3)
    for h in (0.25, 0.375, 0.5):
        for _ in range(50):
            n = int(rng.integers(1, 40))
            x = rng.uniform(-7, 7, (n, 3)).astype(np.float32)
            g, u = oracle.place(x, h)
            assert np.allclose(g.min(axis=0), 2.0, atol=0, rtol=0)
            # box extent rule decided in single precision
            ext = (x.max(0) - x.min(0)).astype(np.float32)
            want = np.ceil((ext / np.float32(h)).astype(np.float32)).astype(int) + 4
            assert np.array_equal(u, want)
            corner_hi = np.floor(g).max(0) + 1
            assert np.all(corner_hi <= u - 1)
            # g is an exact affine image of x
            assert np.allclose((g - 2.0) * h + x.min(0).astype(np.float64), x.astype(np.float64), atol=1e-12)


def test_count_valid_closed_form_matches_enumeration():
    rng = np.random.default_rng(4)
    m = np.arange(-30, 40)
    for _ in range(300):
        dims = rng.integers(6, 30, 3)
        u = rng.integers(4, 20, 3)
        S = rng.integers(1, 12, 3)
        lo = np.array([rng.integers(-3, d) for d in dims])
        c = u // 2
        ok = [(m >= 0) & (m + u[d] <= dims[d] - 1) & (m + c[d] >= lo[d]) & (m + c[d] < lo[d] + S[d])
              for d in range(3)]
        brute = int((ok[0][:, None, None] & ok[1][None, :, None] & ok[2][None, None, :]).sum())
        assert oracle.count_valid(dims, u, lo, S) == brute


# ----------------------------------------------------------- energies: exact

def _pair_energy(lig_xyz, gam_lig, rec: synth.Atoms):
    """Brute-force receptor-ligand pair sum (Eqs. electrostatic, repulsive_LJ,
    attractive_LJ in the R^12 / R^6 factor form), no grid involved."""
    d = np.linalg.norm(lig_xyz[:, None, :] - rec.xyz[None, :, :], axis=-1)
    se = np.sqrt(rec.eps)
    e_el = synth.COULOMB * gam_lig[0][:, None] * rec.q[None, :] / d
    e_r = gam_lig[1][:, None] * (se * rec.R ** 12)[None, :] / d ** 12
    e_a = -2.0 * gam_lig[2][:, None] * (se * rec.R ** 6)[None, :] / d ** 6
    return float((e_el + e_r + e_a).sum())


def test_on_node_energies_equal_brute_force_pair_sums():
    """With every ligand atom on a grid node, the grid energy of every valid
    translation is the pairwise sum of Eq. general_form exactly (grid values
    are the inner sums of Eq. receptor_grid)."""
    h = 0.5
    shape = (24, 22, 26)  # distinct edges catch transposed axes
    rec = synth.receptor_atoms(11, 30, 4.5, 6.5)
    grids, origin = synth.receptor_grids(rec, shape, h)
    # an asymmetric 4-atom ligand on lattice points (spacing h)
    lat = np.array([[0, 0, 0], [2, 0, 0], [2, 1, 0], [2, 1, 3]], dtype=np.float64)
    xyz = (lat * h).astype(np.float32)
    lig = synth.ligand_params(12, 4)
    gam = oracle.gamma(lig.q, lig.eps, lig.R)
    lo, S = (10, 9, 11), (3, 4, 2)
    E, n = oracle.pose_energies(grids, h, lo, S, xyz, gam)
    g, u = oracle.place(xyz, h)
    assert np.allclose(g, np.round(g))
    checked = 0
    for s in itertools.product(*[range(v) for v in S]):
        m = np.array(lo) + np.array(s) - u // 2
        pos = origin + (g + m) * h
        want = _pair_energy(pos, gam, rec)
        assert np.isfinite(E[s])
        assert abs(E[s] - want) <= 2e-6 * max(1.0, abs(want)), (s, E[s], want)
        checked += 1
    assert checked == n == np.prod(S)


def test_multilinear_grids_are_interpolated_exactly():
    """Trilinear interpolation reproduces any multilinear function of the node
    indices exactly, so off-node energies have a closed form."""
    shape = (20, 17, 23)
    i, j, k = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    coef = np.array([[0.5, 0.3, -0.2, 0.7, 0.01, -0.02, 0.015, 0.003],
                     [1.0, -0.1, 0.4, 0.05, 0.0, 0.03, -0.01, -0.002],
                     [-0.3, 0.2, 0.1, -0.6, 0.02, 0.0, 0.01, 0.001]])

    def f(t, x, y, z):
        c = coef[t]
        return c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * y * z + c[6] * x * z + c[7] * x * y * z

    grids = np.stack([f(t, i, j, k) for t in range(3)]).astype(np.float32)
    grids64 = grids.astype(np.float64)
    rng = np.random.default_rng(5)
    h = 0.37
    xyz = rng.uniform(0, 2.2, (5, 3)).astype(np.float32)
    gam = rng.normal(size=(3, 5))
    lo, S = (5, 4, 6), (4, 3, 5)
    E, n = oracle.pose_energies(grids, h, lo, S, xyz, gam)
    g, u = oracle.place(xyz, h)
    # exact multilinear interpolation of the FP32-rounded grid: fit is exact
    # because each grid is multilinear before rounding; compare at FP32 scale
    for s in itertools.product(*[range(v) for v in S]):
        m = np.array(lo) + np.array(s) - u // 2
        if np.any(m < 0) or np.any(m + u > np.array(shape) - 1):
            assert np.isinf(E[s])
            continue
        p = g + m
        want = sum(gam[t, a] * f(t, *p[a]) for t in range(3) for a in range(5))
        scale = np.abs(gam).sum() * np.abs(grids64).max()
        assert abs(E[s] - want) <= 1e-6 * scale


def test_fft_correlation_identity_numpy():
    """Eq. fft_correlation_func: spreading the generalised charges to the
    trilinear corners and correlating with FT^-1[FT(G_R) . FT(G_L)*] (numpy
    FP64, translation by +m) equals the direct energies at every valid m."""
    w = synth.plain_small(n_conf=3)
    r = w.receptors[0]
    lig = w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    N = np.array(r.shape)
    Rf = np.fft.rfftn(r.grids.astype(np.float64), axes=(1, 2, 3))
    for j in range(3):
        E, n = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, lig.coords[j], gam)
        # independent spreading (numpy): 8 corners with trilinear weights
        x = lig.coords[j].astype(np.float64)
        gpos = (x - x.min(0)) / r.h + 2.0
        c0 = np.floor(gpos).astype(int)
        f = gpos - c0
        L = np.zeros((3,) + tuple(N))
        for dx, dy, dz in itertools.product((0, 1), repeat=3):
            wgt = np.where(dx, f[:, 0], 1 - f[:, 0]) * np.where(dy, f[:, 1], 1 - f[:, 1]) * \
                np.where(dz, f[:, 2], 1 - f[:, 2])
            for t in range(3):
                np.add.at(L[t], (c0[:, 0] + dx, c0[:, 1] + dy, c0[:, 2] + dz), wgt * gam[t])
        Lf = np.fft.rfftn(L, axes=(1, 2, 3))
        C = np.fft.irfftn((Rf * np.conj(Lf)).sum(0), s=tuple(N), axes=(0, 1, 2))
        _, u = oracle.place(lig.coords[j], r.h)
        scale = np.abs(r.grids).max() * np.abs(gam).sum()
        cnt = 0
        for s in itertools.product(*[range(v) for v in r.site_n]):
            m = np.array(r.site_lo) + np.array(s) - u // 2
            if np.isfinite(E[s]):
                assert abs(C[tuple(m)] - E[s]) <= 1e-12 * scale
                cnt += 1
        assert cnt == n > 0


# ------------------------------------------------------------ closed forms

def test_constant_grids_give_bpmf_U0():
    shape = (28, 28, 28)
    c = np.array([3.5, 0.25, -1.5])
    grids = (np.ones((3,) + shape) * c[:, None, None, None]).astype(np.float32)
    w = synth.plain_small(n_conf=4)
    lig = w.ligands[0]
    rec = synth.ReceptorInput(grids, 0.375, np.zeros(3), *_site(shape, 12))
    res = oracle.evaluate([rec], lig.coords, lig.params.q, lig.params.eps, lig.params.R, KT)
    gam = res["gamma"]
    U0 = float((c[:, None] * gam).sum())
    assert abs(res["bpmf"][0] - U0) <= 1e-9 * max(1, abs(U0))
    assert np.allclose(res["logZ"][:, 0], -U0 / KT, rtol=1e-12, atol=1e-9)


def test_single_atom_reduces_to_log_mean_exp_of_grid():
    w = synth.plain_small(n_conf=1)
    r = w.receptors[0]
    xyz = np.array([[1.234, -0.5, 2.0]], dtype=np.float32)
    lig = synth.ligand_params(7, 1)
    gam = oracle.gamma(lig.q, lig.eps, lig.R)
    g, u = oracle.place(xyz, r.h)
    assert np.array_equal(g[0], [2.0, 2.0, 2.0]) and np.array_equal(u, [4, 4, 4])
    logS, n, _ = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, xyz[None], gam, KT)
    # valid m: 0 <= m <= N-5, lo <= m + 2 < lo + S; atom sits on node m + 2
    vals = []
    N = r.shape
    for m in itertools.product(*[range(N[d]) for d in range(3)]):
        m = np.array(m)
        if np.all(m + 4 <= np.array(N) - 1) and np.all(m + 2 >= r.site_lo) and \
                np.all(m + 2 < np.array(r.site_lo) + r.site_n):
            node = tuple(m + 2)
            vals.append(sum(gam[t, 0] * float(r.grids[(t,) + node]) for t in range(3)))
    vals = np.array(vals)
    B_ref = -KT * (logsumexp(-vals / KT) - np.log(len(vals)))
    B = oracle.bpmf(logS[:, None], n[:, None], KT)[0]
    assert n[0] == len(vals)
    assert abs(B - B_ref) <= 1e-9 * max(1, abs(B_ref))


def test_identical_configurations_same_logz_and_pooling():
    """Pooling over configurations equals the sample mean over the
    concatenated pose list (Eq. sample_mean_BPMF over all samples)."""
    w = synth.plain_small(n_conf=5)
    r = w.receptors[0]
    lig = w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    coords = np.concatenate([lig.coords, lig.coords[:1]])
    logS, n, _ = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, coords, gam, KT)
    assert logS[0] == logS[-1] and n[0] == n[-1]
    allE = []
    for j in range(coords.shape[0]):
        E, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, coords[j], gam)
        allE.append(E[np.isfinite(E)])
    allE = np.concatenate(allE)
    B_ref = -KT * (logsumexp(-allE / KT) - np.log(allE.size))
    B = oracle.bpmf(logS[:, None], n[:, None], KT)[0]
    assert abs(B - B_ref) <= 1e-9 * max(1, abs(B_ref))
    # bounds: E_min <= B <= E_min + kT ln(N_total)
    assert allE.min() - 1e-9 <= B <= allE.min() + KT * np.log(allE.size) + 1e-9


# --------------------------------------------------------------- invariances

def test_translation_invariance_of_grid_embedding():
    """Embedding the receptor grid with extra nodes on the low side and
    shifting the site box by the same amount leaves every BPMF unchanged
    (the site box is small enough that the grid edges never bind)."""
    h = 0.375
    rec = synth.receptor_atoms(21, 400, 4.0, 10.0)
    grids, origin = synth.receptor_grids(rec, (40, 40, 40), h)
    lo, S = synth.central_site((40, 40, 40), 6)
    r = synth.ReceptorInput(grids, h, origin, lo, S)
    lig = synth.ligand_params(22, 12)
    coords = synth.ligand_configs(23, 12, 6)
    d = (3, 1, 2)
    big = np.zeros((3,) + tuple(np.array(r.shape) + np.array(d)), dtype=np.float32)
    big[:, d[0]:, d[1]:, d[2]:] = r.grids
    r2 = synth.ReceptorInput(big, r.h, r.origin - np.array(d) * r.h,
                             tuple(np.array(r.site_lo) + d), r.site_n)
    a = oracle.evaluate([r], coords, lig.q, lig.eps, lig.R, KT)
    b = oracle.evaluate([r2], coords, lig.q, lig.eps, lig.R, KT)
    assert np.all(a["n_valid"] == np.prod(S))
    assert np.array_equal(a["n_valid"], b["n_valid"])
    assert np.allclose(a["logS"], b["logS"], rtol=0, atol=1e-10)
    assert np.allclose(a["bpmf"], b["bpmf"], rtol=0, atol=1e-10)


def test_axis_permutation_invariance():
    w = synth.plain_small(n_conf=4)
    r = w.receptors[0]
    lig = w.ligands[0]
    perm = (2, 0, 1)
    gp = np.ascontiguousarray(np.transpose(r.grids, (0,) + tuple(p + 1 for p in perm)))
    rp = synth.ReceptorInput(gp, r.h, r.origin[list(perm)], tuple(np.array(r.site_lo)[list(perm)]),
                             tuple(np.array(r.site_n)[list(perm)]))
    cp = np.ascontiguousarray(lig.coords[:, :, list(perm)])
    a = oracle.evaluate([r], lig.coords, lig.params.q, lig.params.eps, lig.params.R, KT)
    b = oracle.evaluate([rp], cp, lig.params.q, lig.params.eps, lig.params.R, KT)
    assert np.array_equal(a["n_valid"], b["n_valid"])
    assert np.allclose(a["logS"], b["logS"], rtol=0, atol=1e-9)


def test_linearity_in_grids():
    w = synth.plain_small(n_conf=2)
    r = w.receptors[0]
    lig = w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    rng = np.random.default_rng(9)
    g2 = rng.normal(size=r.grids.shape).astype(np.float32)
    # combination chosen exactly representable in FP32
    g3 = (r.grids.astype(np.float64) + 2.0 * g2.astype(np.float64)).astype(np.float32)
    resid = g3.astype(np.float64) - r.grids.astype(np.float64) - 2.0 * g2.astype(np.float64)
    E1, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, lig.coords[0], gam)
    E2, _ = oracle.pose_energies(g2, r.h, r.site_lo, r.site_n, lig.coords[0], gam)
    E3, _ = oracle.pose_energies(g3, r.h, r.site_lo, r.site_n, lig.coords[0], gam)
    Er, _ = oracle.pose_energies(resid.astype(np.float32), r.h, r.site_lo, r.site_n, lig.coords[0], gam)
    ok = np.isfinite(E1)
    scale = np.abs(gam).sum() * np.abs(g3).max()
    assert np.allclose(E3[ok], E1[ok] + 2 * E2[ok] + Er[ok], rtol=0, atol=1e-9 * scale)


def test_dG_site_volume_normalisation_invariance():
    """With one receptor, V_site <exp(-B/kT)> = h^3 (1/J) sum_j S_j, so dG does
    not depend on how the per-configuration valid counts normalise B."""
    w = synth.plain_small(n_conf=6)
    r = w.receptors[0]
    lig = w.ligands[0]
    res = oracle.evaluate([r], lig.coords, lig.params.q, lig.params.eps, lig.params.R, KT)
    J = lig.coords.shape[0]
    want = -KT * (logsumexp(res["logS"][:, 0]) - np.log(J) + np.log(r.h ** 3 * oracle.C_STANDARD))
    assert abs(res["dG"] - want) <= 1e-9 * max(1, abs(want))


def test_no_valid_translation_gives_minus_inf():
    w = synth.plain_small(n_conf=1)
    r = w.receptors[0]
    # a ligand longer than the grid: no translation keeps the box inside
    xyz = np.array([[0, 0, 0], [14.0, 0, 0]], dtype=np.float32)
    lig = synth.ligand_params(3, 2)
    gam = oracle.gamma(lig.q, lig.eps, lig.R)
    logS, n, emin = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, xyz[None], gam, KT)
    assert n[0] == 0 and logS[0] == -np.inf and emin[0] == np.inf
    assert oracle.bpmf(logS[:, None], n[:, None], KT)[0] == np.inf
