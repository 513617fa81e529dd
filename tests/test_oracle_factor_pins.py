"""Pins of the oracle parts that enter every energy and every dG through a
factor or a constant (CPU only): the ligand's generalised charges
(``oracle.gamma``), the standard-state concentration (``oracle.C_STANDARD``)
and the learned proposal's box-extent and atom-class features.

Each expected value is written here from its definition, never from the
function under test, and each test also plants the plausible mistake in a
copy of the oracle's arithmetic (on the CPU) to show that the pin fails it.
"""
import numpy as np
import pytest

import oracle
from oracle import proposal as P
import synth


# ----------------------------------------------------------------- gamma

def _pair_sum_from_lj(lig_xyz, lq, leps, lR, rec: synth.Atoms):
    """Receptor-ligand interaction written straight from the pair terms of
    Eq. general_form with Eqs. electrostatic, repulsive_LJ, attractive_LJ in
    the R form of the synthetic recipe and geometric combining:
        332.06 q_i q_j / r  +  sqrt(eps_i eps_j) (R_i R_j)^12 / r^12
                            -  2 sqrt(eps_i eps_j) (R_i R_j)^6  / r^6
    No factorisation into per-atom charges is used."""
    total = 0.0
    for i in range(lig_xyz.shape[0]):
        for j in range(rec.xyz.shape[0]):
            r = float(np.linalg.norm(lig_xyz[i] - rec.xyz[j]))
            e_ij = np.sqrt(float(leps[i]) * float(rec.eps[j]))
            rr = float(lR[i]) * float(rec.R[j])
            total += synth.COULOMB * float(lq[i]) * float(rec.q[j]) / r
            total += e_ij * rr ** 12 / r ** 12
            total -= 2.0 * e_ij * rr ** 6 / r ** 6
    return total


def _on_node_case():
    h = 0.5
    shape = (22, 20, 24)
    rec = synth.receptor_atoms(21, 12, 5.0, 6.5)
    # no clip: every node keeps its pair sum (the clamp is checked below)
    grids, origin = synth.receptor_grids(rec, shape, h, clip=1e30)
    lat = np.array([[0, 0, 0], [2, 0, 0], [2, 1, 0], [0, 1, 3], [1, 3, 2]], dtype=np.float64)
    xyz = (lat * h).astype(np.float32)
    lig = synth.ligand_params(22, lat.shape[0])
    lo, S = (9, 8, 10), (3, 3, 2)
    return h, rec, grids, origin, xyz, lig, lo, S


def _energies_with(gam, case):
    h, rec, grids, origin, xyz, lig, lo, S = case
    E, n = oracle.pose_energies(grids, h, lo, S, xyz, gam)
    assert n == int(np.prod(S))
    return E


def _expected(case):
    h, rec, grids, origin, xyz, lig, lo, S = case
    g, u = oracle.place(xyz, h)
    assert np.allclose(g, np.round(g))  # every atom on a node: no interpolation
    want = np.empty(S)
    for s in np.ndindex(*S):
        m = np.array(lo) + np.array(s) - u // 2
        pos = origin + (g + m) * h
        # no ligand node within the 0.5 A clamp radius of a receptor atom
        assert np.linalg.norm(pos[:, None, :] - rec.xyz[None], axis=-1).min() > 0.5
        want[s] = _pair_sum_from_lj(pos, lig.q, lig.eps, lig.R, rec)
    return want


def test_gamma_reproduces_the_lj_pair_terms():
    """Energies built from oracle.gamma equal the pair sum written from the
    combining rule, translation by translation."""
    case = _on_node_case()
    lig = case[5]
    E = _energies_with(oracle.gamma(lig.q, lig.eps, lig.R), case)
    want = _expected(case)
    assert np.all(np.isfinite(E))
    assert np.max(np.abs(E - want)) <= 2e-6 * max(1.0, np.max(np.abs(want)))


@pytest.mark.parametrize("mistake", ["eps_not_sqrt", "swapped_exponents", "attractive_R12"])
def test_gamma_pin_fails_a_planted_mistake(mistake):
    """The same comparison rejects the plausible mistakes in the charges:
    eps in place of sqrt(eps), the two LJ exponents swapped, R^12 in the
    attractive slot."""
    case = _on_node_case()
    lig = case[5]
    q = lig.q.astype(np.float64)
    eps = lig.eps.astype(np.float64)
    R = lig.R.astype(np.float64)
    if mistake == "eps_not_sqrt":
        bad = np.stack([q, eps * R ** 12, eps * R ** 6])
    elif mistake == "swapped_exponents":
        bad = np.stack([q, np.sqrt(eps) * R ** 6, np.sqrt(eps) * R ** 12])
    else:
        bad = np.stack([q, np.sqrt(eps) * R ** 12, np.sqrt(eps) * R ** 12])
    E = _energies_with(np.ascontiguousarray(bad), case)
    want = _expected(case)
    assert np.max(np.abs(E - want)) > 1e-3 * max(1.0, np.max(np.abs(want)))


def test_gamma_paper_sigma_form_exponents():
    """With (p_rep, p_att) = (6, 3) the factors are the paper's
    sqrt(eps) sigma^6 and sqrt(eps) sigma^3 (Eqs. repulsive_LJ,
    attractive_LJ), written here per atom."""
    lig = synth.ligand_params(5, 7)
    g = oracle.gamma(lig.q, lig.eps, lig.R, 6, 3)
    for i in range(7):
        s = float(lig.R[i])
        assert g[0, i] == float(lig.q[i])
        assert abs(g[1, i] - np.sqrt(float(lig.eps[i])) * s * s * s * s * s * s) <= 1e-15 * g[1, i]
        assert abs(g[2, i] - np.sqrt(float(lig.eps[i])) * s * s * s) <= 1e-15 * g[2, i]


# ------------------------------------------------------------ C_STANDARD

AVOGADRO = 6.02214076e23  # exact (SI 2019)
LITRE_IN_A3 = 1e27         # 1 L = 1 dm^3 = (1e9 A)^3


def test_standard_concentration_is_one_molar():
    """C = 1 mol/L in molecules per A^3 (the standard state of Eq.
    standard_binding_fe): N_A / 1e27."""
    want = AVOGADRO / LITRE_IN_A3
    assert abs(oracle.C_STANDARD - want) <= 1e-9 * want


def test_standard_state_term_in_dg():
    """dG of one receptor with B = 0 is -kT ln(V_site C): with V_site chosen
    as 1 L the term vanishes, with 1 mL it is kT ln 1000."""
    kT = 0.5925
    v_litre = LITRE_IN_A3 / AVOGADRO  # one molecule per litre... in A^3 per molecule at 1 M
    assert abs(oracle.dG([0.0], kT, v_litre)) <= 1e-9
    assert abs(oracle.dG([0.0], kT, v_litre / 1000.0) - kT * np.log(1000.0)) <= 1e-9
    # a planted mistake: C in molecules per nm^3 (a factor 1000) fails
    bad = -kT * np.log(v_litre * oracle.C_STANDARD * 1000.0)
    assert abs(bad - oracle.dG([0.0], kT, v_litre)) > 1.0


# ------------------------------------------------------ proposal features

def _hand_ligand():
    """Five atoms with hand-picked extents and parameter classes."""
    x = np.array([[0.00, 0.00, 0.00],
                  [1.10, 0.00, 0.00],
                  [1.10, 0.30, 0.00],
                  [1.10, 0.30, 2.00],
                  [0.40, 0.10, 1.00]], dtype=np.float32)
    # class bin = 4 (R > 1.75) + 2 (eps > 0.125) + 1 (q > 0)
    R = np.array([1.80, 1.60, 1.90, 1.70, 1.76], dtype=np.float32)
    eps = np.array([0.20, 0.10, 0.05, 0.13, 0.125], dtype=np.float32)
    q = np.array([0.3, -0.2, 0.0, 0.1, -0.2], dtype=np.float32)
    return x, q, eps, R


def test_features_box_extents_by_hand():
    """u_d = ceil(extent_d / h) + 4, the ligand box of "FFT-based BPMF
    Estimation": extents (1.1, 0.3, 2.0) A at h = 0.25 give ceil(4.4) + 4,
    ceil(1.2) + 4 and 8 + 4 (an exact multiple gains no extra node)."""
    x, q, eps, R = _hand_ligand()
    f = P.features(x, q, eps, R, 0.25)
    assert list(f[4:7]) == [9.0, 6.0, 12.0]
    # h = 0.5: ceil(2.2) + 4, ceil(0.6) + 4, 4 + 4
    f = P.features(x, q, eps, R, 0.5)
    assert list(f[4:7]) == [7.0, 5.0, 8.0]


def test_features_atom_classes_by_hand():
    """Counts in the 8 classes (R > 1.75, eps > 0.125, q > 0), strict
    inequalities: atom 0 -> 4+2+1 = 7, atom 1 -> 0, atom 2 -> 4, atom 3 ->
    2+1 = 3, atom 4 -> 4 (R 1.76 > 1.75; eps 0.125 is not above 0.125)."""
    x, q, eps, R = _hand_ligand()
    f = P.features(x, q, eps, R, 0.25)
    want = np.zeros(8)
    for b in (7, 0, 4, 3, 4):
        want[b] += 1
    assert np.array_equal(f[16:24], want)


def test_features_shape_terms_by_hand():
    """Radius of gyration, end-to-end distance and principal moments of a
    planar cross whose moments are known in closed form."""
    a, b = 2.0, 1.0
    x = np.array([[a, 0, 0], [-a, 0, 0], [0, b, 0], [0, -b, 0]], dtype=np.float32)
    z = np.zeros(4, dtype=np.float32)
    f = P.features(x, z, z + 0.1, z + 1.6, 0.25)
    # gyration tensor diag(2a^2/4, 2b^2/4, 0): ascending moments 0, b^2/2, a^2/2
    assert np.allclose(f[7:10], [0.0, b * b / 2, a * a / 2], atol=1e-12)
    assert abs(f[10] - np.sqrt((2 * a * a + 2 * b * b) / 4)) <= 1e-12
    assert abs(f[11] - np.sqrt(a * a + b * b)) <= 1e-6  # first (a,0,0) to last (0,-b,0)
