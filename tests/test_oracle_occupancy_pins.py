"""Pins of the oracle's steric-clash channel (Eq. occupancy_grid) to geometry,
to the paper's own FFT correlation of occupancy grids, and to special cases
(CPU only)."""
import numpy as np

import oracle
import synth

KT = 0.5925
SCALE = 2.0 ** (-1.0 / 6.0)


def _small(n_conf=12):
    return synth.plain_small_occ(n_conf=n_conf)


def test_ligand_occupancy_is_the_union_of_atom_balls():
    """Every node farther than 1e-5 (relative) inside an atom's ball is
    occupied, every node farther than that outside all balls is not; the
    count matches a brute-force FP64 count away from the sphere surfaces."""
    w = _small(4)
    lig = w.ligands[0]
    h = w.receptors[0].h
    for j in range(4):
        nodes = oracle.ligand_occupancy(lig.coords[j], lig.params.R, h)
        got = {tuple(v) for v in nodes}
        assert len(got) == len(nodes)
        x = lig.coords[j].astype(np.float64)
        p = (x - x.min(axis=0)) / h + 2.0
        rad = SCALE * lig.params.R.astype(np.float64) / h
        lo = np.floor(p.min(0) - rad.max()) - 2
        hi = np.ceil(p.max(0) + rad.max()) + 2
        ax = [np.arange(lo[d], hi[d] + 1) for d in range(3)]
        G = np.stack(np.meshgrid(*ax, indexing="ij"), -1).reshape(-1, 3)
        d = np.sqrt(((G[:, None, :] - p[None]) ** 2).sum(-1)) / rad[None]  # [nodes, atoms]
        inside = (d < 1 - 1e-5).any(1)
        outside = (d > 1 + 1e-5).all(1)
        for g, i_, o_ in zip(G.astype(int), inside, outside):
            t = tuple(g)
            if i_:
                assert t in got, t
            elif o_:
                assert t not in got, t
        assert inside.sum() <= len(got) <= inside.sum() + (~inside & ~outside).sum()


def _clash_by_fft(occ_R, nodes, valid_m):
    """The paper's method: the correlation of the ligand and receptor
    occupancy grids (zero padded, so not periodic) is positive exactly at
    the clashing translations."""
    N = np.array(occ_R.shape)
    off = nodes.min(0)
    ext = nodes.max(0) - off + 1
    L = np.zeros(tuple(ext), dtype=np.float64)
    L[tuple((nodes - off).T)] = 1.0
    size = tuple(int(v) for v in N + ext + 1)
    FR = np.fft.rfftn(occ_R.astype(np.float64), size, axes=(0, 1, 2))
    FL = np.fft.rfftn(L, size, axes=(0, 1, 2))
    C = np.fft.irfftn(FR * np.conj(FL), size, axes=(0, 1, 2))  # C(t) = sum_n L(n) R(n + t)
    out = []
    for m in valid_m:
        t = np.asarray(m) + off  # node n - off + m + off = m + n
        out.append(C[tuple(np.mod(t, size))] > 0.5)
    return np.array(out)


def test_clash_flags_equal_fft_correlation_of_occupancy_grids():
    w = _small(6)
    r, lig = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    n_clash = n_free = 0
    for j in range(6):
        E_occ, n = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, lig.coords[j], gam, occ=r.occ,
                                        R=lig.params.R)
        E, n0 = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, lig.coords[j], gam)
        assert n == n0
        _, u = oracle.place(lig.coords[j], r.h)
        valid = np.argwhere(np.isfinite(E))
        ms = [np.array(r.site_lo) + s - np.asarray(u) // 2 for s in valid]
        nodes = oracle.ligand_occupancy(lig.coords[j], lig.params.R, r.h)
        ref = _clash_by_fft(r.occ, nodes, ms)
        got = np.isinf(E_occ[tuple(valid.T)])
        assert np.array_equal(got, ref)
        # energies of the translations that do not clash are untouched
        free = ~got
        assert np.array_equal(E_occ[tuple(valid[free].T)], E[tuple(valid[free].T)])
        n_clash += int(got.sum())
        n_free += int(free.sum())
    assert n_clash > 0 and n_free > 0


def test_empty_and_full_receptor_occupancy():
    w = _small(3)
    r, lig = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    zero = np.zeros_like(r.occ)
    ones = np.ones_like(r.occ)
    a = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, lig.coords, gam, KT)
    b = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, lig.coords, gam, KT, occ=zero, R=lig.params.R)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    logS, nv, emin = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, lig.coords, gam, KT, occ=ones,
                                       R=lig.params.R)
    assert np.array_equal(nv, a[1]) and np.all(nv > 0)
    assert np.all(logS == -np.inf) and np.all(emin == np.inf)
    assert np.all(oracle.bpmf(logS[:, None], nv[:, None], KT) == np.inf)


def test_cutoff_grids_vanish_inside_the_radius():
    """Generator side of the clash treatment: V = 0 for r < 2^(-1/6) R_j."""
    atoms = synth.Atoms(np.array([[0.1, -0.2, 0.05]]), np.array([0.4]), np.array([0.1]), np.array([1.8]))
    shape, h = (24, 24, 24), 0.25
    g, o = synth.receptor_grids(atoms, shape, h, clamp=0.0, clip=0.0, cutoff=SCALE)
    occ = synth.receptor_occupancy(atoms, shape, h)
    X = o[:, None, None, None] + h * np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"))
    r = np.sqrt(((X - atoms.xyz[0][:, None, None, None]) ** 2).sum(0))
    rad = SCALE * 1.8
    far = r > rad * (1 + 1e-9)
    near = r < rad * (1 - 1e-9)
    assert np.all(g[:, near] == 0.0)
    assert np.allclose(g[0, far], synth.COULOMB * 0.4 / r[far], rtol=1e-6)
    assert np.array_equal(occ[near], np.ones(near.sum(), np.uint8)) and not occ[far].any()
