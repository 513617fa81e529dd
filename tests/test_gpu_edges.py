"""Edge cases of the CUDA path against the FP64 oracle: ligands with no
configurations or a single atom in one batch, the largest padded FFT edge
(256), and ligand boxes whose spreading plane exceeds one shared-memory pass."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu
KT = synth.KT
E_TOL, B_TOL = 1e-3, 1e-2


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    import paper_1708_07045_gb300 as p
    p.lib()
    return p


def _run(pkg, recs, ligs):
    from paper_1708_07045_gb300.session import Session
    with Session(0) as s:
        rhs = [s.load_receptor(r) for r in recs]
        lh, _, nconf = s.load_ligands(ligs)
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, n_lig=len(ligs), total_conf=max(sum(nconf), 1))
    return rc, out


def _check(out, ligs, recs):
    off = 0
    for i, l in enumerate(ligs):
        J = l.coords.shape[0]
        if J == 0:
            assert np.all(np.isinf(out["bpmf"][i])) and np.isinf(out["dG"][i])
            continue
        ref = oracle.evaluate(recs, l.coords, l.params.q, l.params.eps, l.params.R, KT)
        assert np.array_equal(out["n_valid"][off:off + J], ref["n_valid"])
        ok = np.isfinite(ref["logZ"])
        if ok.any():
            assert np.abs(out["logZ"][off:off + J][ok] - ref["logZ"][ok]).max() * KT <= E_TOL
        fin = np.isfinite(ref["bpmf"])
        assert np.abs(out["bpmf"][i][fin] - ref["bpmf"][fin]).max() <= B_TOL
        off += J


def test_empty_and_single_atom_ligands_in_one_batch(pkg):
    w = synth.plain_small(n_conf=1)
    r = w.receptors[0]
    ligs = [synth.LigandInput(synth.ligand_params(31, 1), synth.ligand_configs(32, 1, 5)),
            synth.LigandInput(synth.ligand_params(33, 7), np.zeros((0, 7, 3), dtype=np.float32)),
            synth.LigandInput(synth.ligand_params(35, 4), synth.ligand_configs(36, 4, 3))]
    rc, out = _run(pkg, [r], ligs)
    _check(out, ligs, [r])


def test_largest_fft_edge_and_chunked_spreading(pkg):
    h = 0.25
    # x edge 256 (the largest padded edge), y/z edges small
    rec_a = synth.receptor_atoms(41, 200, 2.0, 40.0)
    g1, o1 = synth.receptor_grids(rec_a, (256, 20, 20), h)
    r1 = synth.ReceptorInput(g1, h, o1, (120, 4, 4), (16, 6, 6))
    lig1 = synth.LigandInput(synth.ligand_params(42, 6), synth.ligand_configs(43, 6, 4))
    rc, out = _run(pkg, [r1], [lig1])
    _check(out, [lig1], [r1])
    # a ligand box of 120 x 120 nodes across y and z: the spreading plane needs
    # two shared-memory passes
    g2, o2 = synth.receptor_grids(rec_a, (24, 128, 128), h)
    r2 = synth.ReceptorInput(g2, h, o2, (8, 60, 60), (4, 6, 6))
    xyz = np.array([[[0.0, 0.0, 0.0], [0.2, 14.0, 14.0], [0.1, 29.0, 29.0]]], dtype=np.float32)
    lig2 = synth.LigandInput(synth.ligand_params(44, 3), xyz)
    g, u = oracle.place(xyz[0], h)
    assert u[1] * u[2] * 8 > 96 * 1024  # larger than one pass
    rc, out = _run(pkg, [r2], [lig2])
    _check(out, [lig2], [r2])
    assert out["n_valid"].sum() > 0
