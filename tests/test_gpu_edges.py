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
        if fin.any():
            assert np.abs(out["bpmf"][i][fin] - ref["bpmf"][fin]).max() <= B_TOL
        else:
            assert not np.isfinite(out["bpmf"][i]).any()
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


@pytest.mark.parametrize("n0,edge", [(60, 64), (70, 72), (84, 96), (100, 112), (117, 120), (126, 128)])
def test_fp32_x_edge_rounded_to_the_compile_time_x_pass(pkg, n0, edge):
    """In the FP32 forms the x-axis transform edge is rounded up to the
    compile-time x pass's edges (8 R, R = 8 ... 16) when that costs at most
    5/4 of the edge: zero padding past the grid changes no energy of the site
    window.  The refined form on such edges still meets the tolerances against
    the oracle, and the transform-edge query reports the rounded edge (the
    y and z edges stay the padded ones)."""
    from paper_1708_07045_gb300.session import Session
    h = 0.25
    atoms = synth.receptor_atoms(60 + n0, 300, 3.0, 14.0)
    shape = (n0, 24, 24)
    g, o = synth.receptor_grids(atoms, shape, h)
    lo, sn = synth.central_site(shape, (8, 6, 6))
    r = synth.ReceptorInput(g, h, o, lo, sn)
    lig = synth.LigandInput(synth.ligand_params(61, 5), synth.ligand_configs(62, 5, 4))
    with Session(0) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([lig])
        edges = pkg.bpmf_transform_edges(s.ctx, lh, [rh], 4, pkg.BPMF_MODE_REFINE)
        edges_ff = pkg.bpmf_transform_edges(s.ctx, lh, [rh], 4, pkg.BPMF_MODE_FF)
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=4)
    assert np.all(edges[:, 0, 0] == edge)
    assert np.all(edges[:, 0, 1:] == pkg.bpmf_fft_edge(24))
    assert np.all(edges_ff[:, 0, 0] == pkg.bpmf_fft_edge(n0))
    assert not (rc & pkg.BPMF_WARN_REFINE_FALLBACK)
    _check(out, [lig], [r])


def test_fp32_box_wider_than_the_padded_edge_next_to_a_small_one(pkg):
    """A ligand whose box (90 nodes along x) is wider than the receptor's
    padded edge (84) but not than the rounded x edge of the FP32 forms (96),
    batched with a small ligand: the batch buffers are sized by the boxes
    clamped to the bucket's own edges.  The wide ligand has no valid
    translation; the small one meets the tolerances."""
    from paper_1708_07045_gb300.session import Session
    h = 0.25
    atoms = synth.receptor_atoms(71, 300, 3.0, 14.0)
    shape = (84, 24, 24)
    g, o = synth.receptor_grids(atoms, shape, h)
    lo, sn = synth.central_site(shape, (8, 6, 6))
    r = synth.ReceptorInput(g, h, o, lo, sn)
    small = synth.LigandInput(synth.ligand_params(72, 5), synth.ligand_configs(73, 5, 4))
    wide_xyz = np.zeros((2, 3, 3), dtype=np.float32)
    wide_xyz[:, 1, 0] = 10.0
    wide_xyz[:, 2, 0] = 21.5  # u0 = ceil(21.5 / 0.25) + 4 = 90
    wide_xyz[1, :, 1] = 0.5
    wide = synth.LigandInput(synth.ligand_params(74, 3), wide_xyz)
    ligs = [small, wide]
    with Session(0) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands(ligs)
        edges = pkg.bpmf_transform_edges(s.ctx, lh, [rh], 6, pkg.BPMF_MODE_REFINE)
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=2, total_conf=6)
    assert np.all(edges[:, 0, 0] == 96)
    assert rc & pkg.BPMF_WARN_NO_VALID
    assert np.all(out["n_valid"][4:] == 0)
    _check(out, ligs, [r])


@pytest.mark.parametrize("shape", [(24, 84, 70), (24, 70, 84), (24, 90, 108), (24, 100, 100), (24, 108, 90)])
def test_fp32_yz_inverse_on_composite_edges(pkg, shape):
    """The FP32 forms' fused y + z inverse on compile-time edges A x R with a
    first factor other than 8 (70 = 7 x 10, 84 = 7 x 12, 90 = 9 x 10,
    100 = 10 x 10, 108 = 9 x 12): the refined form meets the tolerances
    against the oracle and the FP32 form stays within its error bound of it."""
    from paper_1708_07045_gb300.session import Session
    h = 0.25
    atoms = synth.receptor_atoms(80 + shape[1], 300, 3.0, 14.0)
    g, o = synth.receptor_grids(atoms, shape, h)
    lo, sn = synth.central_site(shape, (4, 8, 7))
    r = synth.ReceptorInput(g, h, o, lo, sn)
    lig = synth.LigandInput(synth.ligand_params(81, 5), synth.ligand_configs(82, 5, 4))
    with Session(0) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([lig])
        edges = pkg.bpmf_transform_edges(s.ctx, lh, [rh], 4, pkg.BPMF_MODE_REFINE)
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=4)
        _, out32 = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FP32, n_lig=1, total_conf=4)
    assert np.all(edges[:, 0, 1] == shape[1]) and np.all(edges[:, 0, 2] == shape[2])
    assert not (rc & pkg.BPMF_WARN_REFINE_FALLBACK)
    _check(out, [lig], [r])
    ref = oracle.evaluate([r], lig.coords, lig.params.q, lig.params.eps, lig.params.R, KT)
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    bound = sum(8 * 2.0 ** -24 * np.sqrt(np.log2(24.0 * shape[1] * shape[2])) *
                np.sqrt(np.mean(g[t].astype(np.float64) ** 2)) * np.linalg.norm(gam[t]) for t in range(3))
    fin = np.isfinite(ref["logZ"])
    assert np.array_equal(out32["n_valid"], ref["n_valid"])
    assert np.abs(out32["logZ"][fin] - ref["logZ"][fin]).max() * KT <= 2 * bound


def test_crops_from_kept_receptor_stages_match_fresh_receptors(pkg):
    """Receptor crops are x passes of float-pair y stages the receptor keeps
    per edge pair (made on first use, on side streams, ordered by events).
    A ligand evaluated against receptors whose stages and crops another
    ligand made first must give bit for bit the results of the same
    evaluation against freshly loaded copies of the receptors, in the refined
    and the float-pair forms; and the evaluation must use several crops."""
    from paper_1708_07045_gb300.session import Session
    w = synth.protein_scale(n_conf=1600, n_rec=2)
    lig = w.ligands[0]
    first = synth.LigandInput(lig.params, np.ascontiguousarray(lig.coords[:800]))
    second = synth.LigandInput(lig.params, np.ascontiguousarray(lig.coords[800:]))
    J = second.coords.shape[0]
    for mode in (pkg.BPMF_MODE_REFINE, pkg.BPMF_MODE_FF):
        with Session(0) as s:
            kept = [s.load_receptor(r) for r in w.receptors]
            lh1, _, _ = s.load_ligands([first])
            s.eval(lh1, kept, KT, mode, n_lig=1, total_conf=first.coords.shape[0])
            lh2, _, _ = s.load_ligands([second])
            edges = pkg.bpmf_transform_edges(s.ctx, lh2, kept, J, mode)
            classes = {tuple(e) for e in edges[:, 0, :]}
            assert len(classes) >= 3, classes  # several crops (and the full edge) in play
            _, reused = s.eval(lh2, kept, KT, mode, n_lig=1, total_conf=J)
            fresh = [s.load_receptor(r) for r in w.receptors]
            _, direct = s.eval(lh2, fresh, KT, mode, n_lig=1, total_conf=J)
        for k in ("logZ", "n_valid", "bpmf", "dG"):
            assert np.array_equal(reused[k], direct[k]), (mode, k)


def test_receptors_from_host_and_device_grids_agree(pkg):
    """bpmf_receptor_load copies host grids on the context's copy stream (the
    caller's stream waits for the copy; the call returns once it is done).
    Two host-memory loads queued back to back, and the same grids given as
    device memory, give the same results bit for bit; the host buffers may be
    overwritten as soon as each load returns."""
    torch = pytest.importorskip("torch")
    from paper_1708_07045_gb300.session import Session
    w = synth.protein_scale(n_conf=64, n_rec=2)
    lig = w.ligands[0]
    with Session(0) as s:
        host = []
        for r in w.receptors:
            buf = np.array(r.grids, dtype=np.float32, copy=True)
            host.append(s.load_receptor(r, grids=buf))
            buf[...] = np.nan  # the load has returned: the buffer is free again
        dev = [s.load_receptor(r, grids=torch.from_numpy(r.grids).cuda()) for r in w.receptors]
        lh, _, _ = s.load_ligands([lig])
        _, a = s.eval(lh, host, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=64)
        _, b = s.eval(lh, dev, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=64)
    for k in ("logZ", "n_valid", "bpmf", "dG"):
        assert np.array_equal(a[k], b[k]), k
    assert np.all(np.isfinite(a["bpmf"]))
