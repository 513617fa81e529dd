"""Parity of the CUDA hot path (through the C ABI) with the FP64 oracle.

Tolerances (the benchmark spec's figures, stated here once):
  * energies: |E_gpu - E_oracle| <= 1e-3 kcal/mol for every valid translation
    whose oracle energy is within 20 kT of that configuration's minimum;
  * BPMF and standard binding free energy: <= 0.01 kcal/mol;
  * log Z_jk: kT |d log Z| <= 1e-3 kcal/mol (it is a weighted mean of the
    energies inside the same 20 kT window);
  * valid-translation counts and the translation mask: exact.
These bind the float-pair (BPMF_MODE_FF) form.  The plain FP32 form is held to
a bound derived from FP32 FFT roundoff instead (see _fp32_bound).
"""
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


@pytest.fixture(scope="module")
def small():
    return synth.plain_small(n_conf=64)


@pytest.fixture(scope="module")
def small_ref(small):
    r, l = small.receptors[0], small.ligands[0]
    return oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)


def _session(pkg, **kw):
    from paper_1708_07045_gb300.session import Session
    return Session(0, **kw)


def _fp32_bound(grids, gam, P):
    """FP32 FFT-correlation roundoff bound per energy: for each term t,
    8 * eps32 * sqrt(log2 P^3) * rms(G_t) * ||G_L,t||_2 with ||G_L,t||_2 <=
    ||gamma_t||_2 (trilinear weights sum to one per atom), summed over t."""
    eps = 2.0 ** -24
    lg = np.sqrt(np.log2(float(np.prod(P))))
    return sum(8 * eps * lg * np.sqrt(np.mean(grids[t].astype(np.float64) ** 2)) * np.linalg.norm(gam[t])
               for t in range(3))


# ------------------------------------------------------------------ energies
@pytest.mark.parametrize("conf", [0, 1, 13, 63])
def test_export_energies_match_oracle_ff(pkg, small, conf):
    r, l = small.receptors[0], small.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    E_ref, n_ref = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[conf], gam)
    with _session(pkg) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        E = s.export_energies(lh, rh, 0, conf, r.site_n, pkg.BPMF_MODE_FF)
    assert np.array_equal(np.isinf(E), np.isinf(E_ref)), "translation mask differs"
    ok = np.isfinite(E_ref)
    assert ok.sum() == n_ref > 0
    win = ok & (E_ref <= E_ref[ok].min() + 20 * KT)
    err = np.abs(E[ok] - E_ref[ok])
    assert np.abs(E[win] - E_ref[win]).max() <= E_TOL
    # every other valid pose: float-pair roundoff relative to the grid scale
    scale = sum(np.abs(r.grids[t]).max() * np.abs(gam[t]).sum() for t in range(3))
    assert err.max() <= 1e-9 * scale


def test_export_energies_fp32_within_derived_bound(pkg, small):
    r, l = small.receptors[0], small.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    E_ref, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[0], gam)
    with _session(pkg) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        E = s.export_energies(lh, rh, 0, 0, r.site_n, pkg.BPMF_MODE_FP32)
    ok = np.isfinite(E_ref)
    assert np.array_equal(np.isinf(E), ~ok)
    bound = _fp32_bound(r.grids, gam, r.shape)
    err = np.abs(E[ok] - E_ref[ok])
    print(f"FP32 max |dE| {err.max():.3g} kcal/mol, rms {np.sqrt((err ** 2).mean()):.3g}, bound {bound:.3g}")
    assert err.max() <= bound


# --------------------------------------------------------------- full eval
def _check_eval(out, ref, K, n_lig_rows=None):
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    ok = np.isfinite(ref["logZ"])
    assert np.array_equal(np.isfinite(out["logZ"]), ok)
    if ok.any():
        assert np.abs(out["logZ"][ok] - ref["logZ"][ok]).max() * KT <= E_TOL
    fin = np.isfinite(ref["bpmf"])
    assert np.array_equal(np.isfinite(out["bpmf"][0]), fin)
    assert np.abs(out["bpmf"][0][fin] - ref["bpmf"][fin]).max() <= B_TOL
    if np.isfinite(ref["dG"]):
        assert abs(out["dG"][0] - ref["dG"]) <= B_TOL


def test_eval_small_ff(pkg, small, small_ref):
    r, l = small.receptors[0], small.ligands[0]
    with _session(pkg) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=64)
    assert rc in (pkg.BPMF_OK, pkg.BPMF_WARN_NO_VALID)
    _check_eval(out, small_ref, 1)


def test_eval_small_fp32_error_reported(pkg, small, small_ref):
    r, l = small.receptors[0], small.ligands[0]
    with _session(pkg) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FP32, n_lig=1, total_conf=64)
    assert np.array_equal(out["n_valid"], small_ref["n_valid"])
    gam = small_ref["gamma"]
    bound = _fp32_bound(r.grids, gam, r.shape)
    ok = np.isfinite(small_ref["logZ"])
    dz = np.abs(out["logZ"][ok] - small_ref["logZ"][ok]).max() * KT
    dB = abs(out["bpmf"][0, 0] - small_ref["bpmf"][0])
    print(f"FP32: max kT|dlogZ| {dz:.3g}, |dB| {dB:.3g} kcal/mol (energy bound {bound:.3g})")
    assert dz <= bound and dB <= bound


def test_uneven_ligands_receptors_and_no_valid_warning(pkg):
    """Several ligands of uneven size and configuration count against two
    receptor conformations on a non-cubic grid (edges 40, 36, 30: radices 2, 3,
    4, 5, 8) with different site boxes; one configuration is longer than the
    grid and has no valid translation."""
    h = 0.4
    shape = (40, 36, 30)
    base = synth.receptor_atoms(77, 300, 3.0, 9.0)
    recs = []
    for k, (S, off) in enumerate([((10, 8, 6), (0, 0, 0)), ((7, 9, 5), (2, -1, 1))]):
        atoms = synth.jitter(base, 0.3, 78 + k)
        g, o = synth.receptor_grids(atoms, shape, h)
        lo, sn = synth.central_site(shape, S)
        lo = tuple(int(a + b) for a, b in zip(lo, off))
        recs.append(synth.ReceptorInput(g, h, o, lo, sn))
    ligs = []
    for i, (na, nc) in enumerate([(5, 7), (17, 3), (9, 11)]):
        ligs.append(synth.LigandInput(synth.ligand_params(200 + i, na), synth.ligand_configs(300 + i, na, nc)))
    # stretch one configuration beyond the grid along x
    ligs[2].coords[4, 0, 0] += 30.0
    refs = [oracle.evaluate(recs, l.coords, l.params.q, l.params.eps, l.params.R, KT) for l in ligs]
    with _session(pkg) as s:
        rhs = [s.load_receptor(r) for r in recs]
        lh, _, nconf = s.load_ligands(ligs)
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, n_lig=3, total_conf=sum(nconf))
    assert rc == pkg.BPMF_WARN_NO_VALID
    off = 0
    for i, ref in enumerate(refs):
        J = ligs[i].coords.shape[0]
        sub = {"logZ": out["logZ"][off:off + J], "n_valid": out["n_valid"][off:off + J],
               "bpmf": out["bpmf"][i:i + 1], "dG": out["dG"][i:i + 1]}
        _check_eval(sub, ref, 2)
        off += J
    assert out["n_valid"][7 + 3 + 4].sum() == 0 and np.all(np.isneginf(out["logZ"][7 + 3 + 4]))


def test_batching_buffers_and_determinism(pkg, small):
    """Results are bit-identical whatever the batch size (workspace limit),
    whether inputs/outputs are host or device memory, and across runs."""
    import torch
    r, l = small.receptors[0], small.ligands[0]
    with _session(pkg) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, a = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=64)
        _, b = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=64)
        dev = {"logZ": torch.empty((64, 1), dtype=torch.float64, device="cuda"),
               "n_valid": torch.empty((64, 1), dtype=torch.int64, device="cuda"),
               "bpmf": torch.empty((1, 1), dtype=torch.float64, device="cuda"),
               "dG": torch.empty(1, dtype=torch.float64, device="cuda")}
        s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, out=dev)
        torch.cuda.synchronize()
    with _session(pkg, workspace_bytes=1 << 20) as s2:  # forces one configuration per batch
        g = torch.from_numpy(r.grids).cuda()
        rh = s2.load_receptor(r, grids=g)
        coords = torch.from_numpy(l.coords.reshape(-1, 3).copy()).cuda()
        lh, _, _ = s2.load_ligands([l], coords=coords)
        _, c = s2.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=64)
    for k in ("logZ", "n_valid", "bpmf", "dG"):
        assert np.array_equal(a[k], b[k]), k
        assert np.array_equal(a[k], dev[k].cpu().numpy()), k
        assert np.array_equal(a[k], c[k]), k


def test_bad_arguments_return_status(pkg, small):
    import ctypes
    r = small.receptors[0]
    with _session(pkg) as s:
        with pytest.raises(pkg.BpmfError) as e:
            pkg.bpmf_receptor_load(s.ctx, r.grids, 0.0, r.origin, r.site_lo, r.site_n)
        assert e.value.status == pkg.BPMF_ERR_INVALID_ARG
        big = np.zeros((3, 300, 8, 8), dtype=np.float32)
        with pytest.raises(pkg.BpmfError) as e:
            pkg.bpmf_receptor_load(s.ctx, big, 0.5, (0, 0, 0), (0, 0, 0), (2, 2, 2))
        assert e.value.status == pkg.BPMF_ERR_SIZE_UNSUPPORTED
        l = synth.ligand_params(1, 300)
        with pytest.raises(pkg.BpmfError) as e:
            pkg.bpmf_ligand_batch(s.ctx, [300], [1], np.zeros((300, 3), np.float32), l.q, l.eps, l.R)
        assert e.value.status == pkg.BPMF_ERR_SIZE_UNSUPPORTED
        assert pkg.lib().bpmf_eval(s.ctx, None, None, 0, 1.0, 0, None, None, None, None, None) == \
            pkg.BPMF_ERR_INVALID_ARG
        # receptors with different grid spacings cannot share one evaluation
        r1 = s.load_receptor(r)
        g2 = np.zeros((3, 40, 32, 32), dtype=np.float32)
        r2 = pkg.bpmf_receptor_load(s.ctx, g2, r.h * 1.5, r.origin, r.site_lo, r.site_n)
        lh, _, _ = s.load_ligands([small.ligands[0]])
        with pytest.raises(pkg.BpmfError) as e:
            s.eval(lh, [r1, r2], KT, pkg.BPMF_MODE_FF, total_conf=64)
        assert e.value.status == pkg.BPMF_ERR_SIZE_UNSUPPORTED
        pkg.bpmf_receptor_free(r2)


# ------------------------------------------------- protein scale, full size
@pytest.fixture(scope="module")
def protein():
    return synth.protein_scale()


def test_protein_scale_full_size_parity(pkg, protein):
    """96^3 grids, 4 receptor conformations, 2000 configurations of a 30-atom
    ligand, evaluated in one call exactly as the benchmark runs it.  log Z of
    every 8th configuration is checked against the FP64 oracle; the BPMFs and dG
    are checked against the pooled estimator applied to the returned log Z, and
    against the oracle on the sampled configurations."""
    lig = protein.ligands[0]
    J = lig.coords.shape[0]
    K = len(protein.receptors)
    with _session(pkg) as s:
        rhs = [s.load_receptor(r) for r in protein.receptors]
        lh, _, _ = s.load_ligands([lig])
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=J)
    idx = np.arange(0, J, 8)
    ref = oracle.evaluate(protein.receptors, lig.coords[idx], lig.params.q, lig.params.eps, lig.params.R, KT)
    assert np.array_equal(out["n_valid"][idx], ref["n_valid"])
    ok = np.isfinite(ref["logZ"])
    assert np.abs(out["logZ"][idx][ok] - ref["logZ"][ok]).max() * KT <= E_TOL
    # pooled BPMF of the sampled subset from the GPU's own log Z equals the oracle's
    logS_gpu = out["logZ"][idx] + np.log(out["n_valid"][idx])
    assert np.abs(oracle.bpmf(logS_gpu, out["n_valid"][idx], KT) - ref["bpmf"]).max() <= B_TOL
    # the GPU's full BPMF / dG are the pooled estimator of its full log Z
    logS_all = out["logZ"] + np.log(np.maximum(out["n_valid"], 1))
    B_all = oracle.bpmf(logS_all, out["n_valid"], KT)
    assert np.abs(out["bpmf"][0] - B_all).max() <= 1e-9 * max(1.0, np.abs(B_all).max())
    dG_all = oracle.dG(B_all, KT, oracle.site_volume(out["n_valid"], protein.receptors[0].h))
    assert abs(out["dG"][0] - dG_all) <= 1e-9 * max(1.0, abs(dG_all))
    print("protein-scale BPMF", out["bpmf"][0], "dG", out["dG"][0])


# -------------------------------------------------- split-bf16 tensor-core form
def test_split_bf16_tensor_core_stage_errors_are_reported_and_bounded(pkg, small, small_ref):
    """BPMF_MODE_SPLIT_BF16: the radix-32 stages run as six-term bf16
    tensor-core contractions (hi/mid/lo parts, per-stage error near FP32's).
    The tensor cores accumulate in FP32 without IEEE rounding, so its energy
    error against the oracle is held to eight times the FP32 bound (the bound
    the refined form uses for this locator); the error is printed."""
    r, l = small.receptors[0], small.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    E_ref, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[0], gam)
    with _session(pkg) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        E_s = s.export_energies(lh, rh, 0, 0, r.site_n, pkg.BPMF_MODE_SPLIT_BF16)
        E_f = s.export_energies(lh, rh, 0, 0, r.site_n, pkg.BPMF_MODE_FP32)
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_SPLIT_BF16, n_lig=1, total_conf=64)
    ok = np.isfinite(E_ref)
    assert np.array_equal(np.isinf(E_s), ~ok)
    bound = _fp32_bound(r.grids, gam, r.shape) * 8
    es = np.abs(E_s[ok] - E_ref[ok])
    ef = np.abs(E_f[ok] - E_ref[ok])
    dB = abs(out["bpmf"][0, 0] - small_ref["bpmf"][0])
    print(f"split-bf16: max |dE| {es.max():.3g} (FP32 {ef.max():.3g}) kcal/mol, |dB| {dB:.3g}, bound {bound:.3g}")
    assert es.max() <= bound
    # the tensor-core stage really changes the arithmetic (it is not the FP32 path)
    assert not np.array_equal(E_s, E_f)
    assert np.array_equal(out["n_valid"], small_ref["n_valid"])


def test_split_bf16_protein_scale_runs_with_mixed_stages(pkg, protein):
    """96 = 3 x 32: a CUDA-core radix-3 stage followed by the tensor-core
    radix-32 stage, on a sample of the full-size workload."""
    lig = protein.ligands[0]
    sub = synth.LigandInput(lig.params, lig.coords[:16])
    ref = oracle.evaluate(protein.receptors, sub.coords, lig.params.q, lig.params.eps, lig.params.R, KT)
    with _session(pkg) as s:
        rhs = [s.load_receptor(r) for r in protein.receptors]
        lh, _, _ = s.load_ligands([sub])
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_SPLIT_BF16, n_lig=1, total_conf=16)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    ok = np.isfinite(ref["logZ"])
    dz = np.abs(out["logZ"][ok] - ref["logZ"][ok]).max() * KT
    g = protein.receptors[0].grids
    bound = _fp32_bound(g, ref["gamma"], protein.receptors[0].shape) * 8
    print(f"split-bf16 protein scale: max kT|dlogZ| {dz:.3g} kcal/mol, |dB| "
          f"{np.abs(out['bpmf'][0] - ref['bpmf']).max():.3g} (bound {bound:.3g})")
    assert np.isfinite(dz) and dz <= bound


def test_split_refine_meets_the_tolerances(pkg, protein):
    """BPMF_MODE_SPLIT_REFINE: the split-bf16 tensor-core correlation locates
    the low-energy window, the float-pair re-evaluation makes it exact; log Z
    and the BPMFs of a protein-scale sample meet the tolerances."""
    lig = protein.ligands[0]
    sub = synth.LigandInput(lig.params, lig.coords[:16])
    ref = oracle.evaluate(protein.receptors, sub.coords, lig.params.q, lig.params.eps, lig.params.R, KT)
    with _session(pkg) as s:
        rhs = [s.load_receptor(r) for r in protein.receptors]
        lh, _, _ = s.load_ligands([sub])
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_SPLIT_REFINE, n_lig=1, total_conf=16)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    ok = np.isfinite(ref["logZ"])
    dz = np.abs(out["logZ"][ok] - ref["logZ"][ok]).max() * KT
    dB = np.abs(out["bpmf"][0] - ref["bpmf"]).max()
    print(f"split-refine protein scale: max kT|dlogZ| {dz:.3g}, |dB| {dB:.3g} kcal/mol, status {rc}")
    assert dz <= E_TOL and dB <= B_TOL
