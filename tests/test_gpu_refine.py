"""The refined form (BPMF_MODE_REFINE: FP32 correlation, exact float-pair
re-evaluation of every translation that can carry weight, checked against a
certificate) against the FP64 oracle, through the C ABI.

Inside the 20 kT window the energies are the exact direct sum in float pairs,
so they match the oracle to about 2^-44 of the terms (1e-9 of the grid scale
is the bound used here).  log Z, BPMF and dG
must meet the benchmark spec's tolerances (1e-3 and 0.01 kcal/mol); the excluded
translations weigh less than 1e-5 of S by construction, so the measured error
is far below."""
import numpy as np
import pytest

import oracle
from oracle import sampling as S
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


def _session():
    from paper_1708_07045_gb300.session import Session
    return Session(0)


def _scale(r, gam):
    return sum(np.abs(r.grids[t]).max() * np.abs(gam[t]).sum() for t in range(3))


@pytest.mark.parametrize("conf", [0, 7, 30])
def test_refined_energies_exact_in_window(pkg, conf):
    w = synth.plain_small(n_conf=32)
    r, l = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    E_ref, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[conf], gam)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        E = s.export_energies(lh, rh, 0, conf, r.site_n, pkg.BPMF_MODE_REFINE)
    assert np.array_equal(np.isinf(E), np.isinf(E_ref))
    ok = np.isfinite(E_ref)
    win = ok & (E_ref <= E_ref[ok].min() + 20 * KT)
    assert np.abs(E[win] - E_ref[win]).max() <= 1e-9 * _scale(r, gam)


def test_refined_eval_protein_scale_sample(pkg):
    w = synth.protein_scale(n_conf=8, n_rec=4)
    l = w.ligands[0]
    ref = oracle.evaluate(w.receptors, l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=8)
        pmin = np.empty((8, 4))
        pdom = np.empty((1, 6))
        pkg.bpmf_eval_dominant(s.ctx, lh, rhs, KT, pkg.BPMF_MODE_REFINE, np.empty((8, 4)), None, None, None, pmin,
                               pdom)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    fin = np.isfinite(ref["logZ"])
    assert np.array_equal(np.isfinite(out["logZ"]), fin)
    assert np.abs(out["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL
    assert np.abs(out["bpmf"][0] - ref["bpmf"]).max() <= B_TOL
    assert abs(out["dG"][0] - ref["dG"]) <= B_TOL
    # the minimum is a refined energy: exact
    assert np.abs(pmin - ref["Emin"]).max() <= 1e-9 * np.abs(ref["Emin"]).max()
    assert np.abs(pdom[0] - S.dominant(ref["Emin"], KT)).max() <= 1e-6


def test_refined_eval_with_clashes(pkg):
    w = synth.plain_small_occ(n_conf=32)
    r, l = w.receptors[0], w.ligands[0]
    ref = oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=32)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    fin = np.isfinite(ref["logZ"])
    assert np.array_equal(np.isfinite(out["logZ"]), fin) and fin.any()
    assert np.abs(out["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL
    assert abs(out["bpmf"][0, 0] - ref["bpmf"][0]) <= B_TOL


def test_refined_eval_whole_surface_window(pkg):
    w = synth.whole_surface(n_conf=2)
    r0, l = w.receptors[0], w.ligands[0]
    lo, sn = synth.central_site(r0.shape, 64)
    r = synth.ReceptorInput(r0.grids, r0.h, r0.origin, lo, sn)
    ref = oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=2)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    assert np.abs(out["logZ"] - ref["logZ"]).max() * KT <= E_TOL


def test_refined_matches_float_pairs_on_batches(pkg):
    """Uneven ligands and receptor groups in one call: the refined and the
    float-pair forms agree within the tolerance."""
    w = synth.batched_uneven(n_lig=3, n_conf=24, n_rec=3)
    with _session() as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, nconf = s.load_ligands(w.ligands)
        T = sum(nconf)
        _, a = s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, n_lig=3, total_conf=T)
        _, b = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=3, total_conf=T)
    assert np.array_equal(a["n_valid"], b["n_valid"])
    fin = np.isfinite(a["logZ"])
    assert np.array_equal(np.isfinite(b["logZ"]), fin)
    assert np.abs(a["logZ"][fin] - b["logZ"][fin]).max() * KT <= E_TOL
    okb = np.isfinite(a["bpmf"])
    assert np.abs(a["bpmf"][okb] - b["bpmf"][okb]).max() <= B_TOL


def test_refined_protein_scale_full_size_on_cropped_transforms(pkg):
    """All 2000 configurations of the protein-scale workload in one call, as the
    benchmark runs it.  Enough configurations share each receptor crop that the
    transforms run on cropped grids (checked through the launch profile: the
    crops are made and the x pass runs); log Z of every 16th configuration
    against the FP64 oracle, and the BPMFs of that sample."""
    w = synth.protein_scale()
    lig = w.ligands[0]
    J, K = lig.coords.shape[0], len(w.receptors)
    with _session() as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, _ = s.load_ligands([lig])
        pkg.bpmf_profile_enable(s.ctx, True)
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=J)
        prof = pkg.bpmf_profile(s.ctx)
        pkg.bpmf_profile_enable(s.ctx, False)
    assert prof.get("k_crop", (0.0, 0))[1] > 0, sorted(prof)
    assert not (rc & pkg.BPMF_WARN_REFINE_FALLBACK), "the certificate held on the benchmark workload"
    idx = np.arange(0, J, 16)
    ref = oracle.evaluate(w.receptors, lig.coords[idx], lig.params.q, lig.params.eps, lig.params.R, KT)
    assert np.array_equal(out["n_valid"][idx], ref["n_valid"])
    ok = np.isfinite(ref["logZ"])
    assert np.abs(out["logZ"][idx][ok] - ref["logZ"][ok]).max() * KT <= E_TOL
    logS = out["logZ"][idx] + np.log(out["n_valid"][idx])
    assert np.abs(oracle.bpmf(logS, out["n_valid"][idx], KT) - ref["bpmf"]).max() <= B_TOL


def test_refined_certificate_failure_falls_back_to_float_pairs(pkg):
    """With the certificate's bound scaled to zero every re-evaluated
    translation fails the check: the call recomputes the ligand in float pairs,
    says so in its status, and its results are those of the float-pair form
    (bit for bit) and within the tolerances of the oracle."""
    w = synth.plain_small(n_conf=16)
    r, l = w.receptors[0], w.ligands[0]
    ref = oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        rc0, base = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=16)
        assert not (rc0 & pkg.BPMF_WARN_REFINE_FALLBACK)
        _, ff = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=16)
        pkg.bpmf_set_refine_check_scale(s.ctx, 0.0)
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=16)
        E = s.export_energies(lh, rh, 0, 3, r.site_n, pkg.BPMF_MODE_REFINE)
        E_ff = s.export_energies(lh, rh, 0, 3, r.site_n, pkg.BPMF_MODE_FF)
        pkg.bpmf_set_refine_check_scale(s.ctx, 1.0)
    assert rc & pkg.BPMF_WARN_REFINE_FALLBACK
    for k in ("logZ", "n_valid", "bpmf", "dG"):
        assert np.array_equal(out[k], ff[k]), k
    assert np.array_equal(E, E_ff)
    fin = np.isfinite(ref["logZ"])
    assert np.abs(out["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL
    assert abs(out["bpmf"][0, 0] - ref["bpmf"][0]) <= B_TOL
    assert np.abs(base["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL


def test_refined_results_are_deterministic_with_and_without_graphs(pkg):
    """Repeated calls and a CUDA-graph replay give bit-identical results: the
    set of re-evaluated translations depends only on the final minimum, not
    on the order in which the planes ran, and their weights are summed in
    order-independent fixed point."""
    import torch
    w = synth.protein_scale(n_conf=48, n_rec=2)
    lig = w.ligands[0]
    J, K = 48, 2
    with _session() as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, _ = s.load_ligands([lig])
        _, a = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=J)
        _, b = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=J)
        st = torch.cuda.Stream()
        dev = {"logZ": torch.empty((J, K), dtype=torch.float64, device="cuda"),
               "n_valid": torch.empty((J, K), dtype=torch.int64, device="cuda"),
               "bpmf": torch.empty((1, K), dtype=torch.float64, device="cuda"),
               "dG": torch.empty(1, dtype=torch.float64, device="cuda")}
        pkg.bpmf_set_graph_mode(s.ctx, 1)
        for _ in range(2):  # capture, then replay
            s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, out=dev, stream=st.cuda_stream)
            torch.cuda.synchronize()
            assert np.array_equal(dev["n_valid"].cpu().numpy(), a["n_valid"])
            for k in ("logZ", "bpmf", "dG"):
                assert np.array_equal(dev[k].cpu().numpy(), a[k]), k
        pkg.bpmf_set_graph_mode(s.ctx, 0)
    assert np.array_equal(a["n_valid"], b["n_valid"])
    for k in ("logZ", "bpmf", "dG"):
        assert np.array_equal(a[k], b[k]), k


def test_refined_list_overflow_reruns_from_first_pass_minima(pkg):
    """Candidate lists capped at one translation overflow on every pair that
    lists two (every plane lists its own minimum when it runs before the
    pair's lower planes): the call evaluates the ligand again in the refined
    form (lists of the default size, each pair's running minimum starting at
    the first pass's), so the results are the refined form's (no float-pair
    fallback, no warning bit) and bpmf_last_error says what happened.  With
    the certificate also forced to fail, the ligand falls back to float
    pairs, bit for bit."""
    w = synth.plain_small(n_conf=16)
    r, l = w.receptors[0], w.ligands[0]
    ref = oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, base = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=16)
        assert pkg.bpmf_last_error(s.ctx) == ""
        _, ff = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=16)
        pkg.bpmf_set_refine_list_cap(s.ctx, 1)
        rc, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=16)
        note = pkg.bpmf_last_error(s.ctx)
        pkg.bpmf_set_refine_check_scale(s.ctx, 0.0)
        rc2, out2 = s.eval(lh, [rh], KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=16)
        note2 = pkg.bpmf_last_error(s.ctx)
        pkg.bpmf_set_refine_check_scale(s.ctx, 1.0)
        pkg.bpmf_set_refine_list_cap(s.ctx, 0)
    assert not (rc & pkg.BPMF_WARN_REFINE_FALLBACK)
    assert "1 ligand(s) re-run from the first pass's minima" in note, note
    assert np.array_equal(out["n_valid"], base["n_valid"])
    for k in ("logZ", "bpmf", "dG"):
        assert np.allclose(out[k], base[k], rtol=1e-11, atol=0), k
    fin = np.isfinite(ref["logZ"])
    assert np.abs(out["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL
    assert abs(out["bpmf"][0, 0] - ref["bpmf"][0]) <= B_TOL
    assert rc2 & pkg.BPMF_WARN_REFINE_FALLBACK
    assert "recomputed in float pairs (certificate failed: 1" in note2, note2
    for k in ("logZ", "n_valid", "bpmf", "dG"):
        assert np.array_equal(out2[k], ff[k]), k
