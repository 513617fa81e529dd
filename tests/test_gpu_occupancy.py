"""The steric-clash channel (Eq. occupancy_grid) on the GPU against the FP64
oracle, through the C ABI.

The clash flags are integers: the set of +inf energies (filtered or
clashing translations) must equal the oracle's exactly, in every precision
mode.  Energies of the other translations, log Z, BPMF and dG keep the
tolerances of the plain path (1e-3 kcal/mol inside the 20 kT window, 0.01
kcal/mol for BPMF and dG)."""
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
    return synth.plain_small_occ(n_conf=48)


@pytest.fixture(scope="module")
def small_ref(small):
    r, l = small.receptors[0], small.ligands[0]
    return oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)


def _session():
    from paper_1708_07045_gb300.session import Session
    return Session(0)


def _check_energies(E, E_ref):
    assert np.array_equal(np.isinf(E), np.isinf(E_ref)), "clash / filter mask differs"
    ok = np.isfinite(E_ref)
    if ok.any():
        win = ok & (E_ref <= E_ref[ok].min() + 20 * KT)
        assert np.abs(E[win] - E_ref[win]).max() <= E_TOL


@pytest.mark.parametrize("conf", [0, 5, 17, 47])
def test_export_energies_with_clashes(pkg, small, conf):
    r, l = small.receptors[0], small.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    E_ref, n_ref = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[conf], gam, occ=r.occ,
                                        R=l.params.R)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        E = s.export_energies(lh, rh, 0, conf, r.site_n, pkg.BPMF_MODE_FF)
        E32 = s.export_energies(lh, rh, 0, conf, r.site_n, pkg.BPMF_MODE_FP32)
    _check_energies(E, E_ref)
    assert np.array_equal(np.isinf(E32), np.isinf(E_ref))


def test_eval_with_clashes_matches_oracle(pkg, small, small_ref):
    r, l = small.receptors[0], small.ligands[0]
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=48)
    ref = small_ref
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    fin = np.isfinite(ref["logZ"])
    assert np.array_equal(np.isfinite(out["logZ"]), fin)
    assert (~fin).any() and fin.any()  # both all-clash and partly free configurations
    assert np.abs(out["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL
    assert abs(out["bpmf"][0, 0] - ref["bpmf"][0]) <= B_TOL
    assert abs(out["dG"][0] - ref["dG"]) <= B_TOL


def test_empty_full_and_detached_occupancy(pkg, small):
    r, l = small.receptors[0], small.ligands[0]
    plain = synth.ReceptorInput(r.grids, r.h, r.origin, r.site_lo, r.site_n)
    zero = synth.ReceptorInput(r.grids, r.h, r.origin, r.site_lo, r.site_n, np.zeros_like(r.occ))
    full = synth.ReceptorInput(r.grids, r.h, r.origin, r.site_lo, r.site_n, np.ones_like(r.occ))
    with _session() as s:
        lh, _, _ = s.load_ligands([l])
        outs = {}
        for name, rec in (("plain", plain), ("zero", zero), ("full", full)):
            rh = s.load_receptor(rec)
            _, outs[name] = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=48)
        # detaching the grid restores the plain results
        pkg.bpmf_receptor_set_occupancy(s.ctx, rh, None)
        _, outs["detached"] = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=48)
    for k in ("logZ", "n_valid", "bpmf", "dG"):
        assert np.array_equal(outs["zero"][k], outs["plain"][k]), k
        assert np.array_equal(outs["detached"][k], outs["plain"][k]), k
    assert np.array_equal(outs["full"]["n_valid"], outs["plain"]["n_valid"])
    assert np.all(outs["full"]["logZ"] == -np.inf) and np.all(outs["full"]["bpmf"] == np.inf)


def test_graph_replay_and_batching_with_clashes(pkg, small):
    torch = pytest.importorskip("torch")
    r, l = small.receptors[0], small.ligands[0]
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, ref = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=48)
        pkg.bpmf_set_workspace_limit(s.ctx, 64 << 20)  # several batches
        _, small_ws = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=48)
        pkg.bpmf_set_graph_mode(s.ctx, True)
        st = torch.cuda.Stream()
        out = {k: torch.empty(v.shape, dtype=torch.from_numpy(v).dtype, device="cuda") for k, v in ref.items()}
        for _ in range(2):
            pkg.bpmf_eval(s.ctx, lh, [rh], KT, pkg.BPMF_MODE_FF, out["logZ"], out["n_valid"], out["bpmf"], out["dG"],
                          st)
        st.synchronize()
    for k in ref:
        assert np.array_equal(small_ws[k], ref[k]), k
        assert np.array_equal(out[k].cpu().numpy(), ref[k]), k


def test_protein_scale_occupancy_sampled_parity(pkg):
    """The pocket workload (96^3 at 0.25 A, 40^3 site, 30 atoms): exported
    energies of sampled configurations and log Z of a batch of eight, two
    receptor conformations."""
    w = synth.protein_scale_occ(n_conf=8, n_rec=2)
    l = w.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    ref = oracle.evaluate(w.receptors, l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=8)
        for k, j in ((0, 0), (1, 3)):
            r = w.receptors[k]
            E = s.export_energies(lh, rhs[k], 0, j, r.site_n, pkg.BPMF_MODE_FF)
            E_ref, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[j], gam, occ=r.occ,
                                            R=l.params.R)
            _check_energies(E, E_ref)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    fin = np.isfinite(ref["logZ"])
    assert np.array_equal(np.isfinite(out["logZ"]), fin) and fin.any()
    assert np.abs(out["logZ"][fin] - ref["logZ"][fin]).max() * KT <= E_TOL
    assert np.abs(out["bpmf"][0] - ref["bpmf"]).max() <= B_TOL


def test_fp32_form_on_cutoff_grids(pkg):
    """The cutoff grids of the clash treatment are bounded, so the plain FP32
    form's roundoff bound (8 eps sqrt(log2 P^3) rms(G_t) ||gamma_t||, summed
    over t) is small.  The mask must be exact; energies inside the 20 kT
    window stay under that bound (printed next to the 1e-3 tolerance)."""
    w = synth.protein_scale_occ(n_conf=3, n_rec=1)
    r, l = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    eps = 2.0 ** -24
    lg = np.sqrt(np.log2(96.0 ** 3))
    bound = sum(8 * eps * lg * np.sqrt(np.mean(r.grids[t].astype(np.float64) ** 2)) * np.linalg.norm(gam[t])
                for t in range(3))
    worst = 0.0
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        for j in range(3):
            E_ref, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[j], gam, occ=r.occ,
                                            R=l.params.R)
            E = s.export_energies(lh, rh, 0, j, r.site_n, pkg.BPMF_MODE_FP32)
            assert np.array_equal(np.isinf(E), np.isinf(E_ref))
            ok = np.isfinite(E_ref)
            if ok.any():
                win = ok & (E_ref <= E_ref[ok].min() + 20 * KT)
                worst = max(worst, float(np.abs(E[win] - E_ref[win]).max()))
    print(f"FP32 on cutoff grids: max |dE| in the 20 kT window {worst:.2e} kcal/mol, derived bound {bound:.2e}")
    assert worst <= bound
