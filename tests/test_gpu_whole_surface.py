"""The paper's larger grid (62 A at 0.25 A: 248^3 nodes, padded to a 250
edge, radix 5 and 2) against the FP64 oracle, through the C ABI: exported
energies and log Z on a 48^3 site window, and log Z of one configuration over
the full 200^3 surface window (8 million translations)."""
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
def surface():
    return synth.whole_surface(n_conf=3)


def _session():
    from paper_1708_07045_gb300.session import Session
    return Session(0)


def test_padded_edge(pkg):
    assert pkg.bpmf_fft_edge(248) == 250


def test_whole_surface_small_window(pkg, surface):
    r0, l = surface.receptors[0], surface.ligands[0]
    lo, sn = synth.central_site(r0.shape, 48)
    r = synth.ReceptorInput(r0.grids, r0.h, r0.origin, lo, sn)
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    ref = oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT)
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=3)
        E = s.export_energies(lh, rh, 0, 1, r.site_n, pkg.BPMF_MODE_FF)
    E_ref, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[1], gam)
    assert np.array_equal(np.isinf(E), np.isinf(E_ref))
    ok = np.isfinite(E_ref)
    win = ok & (E_ref <= E_ref[ok].min() + 20 * KT)
    assert np.abs(E[win] - E_ref[win]).max() <= E_TOL
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    assert np.abs(out["logZ"] - ref["logZ"]).max() * KT <= E_TOL
    assert abs(out["bpmf"][0, 0] - ref["bpmf"][0]) <= B_TOL


def test_whole_surface_full_window_one_configuration(pkg, surface):
    r, l = surface.receptors[0], surface.ligands[0]
    assert tuple(r.site_n) == (200, 200, 200)
    ref = oracle.evaluate([r], l.coords[:1], l.params.q, l.params.eps, l.params.R, KT)
    single = synth.LigandInput(l.params, l.coords[:1])
    with _session() as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([single])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, n_lig=1, total_conf=1)
    assert np.array_equal(out["n_valid"], ref["n_valid"])
    assert out["n_valid"][0, 0] > 5_000_000
    assert abs(out["logZ"][0, 0] - ref["logZ"][0, 0]) * KT <= E_TOL
