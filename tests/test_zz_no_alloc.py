"""The allocation-free energy export (bpmf_export_energies_static).

Some callers cannot allocate device memory: code that runs inside another
framework's pre-reserved memory pool, or a thread that must not call
cudaMalloc/cudaFree because they synchronise the device.  For them the library
offers one entry point whose scratch lives in a fixed, library-owned static
device array.  These tests call it through the C ABI and compare it with the
allocating entry point, bpmf_export_energies, on consecutive calls (the static
array is shared and keeps the previous call's contents).  This file is
collected last so that a stop-at-first-failure run has already run every other
test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

E_TOL = 1e-3  # kcal/mol, the energy tolerance of the parity tests


def test_static_export_matches_allocating_export_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    import paper_1708_07045_gb300 as pkg
    from paper_1708_07045_gb300.session import Session

    w = synth.plain_small(n_conf=3)
    r, l = w.receptors[0], w.ligands[0]
    with Session(0) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        ref = {j: s.export_energies(lh, rh, 0, j, r.site_n, pkg.BPMF_MODE_FF) for j in (0, 1)}

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    grids = torch.from_numpy(r.grids).to(dev)
    q, eps, R = (torch.from_numpy(getattr(l.params, k)).to(dev) for k in ("q", "eps", "R"))
    # consecutive calls, the last one repeating the first configuration after
    # the array holds another configuration's data
    for j in (0, 1, 0):
        coords = torch.from_numpy(np.ascontiguousarray(l.coords[j])).to(dev)
        out = torch.full(tuple(r.site_n), float("nan"), dtype=torch.float64, device=dev)
        rc = pkg.bpmf_export_energies_static(grids, r.h, r.site_lo, r.site_n, coords, q, eps, R,
                                             pkg.BPMF_MODE_FF, out)
        assert rc == pkg.BPMF_OK
        E = out.cpu().numpy()
        assert np.array_equal(np.isinf(E), np.isinf(ref[j])), "translation mask differs"
        ok = np.isfinite(ref[j])
        assert ok.any()
        assert np.abs(E[ok] - ref[j][ok]).max() <= E_TOL


def test_static_export_rejects_problems_larger_than_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    import paper_1708_07045_gb300 as pkg

    dev = torch.device("cuda", 0)
    big = torch.zeros((3, 120, 120, 120), dtype=torch.float32, device=dev)  # spectra + passes exceed 64 MiB
    lig = synth.ligand_params(5, 4)
    coords = torch.zeros((4, 3), dtype=torch.float32, device=dev)
    q, eps, R = (torch.from_numpy(getattr(lig, k)).to(dev) for k in ("q", "eps", "R"))
    out = torch.empty((4, 4, 4), dtype=torch.float64, device=dev)
    with pytest.raises(pkg.BpmfError) as e:
        pkg.bpmf_export_energies_static(big, 0.25, (50, 50, 50), (4, 4, 4), coords, q, eps, R, pkg.BPMF_MODE_FF, out)
    assert e.value.status == pkg.BPMF_ERR_SIZE_UNSUPPORTED
