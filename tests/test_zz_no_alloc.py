"""The allocation-free energy export (bpmf_export_energies_static).

Some callers cannot allocate device memory: code that runs inside another
framework's pre-reserved memory pool, or a thread that must not call
cudaMalloc/cudaFree because they synchronise the device.  For them the library
offers one entry point whose scratch lives in a fixed, library-owned static
device array.  These tests call it through the C ABI and compare it with the
allocating entry point, bpmf_export_energies, and with the FP64 oracle, on
consecutive calls (the static array is shared and keeps the previous call's
contents), in both arithmetic forms it offers and on a 96^3 grid with a ligand
box near 60 nodes per edge.  This file is collected last so that a
stop-at-first-failure run has already run every other test.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

KT = synth.KT
E_TOL = 1e-3  # kcal/mol, the energy tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    import paper_1708_07045_gb300 as pkg
    pkg.lib()
    torch.cuda.set_device(0)
    return torch, pkg, torch.device("cuda", 0)


def _fp32_bound(grids, gam, P):
    """FP32 FFT-correlation roundoff bound per energy (as the parity tests):
    sum_t 8 eps32 sqrt(log2 P^3) rms(G_t) ||gamma_t||_2."""
    lg = np.sqrt(np.log2(float(np.prod(P))))
    return sum(8 * 2.0 ** -24 * lg * np.sqrt(np.mean(grids[t].astype(np.float64) ** 2)) * np.linalg.norm(gam[t])
               for t in range(3))


def _static(env, r, l, j, mode):
    torch, pkg, dev = env
    grids = torch.from_numpy(r.grids).to(dev)
    q, eps, R = (torch.from_numpy(getattr(l.params, k)).to(dev) for k in ("q", "eps", "R"))
    coords = torch.from_numpy(np.ascontiguousarray(l.coords[j])).to(dev)
    out = torch.full(tuple(r.site_n), float("nan"), dtype=torch.float64, device=dev)
    rc = pkg.bpmf_export_energies_static(grids, r.h, r.site_lo, r.site_n, coords, q, eps, R, mode, out)
    assert rc == pkg.BPMF_OK
    return out.cpu().numpy()


def _allocating(env, r, l, confs, mode):
    _, pkg, _ = env
    from paper_1708_07045_gb300.session import Session
    with Session(0) as s:
        rh = s.load_receptor(r)
        lh, _, _ = s.load_ligands([l])
        return {j: s.export_energies(lh, rh, 0, j, r.site_n, mode) for j in confs}


def _check(E, ref, oracle_E, tol_ref, tol_oracle):
    assert np.array_equal(np.isinf(E), np.isinf(ref)), "translation mask differs from the allocating export"
    assert np.array_equal(np.isinf(E), np.isinf(oracle_E)), "translation mask differs from the oracle"
    ok = np.isfinite(oracle_E)
    assert ok.any()
    assert np.abs(E[ok] - ref[ok]).max() <= tol_ref
    # the oracle's tolerance binds the energies within 20 kT of the minimum
    win = ok & (oracle_E <= oracle_E[ok].min() + 20 * KT)
    assert np.abs(E[win] - oracle_E[win]).max() <= tol_oracle


@pytest.mark.parametrize("mode_name", ["FF", "FP32"])
def test_static_export_matches_allocating_export_on_consecutive_calls(env, mode_name):
    _, pkg, _ = env
    mode = getattr(pkg, "BPMF_MODE_" + mode_name)
    w = synth.plain_small(n_conf=3)
    r, l = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    ref = _allocating(env, r, l, (0, 1), mode)
    orc = {j: oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[j], gam)[0] for j in (0, 1)}
    if mode == pkg.BPMF_MODE_FF:
        tol_ref, tol_oracle = E_TOL, E_TOL
    else:  # both exports are FP32 correlations: each within the derived bound of the exact energies
        b = _fp32_bound(r.grids, gam, [pkg.bpmf_fft_edge(n) for n in r.shape])
        tol_ref, tol_oracle = 2 * b, b
    # consecutive calls, the last one repeating the first configuration after
    # the array holds another configuration's data
    for j in (0, 1, 0):
        _check(_static(env, r, l, j, mode), ref[j], orc[j], tol_ref, tol_oracle)


@pytest.mark.parametrize("mode_name", ["FF", "FP32"])
def test_static_export_protein_scale_grid_and_large_ligand_box(env, mode_name):
    """A 96^3 grid (the protein-scale receptor) and the configuration whose
    ligand box is the largest of the first 120 (about 53 x 64 x 61 nodes): the
    receptor spectra, the receptor temporaries and the ligand buffers that
    overlay them all fit in the static array."""
    _, pkg, _ = env
    mode = getattr(pkg, "BPMF_MODE_" + mode_name)
    w = synth.protein_scale(n_conf=120, n_rec=1)
    r, l = w.receptors[0], w.ligands[0]
    boxes = np.array([np.prod(oracle.place(l.coords[j], r.h)[1]) for j in range(120)])
    jb = int(np.argmax(boxes))
    assert boxes[jb] ** (1 / 3) > 55
    gam = oracle.gamma(l.params.q, l.params.eps, l.params.R)
    ref = _allocating(env, r, l, (0, jb), mode)
    orc = {j: oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, l.coords[j], gam)[0] for j in (0, jb)}
    if mode == pkg.BPMF_MODE_FF:
        tol_ref, tol_oracle = E_TOL, E_TOL
    else:
        b = _fp32_bound(r.grids, gam, [pkg.bpmf_fft_edge(n) for n in r.shape])
        tol_ref, tol_oracle = 2 * b, b
    for j in (jb, 0, jb):
        _check(_static(env, r, l, j, mode), ref[j], orc[j], tol_ref, tol_oracle)


def test_static_export_rejects_host_memory_before_any_work(env):
    """The entry point hands its arrays straight to kernels, so host arrays
    are rejected with INVALID_ARG, and the output stays untouched."""
    torch, pkg, dev = env
    w = synth.plain_small(n_conf=1)
    r, l = w.receptors[0], w.ligands[0]
    q, eps, R = (torch.from_numpy(getattr(l.params, k)).to(dev) for k in ("q", "eps", "R"))
    coords = torch.from_numpy(np.ascontiguousarray(l.coords[0])).to(dev)
    out = torch.full(tuple(r.site_n), 7.0, dtype=torch.float64, device=dev)
    host_grids = np.ascontiguousarray(r.grids)
    with pytest.raises(pkg.BpmfError) as e:
        pkg.bpmf_export_energies_static(host_grids, r.h, r.site_lo, r.site_n, coords, q, eps, R,
                                        pkg.BPMF_MODE_FF, out)
    assert e.value.status == pkg.BPMF_ERR_INVALID_ARG
    host_out = np.full(tuple(r.site_n), 7.0)
    with pytest.raises(pkg.BpmfError) as e:
        pkg.bpmf_export_energies_static(torch.from_numpy(r.grids).to(dev), r.h, r.site_lo, r.site_n, coords, q,
                                        eps, R, pkg.BPMF_MODE_FF, host_out)
    assert e.value.status == pkg.BPMF_ERR_INVALID_ARG
    assert np.all(host_out == 7.0)
    assert bool((out == 7.0).all())


def test_static_export_rejects_problems_larger_than_its_scratch(env):
    torch, pkg, dev = env
    big = torch.zeros((3, 120, 120, 120), dtype=torch.float32, device=dev)  # spectra + passes exceed 64 MiB
    lig = synth.ligand_params(5, 4)
    coords = torch.zeros((4, 3), dtype=torch.float32, device=dev)
    q, eps, R = (torch.from_numpy(getattr(lig, k)).to(dev) for k in ("q", "eps", "R"))
    out = torch.empty((4, 4, 4), dtype=torch.float64, device=dev)
    with pytest.raises(pkg.BpmfError) as e:
        pkg.bpmf_export_energies_static(big, 0.25, (50, 50, 50), (4, 4, 4), coords, q, eps, R, pkg.BPMF_MODE_FF, out)
    assert e.value.status == pkg.BPMF_ERR_SIZE_UNSUPPORTED
