"""Batched evaluation of uneven work: many ligands of uneven atom counts and
receptor conformations of uneven grid sizes in one bpmf_eval call (receptors
grouped by padded FFT edge), CUDA-graph replay, and the launch-shape
autotuner.  Parity against the FP64 oracle at the tolerances of
test_gpu_parity (energies 1e-3 kcal/mol via log Z, BPMF and dG 0.01)."""
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
def uneven():
    """A scaled-down batched workload: 5 ligands of 8-60 atoms, 24
    configurations each, 3 receptor conformations with grid edges drawn from
    64-112 and site edges from 24-40 (0.25 A spacing)."""
    return synth.batched_uneven(n_lig=5, n_conf=24, n_rec=3, seed=1002)


@pytest.fixture(scope="module")
def uneven_ref(uneven):
    return [oracle.evaluate(uneven.receptors, l.coords, l.params.q, l.params.eps, l.params.R, KT)
            for l in uneven.ligands]


def _eval(pkg, w, **kw):
    from paper_1708_07045_gb300.session import Session
    with Session(0) as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, nconf = s.load_ligands(w.ligands)
        rc, out = s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, n_lig=len(w.ligands), total_conf=sum(nconf))
    return rc, out


def _check(out, refs, w):
    off = 0
    for i, ref in enumerate(refs):
        J = w.ligands[i].coords.shape[0]
        nv = out["n_valid"][off:off + J]
        lz = out["logZ"][off:off + J]
        assert np.array_equal(nv, ref["n_valid"])
        ok = np.isfinite(ref["logZ"])
        assert np.array_equal(np.isfinite(lz), ok)
        if ok.any():
            assert np.abs(lz[ok] - ref["logZ"][ok]).max() * KT <= E_TOL
        fin = np.isfinite(ref["bpmf"])
        assert np.abs(out["bpmf"][i][fin] - ref["bpmf"][fin]).max() <= B_TOL
        if np.isfinite(ref["dG"]):
            assert abs(out["dG"][i] - ref["dG"]) <= B_TOL
        off += J


def test_uneven_receptor_sizes_and_ligands_in_one_call(pkg, uneven, uneven_ref):
    shapes = [r.shape for r in uneven.receptors]
    assert len({pkg.bpmf_fft_edge(s[0]) for s in shapes}) >= 2, shapes  # several receptor groups
    rc, out = _eval(pkg, uneven)
    assert rc in (pkg.BPMF_OK, pkg.BPMF_WARN_NO_VALID)
    _check(out, uneven_ref, uneven)


def test_graph_replay_and_autotune_are_bit_identical(pkg, uneven):
    import torch
    from paper_1708_07045_gb300.session import Session
    rc, ref = _eval(pkg, uneven)
    J = sum(l.coords.shape[0] for l in uneven.ligands)
    K = len(uneven.receptors)
    L = len(uneven.ligands)
    st = torch.cuda.Stream()
    with Session(0) as s:
        rhs = [s.load_receptor(r) for r in uneven.receptors]
        lh, _, _ = s.load_ligands(uneven.ligands)
        dev = {"logZ": torch.empty((J, K), dtype=torch.float64, device="cuda"),
               "n_valid": torch.empty((J, K), dtype=torch.int64, device="cuda"),
               "bpmf": torch.empty((L, K), dtype=torch.float64, device="cuda"),
               "dG": torch.empty(L, dtype=torch.float64, device="cuda")}
        pkg.bpmf_autotune(s.ctx, lh, rhs, pkg.BPMF_MODE_FF, st)
        pkg.bpmf_set_graph_mode(s.ctx, True)
        outs = []
        for _ in range(3):  # capture, then two replays
            for v in dev.values():
                v.zero_()
            torch.cuda.synchronize()
            s.eval(lh, rhs, KT, pkg.BPMF_MODE_FF, out=dev, stream=st)
            st.synchronize()
            outs.append({k: v.cpu().numpy() for k, v in dev.items()})
    for o in outs:
        for k in ("logZ", "n_valid", "bpmf", "dG"):
            assert np.array_equal(o[k], ref[k]), k


def test_refined_form_on_uneven_batches_with_the_autotuned_x_plan(pkg, uneven, uneven_ref):
    """The refined form on the uneven workload (FP32 x edges rounded up to
    the compile-time x pass, several receptor groups and crops), before and
    after bpmf_autotune (which may switch a group's x transform back to the
    padded or crop edge): both meet the tolerances against the oracle, with no
    float-pair fallback."""
    import torch
    from paper_1708_07045_gb300.session import Session
    J = sum(l.coords.shape[0] for l in uneven.ligands)
    with Session(0) as s:
        rhs = [s.load_receptor(r) for r in uneven.receptors]
        lh, _, _ = s.load_ligands(uneven.ligands)
        rc0, out0 = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=len(uneven.ligands), total_conf=J)
        st = torch.cuda.Stream()
        pkg.bpmf_autotune(s.ctx, lh, rhs, pkg.BPMF_MODE_REFINE, st)
        rc1, out1 = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=len(uneven.ligands), total_conf=J)
    for rc, out in ((rc0, out0), (rc1, out1)):
        assert not (rc & pkg.BPMF_WARN_REFINE_FALLBACK)
        _check(out, uneven_ref, uneven)
