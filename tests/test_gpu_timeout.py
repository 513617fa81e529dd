"""The bounded waits of the CUDA path report a timeout instead of hanging.

With bpmf_set_wait_test on, the FP32 x pass does not request its first
receptor tile (its TMA copy), so every CTA's short bounded wait on the tile's
mbarrier runs out: the CTA sets the call's error flag and returns (nothing is
in flight, nothing faults).  The refined form synchronises its stream and
returns BPMF_ERR_TIMEOUT; the context stays usable, and the next call without
the setting gives the same results as before, bit for bit."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
KT = synth.KT


@pytest.fixture(scope="module")
def pkg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    import paper_1708_07045_gb300 as p
    p.lib()
    return p


def test_x_pass_wait_runs_out_and_context_stays_usable(pkg):
    from paper_1708_07045_gb300.session import Session
    w = synth.protein_scale(n_conf=8, n_rec=2)  # 96^3: the TMA-staged x pass on edge 96
    with Session(0) as s:
        rhs = [s.load_receptor(r) for r in w.receptors]
        lh, _, _ = s.load_ligands(w.ligands)
        _, before = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=8)
        pkg.bpmf_set_wait_test(s.ctx, 1)
        try:
            with pytest.raises(pkg.BpmfError) as err:
                s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=8)
        finally:
            pkg.bpmf_set_wait_test(s.ctx, 0)
        assert err.value.status == pkg.BPMF_ERR_TIMEOUT
        assert "bounded wait" in str(err.value)
        _, after = s.eval(lh, rhs, KT, pkg.BPMF_MODE_REFINE, n_lig=1, total_conf=8)
    for k in ("logZ", "n_valid", "bpmf", "dG"):
        assert np.array_equal(after[k], before[k]), k
