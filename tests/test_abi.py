"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/bpmf.h declares (CPU only; no compute calls)."""
import ctypes
import os
import re

import pytest

import paper_1708_07045_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "bpmf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bpmf_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("bpmf_create", "bpmf_receptor_load", "bpmf_ligand_batch", "bpmf_eval", "bpmf_export_energies",
              "bpmf_receptor_free", "bpmf_ligand_free", "bpmf_destroy", "bpmf_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol():
    L = ctypes.CDLL(pkg.build())
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing
    assert set(_declared()) == set(pkg._SIGS), "python binding must wrap every C entry point"


def test_host_only_entry_points():
    # pure host functions: no device work
    assert pkg.bpmf_status_string(0) == "ok"
    assert "size" in pkg.bpmf_status_string(pkg.BPMF_ERR_SIZE_UNSUPPORTED)
    assert pkg.bpmf_fft_edge(32) == 32
    assert pkg.bpmf_fft_edge(96) == 96
    assert pkg.bpmf_fft_edge(97) == 98      # 2 * 7^2

    def smooth_even(p):
        if p % 2:
            return False
        for r in (2, 3, 5, 7):
            while p % r == 0:
                p //= r
        return p == 1

    for n in range(2, 257):
        p = pkg.bpmf_fft_edge(n)
        assert p >= n and smooth_even(p)
        assert not any(smooth_even(v) for v in range(n, p))
    assert pkg.bpmf_fft_edge(257) == 0


def test_python_binding_rejects_wrong_dtypes():
    import numpy as np
    with pytest.raises(TypeError):
        pkg._ptr(np.zeros(3, dtype=np.float64), np.float32)
    with pytest.raises(TypeError):
        pkg._ptr(np.zeros((3, 3), dtype=np.float32).T, np.float32)


def test_crop_window_holds_every_node_a_kept_translation_reads():
    """Cropped transforms (bpmf_eval): along one axis, with the ligand box of
    edge u placed at w0 = site_lo - floor(u/2) and translation w0 + s kept for
    s in [max(0, -w0), min(site_n - 1, n - 1 - u - w0)] (the site window and
    the rule that the box stays inside the grid), every receptor node a kept
    translation reads, w0 + s + x for x in [0, u), must lie in the crop
    [c0, c0 + edge) and in the grid; and the ligand box (its y extent rounded
    up to even) must fit the edge.  Exhaustive over small grids."""
    checked = 0
    for n in range(8, 49):
        P = pkg.bpmf_fft_edge(n)
        for site_n in range(1, n + 1, 3):
            for site_lo in range(0, n - site_n + 1, 2):
                for u in range(5, n + 2):
                    edge, c0 = pkg.bpmf_crop_window(n, site_lo, site_n, u)
                    assert edge == P or edge < P
                    assert edge % 2 == 0 and pkg.bpmf_fft_edge(edge) == edge
                    w0 = site_lo - u // 2
                    sa, sb = max(0, -w0), min(site_n - 1, n - 1 - u - w0)
                    if sb < sa:
                        continue
                    lo, hi = w0 + sa, w0 + sb + u - 1
                    assert 0 <= lo and hi <= n - 1
                    assert c0 <= lo and hi <= c0 + edge - 1, (n, site_lo, site_n, u, edge, c0)
                    if edge < P:
                        assert c0 + edge <= n or c0 == 0
                        assert u + (u & 1) <= edge
                    checked += 1
    assert checked > 10000
    # the protein-scale axis: a 40-node site in a 96-node grid crops to 80
    # for ligand boxes up to 41 nodes
    assert pkg.bpmf_crop_window(96, 28, 40, 41) == (80, 8)
    assert pkg.bpmf_crop_window(96, 28, 40, 42)[0] == 96
    with pytest.raises(pkg.BpmfError):
        pkg.bpmf_crop_window(96, 28, 0, 10)
