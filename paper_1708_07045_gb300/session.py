"""Convenience wrapper over the C names: owns a context and the handles it
creates, and allocates outputs.  Argument marshalling only; every step of the
hot path runs in libbpmf.so."""
from __future__ import annotations

import numpy as np

from . import (BPMF_MODE_FF, bpmf_create, bpmf_destroy, bpmf_eval, bpmf_export_energies, bpmf_ligand_batch,
               bpmf_ligand_free, bpmf_receptor_free, bpmf_receptor_load, bpmf_receptor_set_occupancy,
               bpmf_set_workspace_limit)


class Session:
    """One device context.  ``receptors`` are objects with ``grids`` [3,nx,ny,nz]
    float32, ``h``, ``origin``, ``site_lo``, ``site_n``; ligands have ``params``
    (``q``, ``eps``, ``R`` float32 [n_atoms]) and ``coords`` float32
    [n_conf, n_atoms, 3]."""

    def __init__(self, device: int = 0, workspace_bytes: int | None = None):
        self.device = device
        self.ctx = bpmf_create(device)
        self._recs, self._ligs = [], []
        if workspace_bytes is not None:
            bpmf_set_workspace_limit(self.ctx, workspace_bytes)

    # ---------------------------------------------------------------- inputs
    def load_receptor(self, r, grids=None, stream=None):
        h = bpmf_receptor_load(self.ctx, r.grids if grids is None else grids, r.h, r.origin, r.site_lo,
                               r.site_n, stream)
        self._recs.append(h)
        if getattr(r, "occ", None) is not None:
            bpmf_receptor_set_occupancy(self.ctx, h, r.occ, stream)
        return h

    def load_ligands(self, ligands, p_rep=12, p_att=6, coords=None, params=None, stream=None):
        """``coords`` / ``params`` override the concatenated host arrays (e.g.
        with device tensors of the same layout)."""
        n_atoms = [l.params.n_atoms for l in ligands]
        n_conf = [l.coords.shape[0] for l in ligands]
        if coords is None:
            coords = np.ascontiguousarray(np.concatenate([l.coords.reshape(-1, 3) for l in ligands]),
                                          dtype=np.float32)
        if params is None:
            params = [np.ascontiguousarray(np.concatenate([getattr(l.params, k) for l in ligands]),
                                           dtype=np.float32) for k in ("q", "eps", "R")]
        h = bpmf_ligand_batch(self.ctx, n_atoms, n_conf, coords, *params, p_rep=p_rep, p_att=p_att,
                              stream=stream)
        self._ligs.append(h)
        return h, n_atoms, n_conf

    # ------------------------------------------------------------------ eval
    def eval(self, lig, recs, kT, mode=BPMF_MODE_FF, n_lig=1, total_conf=None, stream=None, out=None):
        """Returns (status, dict of numpy outputs).  ``out`` may supply the four
        caller-owned output buffers (numpy or torch)."""
        K = len(recs)
        if out is None:
            out = {"logZ": np.empty((total_conf, K)), "n_valid": np.empty((total_conf, K), dtype=np.int64),
                   "bpmf": np.empty((n_lig, K)), "dG": np.empty(n_lig)}
        rc = bpmf_eval(self.ctx, lig, recs, kT, mode, out["logZ"], out["n_valid"], out["bpmf"], out["dG"],
                       stream)
        return rc, out

    def export_energies(self, lig, rec, lig_index, conf_index, site_n, mode=BPMF_MODE_FF):
        out = np.empty(tuple(int(s) for s in site_n))
        bpmf_export_energies(self.ctx, lig, rec, lig_index, conf_index, mode, out)
        return out

    def close(self):
        for h in self._ligs:
            bpmf_ligand_free(h)
        for h in self._recs:
            bpmf_receptor_free(h)
        self._ligs, self._recs = [], []
        if self.ctx is not None:
            bpmf_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
