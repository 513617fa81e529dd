"""FP64 reference for the dominant-state quantities and pose resampling.

TEST INFRASTRUCTURE ONLY (imported by the tests and the benchmark's CPU
legs, never by the product library).

* ``dominant``  -- the dominant-state approximation (Section "Dominant state
  approximation" of the results): the minimum interaction energy of every
  receptor snapshot in place of the exponential average, combined over
  snapshots by the minimum and by an exponential average.
* ``sir_configs`` / ``sir_translations`` -- sampling importance resampling of
  poses with weight exp(-Psi/kT) (Section "Implicit solvent": poses of the
  bound state resampled before the single-step perturbation), by inverse CDF
  on given uniforms: index = first i whose cumulative weight exceeds
  u * total.  The draw over (configuration, translation) is split exactly into
  configuration j with probability S_j / sum S (S_j = sum over j's valid
  translations of exp(-Psi/kT)) and then translation t with probability
  exp(-Psi_t/kT) / S_j.
"""
from __future__ import annotations

import numpy as np


def dominant(Emin, kT):
    """Emin [J, K] minimum energies per (configuration, receptor) (+inf where
    no translation is valid).  Returns [K + 2]: min_j Emin[j, k] per receptor,
    their minimum, and -kT ln((1/K) sum_k exp(-min_k / kT))."""
    Emin = np.asarray(Emin, dtype=np.float64)
    K = Emin.shape[1]
    per = Emin.min(axis=0) if Emin.shape[0] else np.full(K, np.inf)
    lo = per.min()
    if not np.isfinite(lo):
        return np.concatenate([per, [np.inf, np.inf]])
    ea = lo - kT * np.log(np.mean(np.exp(-(per - lo) / kT)))
    return np.concatenate([per, [lo, ea]])


def _inverse_cdf(w, u):
    """First index i with cumsum(w)[i] > u * sum(w), for every u."""
    c = np.cumsum(np.asarray(w, dtype=np.float64))
    total = c[-1] if c.size else 0.0
    if not total > 0:
        return np.full(np.shape(u), -1, dtype=np.int64)
    return np.searchsorted(c, np.asarray(u, dtype=np.float64) * total, side="right").clip(0, c.size - 1)


def config_weights(logS):
    """Normalised S_j / sum S from log S_j (-inf allowed)."""
    logS = np.asarray(logS, dtype=np.float64)
    m = logS.max() if logS.size else -np.inf
    if not np.isfinite(m):
        return np.zeros_like(logS)
    w = np.exp(logS - m)
    return w / w.sum()


def translation_weights(E, kT):
    """Normalised exp(-E/kT) over one configuration's translations (+inf
    energies have weight 0)."""
    E = np.asarray(E, dtype=np.float64).ravel()
    fin = np.isfinite(E)
    if not fin.any():
        return np.zeros_like(E)
    m = E[fin].min()
    w = np.where(fin, np.exp(-(np.where(fin, E, m) - m) / kT), 0.0)
    return w / w.sum()


def sir_configs(logS, u):
    """Configuration index per uniform (or -1 when every S_j is 0)."""
    return _inverse_cdf(config_weights(logS), u)


def sir_translations(E, kT, u):
    """Flattened translation index per uniform within one configuration."""
    return _inverse_cdf(translation_weights(E, kT), u)


def bootstrap(logS, n_valid, kT, h, u):
    """Bootstrap of the pooled BPMF and the standard binding free energy over
    configurations (results, the BPMF uncertainty: configurations resampled
    with replacement).  logS, n_valid [J, K]; u [R, J] uniforms: replicate r
    draws configuration min(J - 1, floor(u J)) for each of its J slots.
    Returns reps [R, K + 1] (B_k, then dG) and stats [2, K + 1] (mean and
    sample standard deviation, ddof 1, over replicates)."""
    from . import bpmf, dG, site_volume
    logS = np.asarray(logS, dtype=np.float64)
    n = np.asarray(n_valid, dtype=np.int64)
    J, K = logS.shape
    u = np.asarray(u, dtype=np.float64)
    R = u.shape[0]
    reps = np.empty((R, K + 1))
    for r in range(R):
        idx = np.minimum(J - 1, np.floor(u[r] * J).astype(np.int64))
        B = bpmf(logS[idx], n[idx], kT)
        reps[r, :K] = B
        vs = site_volume(n[idx], h)
        reps[r, K] = dG(B, kT, vs) if np.isfinite(B).any() and vs > 0 else np.inf
    stats = np.stack([reps.mean(axis=0), reps.std(axis=0, ddof=1) if R > 1 else np.zeros(K + 1)])
    return reps, stats
