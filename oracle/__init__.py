"""FP64 CPU oracle for the FFT-correlation BPMF hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg import this package; the product
library never does, and this package imports nothing from the product.

Layers (each cites the passage it restates):

* ``gamma``            -- generalised ligand charges of Eq. general_form with the
                          per-term factors of Eqs. electrostatic, repulsive_LJ and
                          attractive_LJ (exponents p_rep / p_att of R).
* ``oracle.c``         -- placement, translation filter and direct per-pose
                          energies (Eqs. receptor_grid, correlation_func; the
                          ligand-box filter of "FFT-based BPMF Estimation"), and
                          log S_jk = log sum exp(-E/kT) over valid translations.
* ``bpmf`` / ``dG``    -- pooled sample-mean BPMF (Eq. sample_mean_BPMF) and the
                          standard binding free energy (Eqs. standard_binding_fe,
                          binding_FE_estimate) with uniform receptor weights.

Every function is pinned by ``tests/test_oracle_pins.py`` against brute-force
pairwise sums, closed forms, invariances and an independent FP64 FFT.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
from scipy.special import logsumexp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

C_STANDARD = 6.02214076e23 / 1e27  # 1 M standard state: N_A molecules per litre, in molecules per A^3


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc, FP64, OpenMP) in-tree."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            ip = ctypes.POINTER(ctypes.c_int)
            dp = ctypes.POINTER(ctypes.c_double)
            fp = ctypes.POINTER(ctypes.c_float)
            lp = ctypes.POINTER(ctypes.c_int64)
            lib.oracle_place.argtypes = [ctypes.c_int, fp, ctypes.c_double, dp, ip]
            lib.oracle_place.restype = ctypes.c_int
            bp = ctypes.POINTER(ctypes.c_ubyte)
            lib.oracle_pose_energies.argtypes = [fp, ip, ctypes.c_double, ip, ip, ctypes.c_int, fp, dp, fp, bp,
                                                 dp, lp]
            lib.oracle_pose_energies.restype = ctypes.c_int
            lib.oracle_logS_batch.argtypes = [fp, ip, ctypes.c_double, ip, ip, ctypes.c_int, ctypes.c_int,
                                              fp, dp, fp, bp, ctypes.c_double, dp, lp, dp]
            lib.oracle_ligand_occupancy.argtypes = [ctypes.c_int, fp, fp, ctypes.c_double, ip, ctypes.c_int]
            lib.oracle_ligand_occupancy.restype = ctypes.c_int
            lib.oracle_logS_batch.restype = ctypes.c_int
            lib.oracle_count_valid.argtypes = [ip, ip, ip, ip]
            lib.oracle_count_valid.restype = ctypes.c_int64
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _i3(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32).reshape(3))


def gamma(q, eps, R, p_rep: int = 12, p_att: int = 6) -> np.ndarray:
    """[3, n] FP64 generalised charges (q, sqrt(eps) R^p_rep, sqrt(eps) R^p_att)
    of the ligand atoms (Eq. general_form with the electrostatic, repulsive and
    attractive factors; the -2 of the attractive term lives in the receptor
    grid)."""
    q = np.asarray(q, dtype=np.float32).astype(np.float64)
    eps = np.asarray(eps, dtype=np.float32).astype(np.float64)
    R = np.asarray(R, dtype=np.float32).astype(np.float64)
    se = np.sqrt(eps)
    return np.ascontiguousarray(np.stack([q, se * R ** p_rep, se * R ** p_att]))


def place(coords, h: float):
    """(g [n,3] FP64 grid units, u [3] int) for one configuration."""
    c = np.ascontiguousarray(coords, dtype=np.float32)
    n = c.shape[0]
    g = np.empty((n, 3), dtype=np.float64)
    u = np.empty(3, dtype=np.int32)
    rc = _load().oracle_place(n, _p(c, ctypes.c_float), float(h), _p(g, ctypes.c_double), _p(u, ctypes.c_int))
    if rc != 0:
        raise ValueError("oracle_place: invalid arguments")
    return g, u


def count_valid(dims, u, site_lo, site_n) -> int:
    return int(_load().oracle_count_valid(_p(_i3(dims), ctypes.c_int), _p(_i3(u), ctypes.c_int),
                                          _p(_i3(site_lo), ctypes.c_int), _p(_i3(site_n), ctypes.c_int)))


def _occ_args(occ, R, shape):
    """(R pointer, occupancy pointer, keep-alive arrays) for the C calls."""
    if occ is None:
        return None, None, ()
    if R is None:
        raise ValueError("an occupancy grid needs the ligand R")
    o = np.ascontiguousarray(occ, dtype=np.uint8)
    if o.shape != tuple(shape):
        raise ValueError("occupancy grid shape differs from the grids")
    r = np.ascontiguousarray(R, dtype=np.float32)
    return _p(r, ctypes.c_float), _p(o, ctypes.c_ubyte), (o, r)


def ligand_occupancy(coords, R, h):
    """Occupied ligand-box nodes [count, 3] of one configuration (Eq.
    occupancy_grid, decided in single precision as documented in oracle.c)."""
    c = np.ascontiguousarray(coords, dtype=np.float32)
    r = np.ascontiguousarray(R, dtype=np.float32)
    lib = _load()
    n = lib.oracle_ligand_occupancy(c.shape[0], _p(c, ctypes.c_float), _p(r, ctypes.c_float), float(h), None, 0)
    if n < 0:
        raise ValueError("oracle_ligand_occupancy failed")
    out = np.empty((max(n, 1), 3), dtype=np.int32)
    lib.oracle_ligand_occupancy(c.shape[0], _p(c, ctypes.c_float), _p(r, ctypes.c_float), float(h),
                                _p(out, ctypes.c_int), n)
    return out[:n]


def pose_energies(grids, h, site_lo, site_n, coords, gam, occ=None, R=None):
    """FP64 energies [S0, S1, S2] of one configuration over the site window
    (+inf where the translation is filtered out or, with a receptor occupancy
    grid ``occ`` and the ligand's ``R``, clashes), and the valid count
    (clashing translations included)."""
    g = np.ascontiguousarray(grids, dtype=np.float32)
    c = np.ascontiguousarray(coords, dtype=np.float32)
    gm = np.ascontiguousarray(gam, dtype=np.float64)
    sn = _i3(site_n)
    E = np.empty(tuple(int(v) for v in sn), dtype=np.float64)
    n = np.zeros(1, dtype=np.int64)
    rp, op, _keep = _occ_args(occ, R, g.shape[1:])
    rc = _load().oracle_pose_energies(_p(g, ctypes.c_float), _p(_i3(g.shape[1:]), ctypes.c_int), float(h),
                                      _p(_i3(site_lo), ctypes.c_int), _p(sn, ctypes.c_int), c.shape[0],
                                      _p(c, ctypes.c_float), _p(gm, ctypes.c_double), rp, op,
                                      _p(E, ctypes.c_double), _p(n, ctypes.c_int64))
    if rc != 0:
        raise ValueError("oracle_pose_energies: invalid arguments")
    return E, int(n[0])


def logS_batch(grids, h, site_lo, site_n, coords, gam, kT, occ=None, R=None):
    """log S_jk, n_jk and min E_jk for every configuration j of ``coords``
    [J, n, 3] against one receptor (clashes as in ``pose_energies``)."""
    g = np.ascontiguousarray(grids, dtype=np.float32)
    c = np.ascontiguousarray(coords, dtype=np.float32)
    gm = np.ascontiguousarray(gam, dtype=np.float64)
    J, n = c.shape[0], c.shape[1]
    logS = np.empty(J, dtype=np.float64)
    nv = np.empty(J, dtype=np.int64)
    emin = np.empty(J, dtype=np.float64)
    rp, op, _keep = _occ_args(occ, R, g.shape[1:])
    rc = _load().oracle_logS_batch(_p(g, ctypes.c_float), _p(_i3(g.shape[1:]), ctypes.c_int), float(h),
                                   _p(_i3(site_lo), ctypes.c_int), _p(_i3(site_n), ctypes.c_int), J, n,
                                   _p(c, ctypes.c_float), _p(gm, ctypes.c_double), rp, op, float(kT),
                                   _p(logS, ctypes.c_double), _p(nv, ctypes.c_int64), _p(emin, ctypes.c_double))
    if rc != 0:
        raise ValueError("oracle_logS_batch: invalid arguments")
    return logS, nv, emin


def bpmf(logS, n_valid, kT):
    """Pooled sample-mean BPMF per receptor (Eq. sample_mean_BPMF over every
    valid sampled pose): logS, n_valid are [J, K]; returns B [K]
    (+inf when no pose is valid)."""
    logS = np.asarray(logS, dtype=np.float64)
    n = np.asarray(n_valid, dtype=np.float64)
    tot = n.sum(axis=0)
    with np.errstate(divide="ignore", invalid="ignore"):
        out = -kT * (logsumexp(logS, axis=0) - np.log(tot))
    return np.where(tot > 0, out, np.inf)


def log_z(logS, n_valid):
    """Per-configuration log Z_jk = log S_jk - ln n_jk (-inf when n_jk = 0)."""
    n = np.asarray(n_valid, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return np.where(n > 0, np.asarray(logS, dtype=np.float64) - np.log(np.maximum(n, 1)), -np.inf)


def site_volume(n_valid, h):
    """V_site = h^3 times the mean number of valid translations (the average
    rectangular region where the ligand box stays inside the grid)."""
    return float(h) ** 3 * float(np.mean(np.asarray(n_valid, dtype=np.float64)))


def dG(B, kT, v_site, weights=None):
    """Standard binding free energy from the receptor BPMFs (Eqs.
    standard_binding_fe / binding_FE_estimate with Omega / 8 pi^2 = V_site):
    dG = -kT ln sum_k W_k exp(-B_k / kT) - kT ln(V_site C)."""
    B = np.asarray(B, dtype=np.float64)
    W = np.full(B.shape, 1.0 / B.size) if weights is None else np.asarray(weights, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return float(-kT * logsumexp(-B / kT, b=W) - kT * np.log(v_site * C_STANDARD))


def evaluate(receptors, coords, q, eps, R, kT, p_rep: int = 12, p_att: int = 6):
    """Full oracle for one ligand: per-config log Z [J, K], n [J, K], logS,
    B [K] and dG.  ``receptors``: objects with grids, h, site_lo, site_n."""
    gam = gamma(q, eps, R, p_rep, p_att)
    J, K = coords.shape[0], len(receptors)
    logS = np.empty((J, K))
    nv = np.empty((J, K), dtype=np.int64)
    emin = np.empty((J, K))
    for k, r in enumerate(receptors):
        occ = getattr(r, "occ", None)
        logS[:, k], nv[:, k], emin[:, k] = logS_batch(r.grids, r.h, r.site_lo, r.site_n, coords, gam, kT,
                                                      occ=occ, R=R if occ is not None else None)
    B = bpmf(logS, nv, kT)
    h = receptors[0].h
    vs = site_volume(nv, h)
    return {"logS": logS, "n_valid": nv, "logZ": log_z(logS, nv), "Emin": emin, "bpmf": B,
            "dG": dG(B, kT, vs) if np.isfinite(B).any() and vs > 0 else np.inf, "gamma": gam}
