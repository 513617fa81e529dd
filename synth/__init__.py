"""Seeded synthetic workloads shaped like the paper's (Methodology: T4L-sized
binding-site grids at 0.25-0.375 A spacing, ~1000 rigid ligand configurations
each drawn from an apo ensemble and randomly rotated about the centroid).

This module draws random numbers and builds the receptor potential grids that
both the FP64 oracle and the CUDA path take as INPUTS.  It holds none of the
hot path's arithmetic (placement, spreading, correlation, exponential
averaging); the grid builder in ``gridgen.c`` is the input side of
Eq. (receptor_grid).

Recipe (all draws from numpy PCG64; workload ``i`` uses seed ``1000 + i`` and
receptor conformation ``k`` uses ``1000 + i + 100 k``):

* receptor atoms uniform in volume in a spherical shell [r1, r2] around the
  grid centre, Haar directions; charges N(0, sigma_q) shifted to net zero;
  R ~ U[1.5, 2.0] A, eps ~ U[0.05, 0.2] kcal/mol;
* conformations: independent Gaussian jitter (sigma 0.3 A) of a base structure;
* grids: elec = 332.06 sum q/r, LJr = min(clip, sum sqrt(eps) R^12 / r^12),
  LJa = -2 sum sqrt(eps) R^6 / r^6, r clamped to >= 0.5 A; node n at
  centre + (n - N/2) h;
* ligand: chain with 1.5 A bonds and 109.5 degree angles, charges N(0, 0.3)
  neutralised, same LJ ranges; each configuration draws every torsion from
  U[0, 2 pi) and a Haar-random rotation about the centroid.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_gridgen.so")
_lock = threading.Lock()
_lib = None

COULOMB = 332.06
KT = 0.5925  # kcal/mol


def build(force: bool = False) -> str:
    """Compile gridgen.c into an in-tree shared object (gcc, OpenMP)."""
    src = os.path.join(_HERE, "gridgen.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            d = ctypes.POINTER(ctypes.c_double)
            lib.gridgen_build.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, d, ctypes.c_int, d, d, d, d,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, ctypes.c_double]
            lib.gridgen_build.restype = ctypes.c_int
            lib.gridgen_occupancy.argtypes = [ctypes.POINTER(ctypes.c_ubyte), ctypes.c_int, ctypes.c_int,
                                              ctypes.c_int, ctypes.c_double, d, ctypes.c_int, d, d,
                                              ctypes.c_double]
            lib.gridgen_occupancy.restype = None
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Atoms:
    """Point atoms with charge q (e), well depth eps (kcal/mol), radius R (A)."""
    xyz: np.ndarray  # [n, 3] float64
    q: np.ndarray
    eps: np.ndarray
    R: np.ndarray


def _haar_directions(rng, n):
    d = rng.normal(size=(n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def receptor_atoms(seed: int, n_atoms: int, r1: float, r2: float, sigma_q: float = 0.35) -> Atoms:
    rng = np.random.default_rng(seed)
    r = rng.uniform(r1 ** 3, r2 ** 3, n_atoms) ** (1.0 / 3.0)
    xyz = _haar_directions(rng, n_atoms) * r[:, None]
    q = rng.normal(0.0, sigma_q, n_atoms)
    q -= q.mean()
    R = rng.uniform(1.5, 2.0, n_atoms)
    eps = rng.uniform(0.05, 0.2, n_atoms)
    return Atoms(xyz, q, eps, R)


def jitter(atoms: Atoms, sigma: float, seed: int) -> Atoms:
    rng = np.random.default_rng(seed)
    return Atoms(atoms.xyz + rng.normal(0.0, sigma, atoms.xyz.shape), atoms.q.copy(),
                 atoms.eps.copy(), atoms.R.copy())


def grid_origin(shape, h: float) -> np.ndarray:
    """Origin (node 0) of a grid centred on the atoms' frame origin."""
    return -np.asarray([n // 2 for n in shape], dtype=np.float64) * h


OCC_SCALE = 2.0 ** (-1.0 / 6.0)  # occupancy / cutoff radius in units of R (sigma)


def receptor_grids(atoms: Atoms, shape, h: float, clamp: float = 0.5, clip: float = 1e4,
                   p_rep: float = 12.0, p_att: float = 6.0, coulomb: float = COULOMB, cutoff: float = 0.0):
    """Return (grids float32 [3, nx, ny, nz] = elec, LJr, LJa; origin float64 [3]).
    ``cutoff`` > 0 zeroes every term of atom j within cutoff * R_j (used with
    occupancy grids, clamp and clip then 0)."""
    nx, ny, nz = (int(s) for s in shape)
    origin = grid_origin((nx, ny, nz), h)
    out = np.empty((3, nx, ny, nz), dtype=np.float32)
    xyz = np.ascontiguousarray(atoms.xyz, dtype=np.float64)
    q = np.ascontiguousarray(atoms.q, dtype=np.float64)
    eps = np.ascontiguousarray(atoms.eps, dtype=np.float64)
    R = np.ascontiguousarray(atoms.R, dtype=np.float64)
    o = np.ascontiguousarray(origin)
    rc = _load().gridgen_build(out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nx, ny, nz, float(h),
                               _dp(o), len(q), _dp(xyz), _dp(q), _dp(eps), _dp(R), float(p_rep),
                               float(p_att), float(coulomb), float(clamp), float(clip), float(cutoff))
    if rc != 0:
        raise MemoryError("gridgen_build failed")
    return out, origin


def receptor_occupancy(atoms: Atoms, shape, h: float, scale: float = OCC_SCALE) -> np.ndarray:
    """uint8 [nx, ny, nz]: 1 where some atom j has |r_j - n| < scale * R_j."""
    nx, ny, nz = (int(s) for s in shape)
    o = np.ascontiguousarray(grid_origin((nx, ny, nz), h))
    out = np.empty((nx, ny, nz), dtype=np.uint8)
    _load().gridgen_occupancy(out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), nx, ny, nz, float(h), _dp(o),
                              len(atoms.R), _dp(np.ascontiguousarray(atoms.xyz, dtype=np.float64)),
                              _dp(np.ascontiguousarray(atoms.R, dtype=np.float64)), float(scale))
    return out


@dataclass
class Ligand:
    """Per-atom ligand parameters (float32, as the hot path takes them)."""
    q: np.ndarray
    eps: np.ndarray
    R: np.ndarray

    @property
    def n_atoms(self) -> int:
        return int(self.q.shape[0])


def ligand_params(seed: int, n_atoms: int, sigma_q: float = 0.3) -> Ligand:
    rng = np.random.default_rng(seed)
    q = rng.normal(0.0, sigma_q, n_atoms)
    q -= q.mean()
    R = rng.uniform(1.5, 2.0, n_atoms)
    eps = rng.uniform(0.05, 0.2, n_atoms)
    return Ligand(q.astype(np.float32), eps.astype(np.float32), R.astype(np.float32))


def _chain(n: int, torsions: np.ndarray, bond: float = 1.5, angle_deg: float = 109.5) -> np.ndarray:
    """Cartesian chain from internal coordinates (fixed bond and angle)."""
    th = np.deg2rad(angle_deg)
    x = np.zeros((n, 3))
    if n > 1:
        x[1] = [bond, 0.0, 0.0]
    if n > 2:
        x[2] = x[1] + bond * np.array([-np.cos(th), np.sin(th), 0.0])
    for i in range(3, n):
        a, b, c = x[i - 3], x[i - 2], x[i - 1]
        bc = c - b
        bc /= np.linalg.norm(bc)
        nrm = np.cross(b - a, bc)
        nrm /= np.linalg.norm(nrm)
        m = np.stack([bc, np.cross(nrm, bc), nrm], axis=1)
        phi = torsions[i - 3]
        d = bond * np.array([-np.cos(th), np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi)])
        x[i] = c + m @ d
    return x


def random_rotations(rng, n: int) -> np.ndarray:
    """Haar-distributed rotation matrices from normalised 4D Gaussians."""
    qv = rng.normal(size=(n, 4))
    qv /= np.linalg.norm(qv, axis=1, keepdims=True)
    w, x, y, z = qv.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1)], 1)


def _chains(n: int, torsions: np.ndarray, bond: float = 1.5, angle_deg: float = 109.5) -> np.ndarray:
    """_chain for many torsion sets at once: torsions [J, n - 3] -> [J, n, 3]
    (the same construction, vectorised over configurations)."""
    J = torsions.shape[0]
    th = np.deg2rad(angle_deg)
    x = np.zeros((J, n, 3))
    if n > 1:
        x[:, 1] = [bond, 0.0, 0.0]
    if n > 2:
        x[:, 2] = x[:, 1] + bond * np.array([-np.cos(th), np.sin(th), 0.0])
    for i in range(3, n):
        a, b, c = x[:, i - 3], x[:, i - 2], x[:, i - 1]
        bc = c - b
        bc /= np.linalg.norm(bc, axis=1, keepdims=True)
        nrm = np.cross(b - a, bc)
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        m = np.stack([bc, np.cross(nrm, bc), nrm], axis=2)  # [J, 3, 3], columns as in _chain
        phi = torsions[:, i - 3]
        d = bond * np.stack([np.full(J, -np.cos(th)), np.sin(th) * np.cos(phi), np.sin(th) * np.sin(phi)], axis=1)
        x[:, i] = c + np.einsum("jrk,jk->jr", m, d)
    return x


def ligand_configs(seed: int, n_atoms: int, n_conf: int) -> np.ndarray:
    """[n_conf, n_atoms, 3] float32: random torsions, then a Haar rotation about
    the centroid (all rotations are drawn first, then each configuration's
    torsions in turn)."""
    rng = np.random.default_rng(seed)
    rots = random_rotations(rng, n_conf)
    tors = rng.uniform(0.0, 2 * np.pi, (n_conf, max(n_atoms - 3, 0)))
    x = _chains(n_atoms, tors)
    x -= x.mean(axis=1, keepdims=True)
    return np.einsum("jnk,jrk->jnr", x, rots).astype(np.float32)


@dataclass
class ReceptorInput:
    grids: np.ndarray  # float32 [3, nx, ny, nz]
    h: float
    origin: np.ndarray
    site_lo: tuple
    site_n: tuple
    occ: np.ndarray | None = None  # uint8 [nx, ny, nz] occupancy grid, or None

    @property
    def shape(self):
        return tuple(self.grids.shape[1:])


@dataclass
class LigandInput:
    params: Ligand
    coords: np.ndarray  # float32 [J, n_atoms, 3]


@dataclass
class Workload:
    name: str
    receptors: list
    ligands: list
    kT: float = KT


def central_site(shape, S):
    S = (S, S, S) if np.isscalar(S) else tuple(S)
    return tuple((n - s) // 2 for n, s in zip(shape, S)), tuple(int(s) for s in S)


def plain_small(n_conf: int = 64, seed: int = 1000, clip: float = 1e4) -> Workload:
    """32^3 grid at 0.375 A, 400 receptor atoms in a 4-10 A shell, 12-atom
    ligand, 16^3 site box, one receptor conformation."""
    atoms = receptor_atoms(seed, 400, 4.0, 10.0)
    g, o = receptor_grids(atoms, (32, 32, 32), 0.375, clip=clip)
    lo, sn = central_site((32, 32, 32), 16)
    lig = ligand_params(seed + 1, 12)
    coords = ligand_configs(seed + 2, 12, n_conf)
    return Workload("plain 32^3 h=0.375 J=%d K=1 12 atoms" % n_conf,
                    [ReceptorInput(g, 0.375, o, lo, sn)], [LigandInput(lig, coords)])


def protein_scale(n_conf: int = 2000, n_rec: int = 4, seed: int = 1001, clip: float = 1e4,
                  n_atoms_lig: int = 30) -> Workload:
    """96^3 grid at 0.25 A, 2600 receptor atoms in a 5-20 A shell, 30-atom
    ligand, 40^3 site box, conformations as 0.3 A Gaussian jitters."""
    base = receptor_atoms(seed, 2600, 5.0, 20.0)
    recs = []
    for k in range(n_rec):
        atoms = jitter(base, 0.3, seed + 100 * (k + 1))
        g, o = receptor_grids(atoms, (96, 96, 96), 0.25, clip=clip)
        lo, sn = central_site((96, 96, 96), 40)
        recs.append(ReceptorInput(g, 0.25, o, lo, sn))
    lig = ligand_params(seed + 1, n_atoms_lig)
    coords = ligand_configs(seed + 2, n_atoms_lig, n_conf)
    return Workload("protein-scale 96^3 h=0.25 J=%d K=%d %d atoms" % (n_conf, n_rec, n_atoms_lig),
                    recs, [LigandInput(lig, coords)])


def plain_small_occ(n_conf: int = 64, seed: int = 1000, shell=(6.0, 12.0), n_atoms: int = 200) -> Workload:
    """plain_small with the paper's clash treatment: grids with V = 0 inside
    2^(-1/6) R_j (no clamp, no clip) and the receptor occupancy grid."""
    atoms = receptor_atoms(seed, n_atoms, *shell)
    g, o = receptor_grids(atoms, (32, 32, 32), 0.375, clamp=0.0, clip=0.0, cutoff=OCC_SCALE)
    occ = receptor_occupancy(atoms, (32, 32, 32), 0.375)
    lo, sn = central_site((32, 32, 32), 16)
    lig = ligand_params(seed + 1, 12)
    coords = ligand_configs(seed + 2, 12, n_conf)
    return Workload("occupancy 32^3 h=0.375 J=%d K=1 12 atoms" % n_conf,
                    [ReceptorInput(g, 0.375, o, lo, sn, occ)], [LigandInput(lig, coords)])


def protein_scale_occ(n_conf: int = 2000, n_rec: int = 4, seed: int = 1001, n_atoms_lig: int = 30) -> Workload:
    """protein_scale with the paper's clash treatment (cutoff grids and
    receptor occupancy grids).  The receptor is a 10-22 A shell at 0.05
    atoms per A^3 (2020 atoms), so the 30-atom ligand fits the pocket at part
    of its translations."""
    base = receptor_atoms(seed, 2020, 10.0, 22.0)
    recs = []
    for k in range(n_rec):
        atoms = jitter(base, 0.3, seed + 100 * (k + 1))
        g, o = receptor_grids(atoms, (96, 96, 96), 0.25, clamp=0.0, clip=0.0, cutoff=OCC_SCALE)
        occ = receptor_occupancy(atoms, (96, 96, 96), 0.25)
        lo, sn = central_site((96, 96, 96), 40)
        recs.append(ReceptorInput(g, 0.25, o, lo, sn, occ))
    lig = ligand_params(seed + 1, n_atoms_lig)
    coords = ligand_configs(seed + 2, n_atoms_lig, n_conf)
    return Workload("occupancy protein-scale 96^3 h=0.25 J=%d K=%d %d atoms" % (n_conf, n_rec, n_atoms_lig),
                    recs, [LigandInput(lig, coords)])


def whole_surface(n_conf: int = 64, n_rec: int = 1, seed: int = 1003, n_atoms_lig: int = 30, site: int = 200,
                  n_atoms_rec: int = 1600) -> Workload:
    """The larger grid of the paper: 248^3 nodes at 0.25 A (62 A) around a
    whole protein-sized receptor (a 20 A ball of 1600 atoms), with a central
    site box of ``site``^3 translations that covers the surface; 30-atom
    ligand."""
    base = receptor_atoms(seed, n_atoms_rec, 0.0, 20.0)
    recs = []
    for k in range(n_rec):
        atoms = jitter(base, 0.3, seed + 100 * (k + 1))
        g, o = receptor_grids(atoms, (248, 248, 248), 0.25)
        lo, sn = central_site((248, 248, 248), site)
        recs.append(ReceptorInput(g, 0.25, o, lo, sn))
    lig = ligand_params(seed + 1, n_atoms_lig)
    coords = ligand_configs(seed + 2, n_atoms_lig, n_conf)
    return Workload("whole-surface 248^3 h=0.25 J=%d K=%d %d atoms, %d^3 site" % (n_conf, n_rec, n_atoms_lig, site),
                    recs, [LigandInput(lig, coords)])


def batched_uneven(n_lig: int = 141, n_conf: int = 500, n_rec: int = 10, seed: int = 1002,
                   clip: float = 1e4, sizes=(64, 112), sites=(24, 40), atoms_range=(8, 60)) -> Workload:
    """Many ligands of uneven atom counts against receptor conformations of
    uneven grid edges (0.25 A) and site boxes."""
    rng = np.random.default_rng(seed)
    base = receptor_atoms(seed, 2600, 5.0, 20.0)
    recs = []
    edges = rng.integers(sizes[0], sizes[1] + 1, n_rec)
    site = rng.integers(sites[0], sites[1] + 1, n_rec)
    for k in range(n_rec):
        atoms = jitter(base, 0.3, seed + 100 * (k + 1))
        shp = (int(edges[k]),) * 3
        g, o = receptor_grids(atoms, shp, 0.25, clip=clip)
        lo, sn = central_site(shp, int(site[k]))
        recs.append(ReceptorInput(g, 0.25, o, lo, sn))
    natoms = rng.integers(atoms_range[0], atoms_range[1] + 1, n_lig)
    ligs = []
    for i in range(n_lig):
        s = seed + 10_000 + 2 * i
        ligs.append(LigandInput(ligand_params(s, int(natoms[i])), ligand_configs(s + 1, int(natoms[i]), n_conf)))
    return Workload("batched %d ligands x %d conf x %d receptors" % (n_lig, n_conf, n_rec), recs, ligs)
