"""GB300 (sm_103a) FFT-correlation BPMF library: thin Python binding.

The compute path is ``libbpmf.so`` (hand-written CUDA kernels behind the C ABI
declared in ``include/bpmf.h``).  This module only marshals arguments: numpy
arrays (host memory) or torch tensors (host or device memory) are passed as raw
pointers, and every entry point keeps the C name.  Importing this module does
not need a GPU; calling into the library does, and there is no CPU fallback:
if the library is missing or no GPU is visible, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(_ROOT, "include")
LIB_PATH = os.path.join(_HERE, "libbpmf.so")
_SOURCES = ["kernels.cu", "xpass.cu", "yzinv.cu", "ligspec.cu", "occupancy.cu", "refine.cu", "bpmf_api.cu", "bpmf_static.cu", "proposal.cu", "bpmf_proposal.cu"]
_HEADERS = ["arith.cuh", "fft.cuh", "kernels.cuh", "proposal.cuh", "tc_dft.cuh", "tc05.cuh", "tma.cuh"]

BPMF_OK = 0
BPMF_ERR_INVALID_ARG = -1
BPMF_ERR_OOM = -2
BPMF_ERR_CUDA = -3
BPMF_ERR_TIMEOUT = -4
BPMF_ERR_SIZE_UNSUPPORTED = -5
BPMF_WARN_NO_VALID = 1
BPMF_WARN_REFINE_FALLBACK = 2
BPMF_MODE_FP32 = 0
BPMF_MODE_FF = 1
BPMF_MODE_SPLIT_BF16 = 2
BPMF_MODE_REFINE = 3
BPMF_MODE_SPLIT_REFINE = 4
BPMF_MAX_ATOMS = 256
BPMF_MAX_FFT_EDGE = 256

NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "-I" + _INCLUDE]


class BpmfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: status {status} ({_status_text(status)}){': ' + detail if detail else ''}")


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB_PATH):
        return True
    t = os.path.getmtime(LIB_PATH)
    deps = [os.path.join(_CSRC, f) for f in _SOURCES + _HEADERS] + [os.path.join(_INCLUDE, "bpmf.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the CUDA sources for sm_103a into an in-tree libbpmf.so
    (translation units in parallel, then one link)."""
    if not force and not _stale():
        return LIB_PATH
    nvcc = _nvcc()
    objdir = os.path.join(_HERE, "_build")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *NVCC_FLAGS, "-c", os.path.join(_CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(len(_SOURCES)) as ex:
        objs = list(ex.map(compile_one, _SOURCES))
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    r = subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "bpmf_create": (_I, [_I, ctypes.POINTER(_P)]),
    "bpmf_destroy": (None, [_P]),
    "bpmf_status_string": (ctypes.c_char_p, [_I]),
    "bpmf_last_error": (ctypes.c_char_p, [_P]),
    "bpmf_receptor_load": (_I, [_P, _P, _I, _I, _I, _D, _P, _P, _P, _P, ctypes.POINTER(_P)]),
    "bpmf_receptor_free": (None, [_P]),
    "bpmf_ligand_batch": (_I, [_P, _I, _P, _P, _P, _P, _P, _P, _I, _I, _P, ctypes.POINTER(_P)]),
    "bpmf_ligand_free": (None, [_P]),
    "bpmf_eval": (_I, [_P, _P, _P, _I, _D, ctypes.c_uint, _P, _P, _P, _P, _P]),
    "bpmf_eval_dominant": (_I, [_P, _P, _P, _I, _D, ctypes.c_uint, _P, _P, _P, _P, _P, _P, _P]),
    "bpmf_export_energies": (_I, [_P, _P, _P, _I, _I, ctypes.c_uint, _P, _P]),
    "bpmf_receptor_set_occupancy": (_I, [_P, _P, _P, _P]),
    "bpmf_fft_edge": (_I, [_I]),
    "bpmf_crop_window": (_I, [_I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "bpmf_set_workspace_limit": (_I, [_P, ctypes.c_size_t]),
    "bpmf_profile_enable": (_I, [_P, _I]),
    "bpmf_profile_count": (_I, [_P]),
    "bpmf_profile_entry": (_I, [_P, _I, ctypes.c_char_p, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_int64)]),
    "bpmf_set_graph_mode": (_I, [_P, _I]),
    "bpmf_transform_edges": (_I, [_P, _P, _P, _I, ctypes.c_uint, _P]),
    "bpmf_set_refine_check_scale": (_I, [_P, _D]),
    "bpmf_set_refine_list_cap": (_I, [_P, _I]),
    "bpmf_set_wait_test": (_I, [_P, _I]),
    "bpmf_features": (_I, [_P, _P, _D, _P, _P]),
    "bpmf_valid_counts": (_I, [_P, _P, _P, _I, _P]),
    "bpmf_mlp_param_count": (ctypes.c_longlong, [_I, _I, _I]),
    "bpmf_mlp_create": (_I, [_P, _I, _I, _I, _P, _P, ctypes.POINTER(_P)]),
    "bpmf_mlp_free": (None, [_P]),
    "bpmf_mlp_get_params": (_I, [_P, _P]),
    "bpmf_mlp_forward": (_I, [_P, _P, _P, _I, _P, _P]),
    "bpmf_mlp_train_step": (_I, [_P, _P, _P, _P, _I, ctypes.c_float, _I, _P, _P, _P]),
    "bpmf_proposal_sample": (_I, [_P, _P, _I, _D, _D, _P, _I, _P, _P, _P]),
    "bpmf_config_targets": (_I, [_P, _P, _P, _I, _I, _D, _P, _P, _P]),
    "bpmf_proposal_chi2": (_I, [_P, _P, _P, _I, _D, _D, _P, _P]),
    "bpmf_proposal_bpmf": (_I, [_P, _P, _P, _P, _I, _I, _P, _D, _P, _P]),
    "bpmf_sir_poses": (_I, [_P, _P, _I, _P, _I, _I, _D, ctypes.c_uint, _P, _P, _P, _P, _I, _P, _P, _P]),
    "bpmf_bootstrap": (_I, [_P, _P, _P, _I, _I, _D, _D, _P, _I, _P, _P, _P]),
    "bpmf_autotune": (_I, [_P, _P, _P, _I, ctypes.c_uint, _P]),
    "bpmf_export_energies_static": (_I, [_P, _I, _I, _I, _D, _P, _P, _I, _P, _P, _P, _P, _I, _I, ctypes.c_uint, _P,
                                         _P]),
}


def lib():
    """Load libbpmf.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _status_text(s):
    try:
        return lib().bpmf_status_string(int(s)).decode()
    except Exception:  # library not loadable: describe without it
        return str(s)


# ------------------------------------------------------------------ marshalling
def _ptr(a, dtype):
    """Raw pointer of a numpy array or torch tensor (contiguous, given dtype)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):  # torch tensor
        import torch
        tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32,
               np.int64: torch.int64}[dtype]
        if a.dtype != tdt or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {tdt}")
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"array must be a C-contiguous numpy {np.dtype(dtype).name} array")
    return ctypes.c_void_p(a.ctypes.data)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _check(rc, where, ctx=None):
    if rc < 0:
        detail = ""
        if ctx is not None:
            try:
                detail = lib().bpmf_last_error(ctx).decode()
            except Exception:
                pass
        raise BpmfError(rc, where, detail)
    return rc


# -------------------------------------------------------------------- C names
def bpmf_create(device: int = 0):
    h = ctypes.c_void_p()
    _check(lib().bpmf_create(int(device), ctypes.byref(h)), "bpmf_create")
    return h


def bpmf_destroy(ctx):
    lib().bpmf_destroy(ctx)


def bpmf_status_string(status: int) -> str:
    return lib().bpmf_status_string(int(status)).decode()


def bpmf_last_error(ctx) -> str:
    return lib().bpmf_last_error(ctx).decode()


def bpmf_fft_edge(n: int) -> int:
    return int(lib().bpmf_fft_edge(int(n)))


def bpmf_crop_window(n: int, site_lo: int, site_n: int, u: int):
    """(transform edge, first receptor node) of the cropped transform along one
    axis for a ligand box of edge u (host only)."""
    edge, c0 = ctypes.c_int(), ctypes.c_int()
    _check(lib().bpmf_crop_window(int(n), int(site_lo), int(site_n), int(u), ctypes.byref(edge), ctypes.byref(c0)),
           "bpmf_crop_window", None)
    return edge.value, c0.value


def bpmf_set_workspace_limit(ctx, nbytes: int):
    _check(lib().bpmf_set_workspace_limit(ctx, int(nbytes)), "bpmf_set_workspace_limit", ctx)


def bpmf_receptor_load(ctx, grids, h, origin, site_lo, site_n, stream=None):
    """grids: [3, nx, ny, nz] float32 (numpy or torch, host or device)."""
    nx, ny, nz = (int(v) for v in tuple(grids.shape)[1:])
    o = np.ascontiguousarray(np.asarray(origin, dtype=np.float64).reshape(3))
    lo = np.ascontiguousarray(np.asarray(site_lo, dtype=np.int32).reshape(3))
    sn = np.ascontiguousarray(np.asarray(site_n, dtype=np.int32).reshape(3))
    out = ctypes.c_void_p()
    rc = lib().bpmf_receptor_load(ctx, _ptr(grids, np.float32), nx, ny, nz, float(h), _ptr(o, np.float64),
                                  _ptr(lo, np.int32), _ptr(sn, np.int32), _stream(stream), ctypes.byref(out))
    _check(rc, "bpmf_receptor_load", ctx)
    return out


def bpmf_receptor_free(rec):
    lib().bpmf_receptor_free(rec)


def bpmf_receptor_set_occupancy(ctx, rec, occ, stream=None):
    """occ: uint8 [nx, ny, nz] (numpy or torch, host or device), or None to detach."""
    if occ is None:
        p = None
    elif hasattr(occ, "data_ptr"):
        import torch
        if occ.dtype != torch.uint8 or not occ.is_contiguous():
            raise TypeError("occupancy tensor must be contiguous uint8")
        p = ctypes.c_void_p(occ.data_ptr())
    else:
        a = np.ascontiguousarray(occ, dtype=np.uint8)
        occ = a
        p = ctypes.c_void_p(a.ctypes.data)
    _check(lib().bpmf_receptor_set_occupancy(ctx, rec, p, _stream(stream)), "bpmf_receptor_set_occupancy", ctx)


def bpmf_ligand_batch(ctx, n_atoms, n_conf, coords, q, eps, R, p_rep=12, p_att=6, stream=None):
    """n_atoms, n_conf: per-ligand counts (host); coords float32 [sum conf*atoms, 3];
    q, eps, R float32 [sum atoms] (numpy or torch, host or device)."""
    na = np.ascontiguousarray(np.asarray(n_atoms, dtype=np.int32).reshape(-1))
    nc = np.ascontiguousarray(np.asarray(n_conf, dtype=np.int32).reshape(-1))
    out = ctypes.c_void_p()
    rc = lib().bpmf_ligand_batch(ctx, int(na.size), _ptr(na, np.int32), _ptr(nc, np.int32),
                                 _ptr(coords, np.float32), _ptr(q, np.float32), _ptr(eps, np.float32),
                                 _ptr(R, np.float32), int(p_rep), int(p_att), _stream(stream), ctypes.byref(out))
    _check(rc, "bpmf_ligand_batch", ctx)
    return out


def bpmf_ligand_free(lig):
    lib().bpmf_ligand_free(lig)


def bpmf_eval(ctx, lig, recs, kT, mode, logZ, n_valid=None, bpmf=None, dG=None, stream=None) -> int:
    """Outputs are caller-allocated (numpy or torch, host or device):
    logZ float64 [total_conf, K], n_valid int64 [total_conf, K], bpmf float64
    [n_lig, K], dG float64 [n_lig].  Returns BPMF_OK or BPMF_WARN_NO_VALID."""
    K = len(recs)
    arr = (ctypes.c_void_p * K)(*[r.value if isinstance(r, ctypes.c_void_p) else r for r in recs])
    rc = lib().bpmf_eval(ctx, lig, ctypes.cast(arr, ctypes.c_void_p), K, float(kT), int(mode),
                         _ptr(logZ, np.float64), _ptr(n_valid, np.int64), _ptr(bpmf, np.float64),
                         _ptr(dG, np.float64), _stream(stream))
    return _check(rc, "bpmf_eval", ctx)


def bpmf_eval_dominant(ctx, lig, recs, kT, mode, logZ, n_valid=None, bpmf=None, dG=None, psi_min=None,
                       psi_dom=None, stream=None) -> int:
    """bpmf_eval plus psi_min float64 [total_conf, K] (minimum energy over the
    valid translations) and psi_dom float64 [n_lig, K + 2] (per receptor
    minimum over configurations, their minimum, their exponential average)."""
    K = len(recs)
    arr = (ctypes.c_void_p * K)(*[r.value if isinstance(r, ctypes.c_void_p) else r for r in recs])
    rc = lib().bpmf_eval_dominant(ctx, lig, ctypes.cast(arr, ctypes.c_void_p), K, float(kT), int(mode),
                                  _ptr(logZ, np.float64), _ptr(n_valid, np.int64), _ptr(bpmf, np.float64),
                                  _ptr(dG, np.float64), _ptr(psi_min, np.float64), _ptr(psi_dom, np.float64),
                                  _stream(stream))
    return _check(rc, "bpmf_eval_dominant", ctx)


def bpmf_export_energies(ctx, lig, rec, lig_index, conf_index, mode, out, stream=None) -> int:
    """out: float64 [S0, S1, S2] (the receptor's site box), host or device."""
    rc = lib().bpmf_export_energies(ctx, lig, rec, int(lig_index), int(conf_index), int(mode),
                                    _ptr(out, np.float64), _stream(stream))
    return _check(rc, "bpmf_export_energies", ctx)


def bpmf_set_graph_mode(ctx, on: bool = True):
    _check(lib().bpmf_set_graph_mode(ctx, 1 if on else 0), "bpmf_set_graph_mode", ctx)


def bpmf_autotune(ctx, lig, recs, mode, stream=None):
    K = len(recs)
    arr = (ctypes.c_void_p * K)(*[r.value if isinstance(r, ctypes.c_void_p) else r for r in recs])
    _check(lib().bpmf_autotune(ctx, lig, ctypes.cast(arr, ctypes.c_void_p), K, int(mode), _stream(stream)),
           "bpmf_autotune", ctx)


def bpmf_profile_enable(ctx, on: bool = True):
    _check(lib().bpmf_profile_enable(ctx, 1 if on else 0), "bpmf_profile_enable", ctx)


def bpmf_profile_count(ctx) -> int:
    return _check(lib().bpmf_profile_count(ctx), "bpmf_profile_count", ctx)


def bpmf_profile_entry(ctx, i: int):
    """(kernel name, total device ms, launches) of recorded kernel i."""
    buf = ctypes.create_string_buffer(128)
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(lib().bpmf_profile_entry(ctx, int(i), buf, 128, ctypes.byref(ms), ctypes.byref(n)),
           "bpmf_profile_entry", ctx)
    return buf.value.decode(), ms.value, n.value


def bpmf_profile(ctx) -> dict:
    """{kernel name: (total ms, launches)} recorded since profiling was enabled."""
    return {name: (ms, n) for name, ms, n in (bpmf_profile_entry(ctx, i) for i in range(bpmf_profile_count(ctx)))}


BPMF_STATIC_SCRATCH_BYTES = 64 * 1024 * 1024


def bpmf_export_energies_static(grids, h, site_lo, site_n, coords, q, eps, R, mode, out, p_rep=12, p_att=6,
                                stream=None) -> int:
    """Energy export that allocates no device memory (scratch lives in the
    library's static device array).  grids, coords, q, eps, R and out must be
    device tensors on the current device; returns the status code."""
    nx, ny, nz = (int(v) for v in tuple(grids.shape)[1:])
    lo = np.ascontiguousarray(np.asarray(site_lo, dtype=np.int32).reshape(3))
    sn = np.ascontiguousarray(np.asarray(site_n, dtype=np.int32).reshape(3))
    n_atoms = int(tuple(coords.shape)[0])
    rc = lib().bpmf_export_energies_static(_ptr(grids, np.float32), nx, ny, nz, float(h), _ptr(lo, np.int32),
                                           _ptr(sn, np.int32), n_atoms, _ptr(coords, np.float32),
                                           _ptr(q, np.float32), _ptr(eps, np.float32), _ptr(R, np.float32),
                                           int(p_rep), int(p_att), int(mode), _ptr(out, np.float64),
                                           _stream(stream))
    return _check(rc, "bpmf_export_energies_static")


BPMF_N_FEATURES = 24


def bpmf_features(ctx, lig, h, out, stream=None):
    """out: float32 [total_conf, 24] (numpy or torch, host or device)."""
    _check(lib().bpmf_features(ctx, lig, float(h), _ptr(out, np.float32), _stream(stream)), "bpmf_features", ctx)


def bpmf_mlp_param_count(n_in, width, depth) -> int:
    return int(lib().bpmf_mlp_param_count(int(n_in), int(width), int(depth)))


def bpmf_mlp_create(ctx, n_in, width, depth, params, norm):
    p = np.ascontiguousarray(params, dtype=np.float32)
    nm = np.ascontiguousarray(norm, dtype=np.float32)
    if p.size != bpmf_mlp_param_count(n_in, width, depth) or nm.size != 2 * n_in + 2:
        raise ValueError("parameter / normalisation sizes do not match the network shape")
    out = ctypes.c_void_p()
    _check(lib().bpmf_mlp_create(ctx, int(n_in), int(width), int(depth), _ptr(p, np.float32),
                                 _ptr(nm, np.float32), ctypes.byref(out)), "bpmf_mlp_create", ctx)
    return out


def bpmf_mlp_free(mlp):
    lib().bpmf_mlp_free(mlp)


def bpmf_mlp_get_params(mlp, n_params):
    out = np.empty(int(n_params), dtype=np.float32)
    _check(lib().bpmf_mlp_get_params(mlp, _ptr(out, np.float32)), "bpmf_mlp_get_params")
    return out


def bpmf_mlp_forward(ctx, mlp, X, y, stream=None):
    B = int(tuple(X.shape)[0])
    _check(lib().bpmf_mlp_forward(ctx, mlp, _ptr(X, np.float32), B, _ptr(y, np.float32), _stream(stream)),
           "bpmf_mlp_forward", ctx)


def bpmf_mlp_train_step(ctx, mlp, X, t, lr, apply=True, grads=None, stream=None) -> float:
    B = int(tuple(X.shape)[0])
    loss = np.zeros(1, dtype=np.float32)
    _check(lib().bpmf_mlp_train_step(ctx, mlp, _ptr(X, np.float32), _ptr(t, np.float32), B, float(lr),
                                     1 if apply else 0, _ptr(loss, np.float32),
                                     _ptr(grads, np.float32) if grads is not None else None, _stream(stream)),
           "bpmf_mlp_train_step", ctx)
    return float(loss[0])


def bpmf_proposal_sample(ctx, pred, mix, u, idx, q_s, stream=None, tau=1.0):
    J = int(tuple(pred.shape)[0])
    M = int(tuple(u.shape)[0])
    _check(lib().bpmf_proposal_sample(ctx, _ptr(pred, np.float32), J, float(mix), float(tau), _ptr(u, np.float64), M,
                                      _ptr(idx, np.int32), _ptr(q_s, np.float64), _stream(stream)),
           "bpmf_proposal_sample", ctx)


def bpmf_config_targets(ctx, logZ, n_valid, clip, ls, t, stream=None):
    """logZ float64 [J, K], n_valid int64 [J, K] -> ls float64 [J], t float32 [J] (device)."""
    J, K = (int(v) for v in tuple(logZ.shape))
    _check(lib().bpmf_config_targets(ctx, _ptr(logZ, np.float64), _ptr(n_valid, np.int64), J, K, float(clip),
                                     _ptr(ls, np.float64), _ptr(t, np.float32), _stream(stream)),
           "bpmf_config_targets", ctx)


def bpmf_proposal_chi2(ctx, pred, ls, mix, tau, out, stream=None):
    """Exact relative variance of one importance-sampling draw; out float64 [1] (device)."""
    J = int(tuple(pred.shape)[0])
    _check(lib().bpmf_proposal_chi2(ctx, _ptr(pred, np.float32), _ptr(ls, np.float64), J, float(mix), float(tau),
                                    _ptr(out, np.float64), _stream(stream)),
           "bpmf_proposal_chi2", ctx)


def bpmf_proposal_bpmf(ctx, logZ_s, n_s, q_s, n_tot, kT, bpmf, stream=None):
    M, K = (int(v) for v in tuple(logZ_s.shape))
    _check(lib().bpmf_proposal_bpmf(ctx, _ptr(logZ_s, np.float64), _ptr(n_s, np.int64), _ptr(q_s, np.float64), M,
                                    K, _ptr(n_tot, np.int64), float(kT), _ptr(bpmf, np.float64), _stream(stream)),
           "bpmf_proposal_bpmf", ctx)


def bpmf_sir_poses(ctx, lig, lig_index, rec, k, kT, mode, logZ, n_valid, u1, u2, conf, pose, stream=None):
    """Device tensors: logZ float64 [J, K], n_valid int64 [J, K] of ligand
    lig_index, u1/u2 float64 [M]; conf/pose int32 [M] out."""
    J, K = (int(v) for v in tuple(logZ.shape))
    M = int(tuple(u1.shape)[0])
    if tuple(u2.shape)[0] != M or tuple(conf.shape)[0] != M or tuple(pose.shape)[0] != M:
        raise ValueError("u1, u2, conf and pose must have the same length")
    _check(lib().bpmf_sir_poses(ctx, lig, int(lig_index), rec, K, int(k), float(kT), int(mode),
                                _ptr(logZ, np.float64), _ptr(n_valid, np.int64), _ptr(u1, np.float64),
                                _ptr(u2, np.float64), M, _ptr(conf, np.int32), _ptr(pose, np.int32),
                                _stream(stream)), "bpmf_sir_poses", ctx)


def bpmf_bootstrap(ctx, logZ, n_valid, kT, h, u, rep=None, stats=None, stream=None):
    """Device tensors: logZ float64 [J, K], n_valid int64 [J, K], u float64
    [R, J]; rep float64 [R, K + 1] and / or stats float64 [2, K + 1] out."""
    J, K = (int(v) for v in tuple(logZ.shape))
    R = int(tuple(u.shape)[0])
    if tuple(u.shape) != (R, J):
        raise ValueError("u must be [R, J]")
    _check(lib().bpmf_bootstrap(ctx, _ptr(logZ, np.float64), _ptr(n_valid, np.int64), J, K, float(kT), float(h),
                                _ptr(u, np.float64), R, _ptr(rep, np.float64), _ptr(stats, np.float64),
                                _stream(stream)), "bpmf_bootstrap", ctx)


def bpmf_valid_counts(ctx, lig, recs, total_conf):
    K = len(recs)
    arr = (ctypes.c_void_p * K)(*[r.value if isinstance(r, ctypes.c_void_p) else r for r in recs])
    out = np.empty((int(total_conf), K), dtype=np.int64)
    _check(lib().bpmf_valid_counts(ctx, lig, ctypes.cast(arr, ctypes.c_void_p), K, _ptr(out, np.int64)),
           "bpmf_valid_counts", ctx)
    return out


def bpmf_transform_edges(ctx, lig, recs, total_conf, mode):
    """int32 [total_conf, K, 3]: the transform edges bpmf_eval uses for each
    (configuration, receptor) pair in ``mode`` (host-only query)."""
    K = len(recs)
    arr = (ctypes.c_void_p * K)(*[r.value if isinstance(r, ctypes.c_void_p) else r for r in recs])
    out = np.empty((int(total_conf), K, 3), dtype=np.int32)
    _check(lib().bpmf_transform_edges(ctx, lig, ctypes.cast(arr, ctypes.c_void_p), K, int(mode), _ptr(out, np.int32)),
           "bpmf_transform_edges", ctx)
    return out


def bpmf_set_refine_check_scale(ctx, scale):
    """Scale of B in the refined form's certificate check (testing)."""
    return _check(lib().bpmf_set_refine_check_scale(ctx, float(scale)), "bpmf_set_refine_check_scale", ctx)


def bpmf_set_wait_test(ctx, on):
    """Testing: the x pass's first receptor-tile wait runs out (BPMF_ERR_TIMEOUT)."""
    return _check(lib().bpmf_set_wait_test(ctx, int(bool(on))), "bpmf_set_wait_test", ctx)


def bpmf_set_refine_list_cap(ctx, cap):
    """Candidate-list capacity per pair in the refined form (0: the default rule; testing)."""
    return _check(lib().bpmf_set_refine_list_cap(ctx, int(cap)), "bpmf_set_refine_list_cap", ctx)
