"""FP64 reference of the learned-proposal pieces (TEST INFRASTRUCTURE ONLY;
shares no code with the CUDA library).

* ``mlp_forward`` / ``mlp_grads`` -- the MLP n_in -> width (ReLU) x depth -> 1
  with mean-squared-error loss in normalised units; ``bf16=True`` rounds both
  operands of every matrix product to bfloat16 (round to nearest even) exactly
  where the GPU kernels do, everything else in FP64.
* ``proposal`` -- q = mix softmax(pred / tau) + (1 - mix)/J and inverse-CDF draws.
* ``config_targets`` -- per-configuration weights ls_j = ln sum_k S_jk of one
  ligand and the training targets max(ls_j - max ls, -clip).
* ``chi2`` -- exact relative variance of one importance-sampling draw of Z.
* ``is_bpmf`` -- importance-weighted BPMF (Eq. sample_mean_BPMF with
  configurations drawn from q): Z_k ~ (1/M) sum_s S_{j_s k}/q_{j_s},
  B_k = -kT [ln Z_k - ln N_k].
"""
from __future__ import annotations

import numpy as np
from scipy.special import logsumexp


def bf16(x):
    """Round float values to bfloat16 (nearest, ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, n_in, width, depth):
    """Packed parameters -> list of (W [in, out], b [out]) in FP64."""
    p = np.asarray(params, dtype=np.float64)
    layers, o = [], 0
    for l in range(depth + 1):
        fi = n_in if l == 0 else width
        fo = 1 if l == depth else width
        W = p[o:o + fi * fo].reshape(fi, fo)
        o += fi * fo
        b = p[o:o + fo]
        o += fo
        layers.append((W, b))
    assert o == p.size
    return layers


def _mm(A, B, rnd):
    return (bf16(A) @ bf16(B)) if rnd else A @ B


def mlp_forward(params, norm, X, n_in, width, depth, bf16_ops=True, return_cache=False):
    layers = unpack(params, n_in, width, depth)
    norm = np.asarray(norm, dtype=np.float64)
    Xn = (np.asarray(X, dtype=np.float64) - norm[:n_in]) / norm[n_in:2 * n_in]
    if bf16_ops:
        Xn = Xn.astype(np.float32).astype(np.float64)
    Z, a = [], Xn
    for l, (W, b) in enumerate(layers):
        z = _mm(a, W, bf16_ops) + b
        Z.append(z)
        a = np.maximum(z, 0.0)
    y_n = Z[-1][:, 0]
    y = y_n * norm[2 * n_in + 1] + norm[2 * n_in]
    return (y, Xn, Z) if return_cache else y


def mlp_grads(params, norm, X, t, n_in, width, depth, bf16_ops=True):
    """(loss, packed gradient) of mean((y_n - t_n)^2) in normalised units."""
    layers = unpack(params, n_in, width, depth)
    norm = np.asarray(norm, dtype=np.float64)
    _, Xn, Z = mlp_forward(params, norm, X, n_in, width, depth, bf16_ops, return_cache=True)
    tn = (np.asarray(t, dtype=np.float64) - norm[2 * n_in]) / norm[2 * n_in + 1]
    B = Xn.shape[0]
    d = Z[-1][:, 0] - tn
    loss = float(np.mean(d * d))
    dZ = (2.0 * d / B)[:, None]
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a_in = Xn if l == 0 else np.maximum(Z[l - 1], 0.0)
        gW = _mm(a_in.T, dZ, bf16_ops)
        gb = dZ.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dA = _mm(dZ, W.T, bf16_ops)
            dZ = dA * (Z[l - 1] > 0)
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return loss, flat


def proposal(pred, mix, tau=1.0):
    p = np.asarray(pred, dtype=np.float64) / tau
    w = np.exp(p - p.max())
    return mix * w / w.sum() + (1.0 - mix) / p.size


def config_targets(logZ, n_valid, clip):
    """(ls [J], t [J]): ls_j = ln sum_k n_jk exp(logZ_jk) (-inf without a valid
    translation) and t_j = max(ls_j - max ls, -clip) for one ligand."""
    logZ = np.asarray(logZ, dtype=np.float64)
    n = np.asarray(n_valid, dtype=np.float64)
    with np.errstate(divide="ignore"):
        terms = np.where(n > 0, logZ + np.log(np.maximum(n, 1)), -np.inf)
    ls = logsumexp(terms, axis=1)
    ls = np.where(np.isfinite(ls), ls, -np.inf)
    mx = ls.max()
    t = np.where(np.isfinite(ls), np.maximum(ls - mx, -clip), -clip) if np.isfinite(mx) else np.full(ls.shape, -clip)
    return ls, t


def chi2(pred, ls, mix, tau):
    """sum_j S_j^2 / (q_j Z^2) - 1 with S_j = exp(ls_j), Z = sum S_j, q the
    proposal: the relative variance of (S_j / q_j) / Z for one draw j ~ q."""
    q = proposal(pred, mix, tau)
    ls = np.asarray(ls, dtype=np.float64)
    ok = np.isfinite(ls)
    w = np.exp(ls[ok] - ls[ok].max())
    w /= w.sum()
    return float(np.sum(w * w / q[ok]) - 1.0)


def draw(q, u):
    """Inverse-CDF draws: first index whose cumulative q exceeds u * total."""
    cdf = np.cumsum(q)
    return np.searchsorted(cdf, np.asarray(u) * cdf[-1], side="right")


def is_bpmf(logZ_s, n_s, q_s, n_tot, kT):
    """Importance-weighted BPMF per receptor; q_s are the proposal
    probabilities of the drawn configurations."""
    logZ_s = np.asarray(logZ_s, dtype=np.float64)
    n_s = np.asarray(n_s, dtype=np.float64)
    q_s = np.asarray(q_s, dtype=np.float64)
    M = logZ_s.shape[0]
    with np.errstate(divide="ignore"):
        terms = np.where(n_s > 0, logZ_s + np.log(np.maximum(n_s, 1)), -np.inf) - np.log(q_s)[:, None]
    lz = logsumexp(terms, axis=0) - np.log(M)
    return -kT * (lz - np.log(np.asarray(n_tot, dtype=np.float64)))


def features(coords, q, eps, R, h):
    """FP64 features of one configuration, in the order bpmf_features uses
    (independent implementation: numpy eigh and scipy rotations)."""
    from scipy.spatial.transform import Rotation
    x = np.asarray(coords, dtype=np.float64)
    c = x.mean(axis=0)
    r = x - c
    g = r.T @ r / x.shape[0]
    w, v = np.linalg.eigh(g)  # ascending
    e = v.T.copy()            # rows = axes
    for a in range(2):
        if np.sum((r @ e[a]) ** 3) < 0:
            e[a] = -e[a]
    e[2] = np.cross(e[0], e[1])
    M = e.T                   # columns = principal axes (principal frame -> lab)
    qx, qy, qz, qw = Rotation.from_matrix(M).as_quat()
    quat = np.array([qw, qx, qy, qz])
    if quat[0] < 0:
        quat = -quat
    xf = np.asarray(coords, dtype=np.float32)
    ext = (xf.max(0) - xf.min(0)).astype(np.float32)
    u = np.ceil((ext / np.float32(h)).astype(np.float32)) + 4
    f = [*quat, *u, *w, np.sqrt(w.sum()), np.linalg.norm(x[-1] - x[0])]
    for k in range(2):
        if x.shape[0] >= 4 + k:
            b1, b2, b3 = x[k + 1] - x[k], x[k + 2] - x[k + 1], x[k + 3] - x[k + 2]
            n1, n2 = np.cross(b1, b2), np.cross(b2, b3)
            m = np.cross(n1, b2 / np.linalg.norm(b2))
            ang = np.arctan2(m @ n2, n1 @ n2)
            f += [np.sin(ang), np.cos(ang)]
        else:
            f += [0.0, 1.0]
    counts = np.zeros(8)
    bins = (np.asarray(R) > 1.75) * 4 + (np.asarray(eps) > 0.125) * 2 + (np.asarray(q) > 0) * 1
    for b in bins:
        counts[b] += 1
    return np.array(f + list(counts))
