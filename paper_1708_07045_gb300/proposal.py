"""Learned-proposal workflow over the C entry points (argument marshalling and
loops only; features, the MLP, sampling and the estimator run in the library's
kernels).

Flow for one ligand with J configurations against K receptors:
  features (bpmf_features) -> prediction (bpmf_mlp_forward) ->
  q = mix softmax(pred) + (1 - mix)/J and M draws (bpmf_proposal_sample, on
  uniforms from a seeded numpy generator) -> bpmf_eval on the drawn
  configurations -> importance-weighted BPMF (bpmf_proposal_bpmf) with the
  valid-translation totals of all J configurations (bpmf_valid_counts).
"""
from __future__ import annotations

import numpy as np

from . import (BPMF_MODE_FF, BPMF_N_FEATURES, bpmf_eval, bpmf_features, bpmf_ligand_batch, bpmf_ligand_free,
               bpmf_mlp_create, bpmf_mlp_forward, bpmf_mlp_free, bpmf_mlp_param_count, bpmf_mlp_train_step,
               bpmf_proposal_bpmf, bpmf_proposal_sample, bpmf_valid_counts)


def init_params(n_in: int, width: int, depth: int, seed: int = 0) -> np.ndarray:
    """He-uniform weights, zero biases, packed as bpmf_mlp_create expects."""
    rng = np.random.default_rng(seed)
    out = []
    for l in range(depth + 1):
        fi = n_in if l == 0 else width
        fo = 1 if l == depth else width
        lim = np.sqrt(6.0 / fi)
        out += [rng.uniform(-lim, lim, fi * fo), np.zeros(fo)]
    p = np.concatenate(out).astype(np.float32)
    assert p.size == bpmf_mlp_param_count(n_in, width, depth)
    return p


def fit_norm(X: np.ndarray, t: np.ndarray) -> np.ndarray:
    sd = X.std(axis=0)
    sd = np.where(sd > 1e-6, sd, 1.0)
    ts = t.std() if t.std() > 1e-6 else 1.0
    return np.concatenate([X.mean(axis=0), sd, [t.mean(), ts]]).astype(np.float32)


def config_targets(logZ: np.ndarray, n_valid: np.ndarray) -> np.ndarray:
    """Per-configuration weight in the pooled sample mean summed over
    receptors: log sum_k S_jk (-inf when no translation is valid)."""
    with np.errstate(divide="ignore"):
        ls = np.where(n_valid > 0, logZ + np.log(np.maximum(n_valid, 1)), -np.inf)
    m = ls.max(axis=1, keepdims=True)
    with np.errstate(invalid="ignore", divide="ignore"):
        s = np.where(np.isfinite(m[:, 0]), m[:, 0] + np.log(np.exp(ls - np.where(np.isfinite(m), m, 0)).sum(1)),
                     -np.inf)
    return s


class LearnedProposal:
    """MLP n_in -> width x depth -> 1 held by the library (FP32 master weights,
    bf16 tensor-core GEMMs)."""

    def __init__(self, ctx, norm, n_in=BPMF_N_FEATURES, width=128, depth=3, seed=0):
        self.ctx, self.n_in, self.width, self.depth = ctx, n_in, width, depth
        self.mlp = bpmf_mlp_create(ctx, n_in, width, depth, init_params(n_in, width, depth, seed), norm)

    def fit(self, X, t, epochs=30, batch=256, lr=1e-3, seed=0):
        """X [N, n_in], t [N] float32 device tensors; finite targets only."""
        import torch
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        N = X.shape[0]
        for _ in range(epochs):
            perm = torch.randperm(N, generator=g).to(X.device)
            for i in range(0, N, batch):
                idx = perm[i:i + batch]
                losses.append(bpmf_mlp_train_step(self.ctx, self.mlp, X[idx].contiguous(), t[idx].contiguous(), lr))
        return losses

    def predict(self, X):
        import torch
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        bpmf_mlp_forward(self.ctx, self.mlp, X, y)
        return y

    def free(self):
        if self.mlp is not None:
            bpmf_mlp_free(self.mlp)
            self.mlp = None


def features(ctx, lig_handle, total_conf, h, device):
    import torch
    out = torch.empty((total_conf, BPMF_N_FEATURES), dtype=torch.float32, device=device)
    bpmf_features(ctx, lig_handle, h, out)
    return out


def proposal_bpmf(ctx, recs, kT, coords, params, pred, budget, mix=0.8, seed=0, mode=BPMF_MODE_FF,
                  n_tot=None, lig_full=None, stream=None):
    """Importance-sampled BPMF per receptor for one ligand.

    coords: device float32 [J, n_atoms, 3]; params: (q, eps, R) device float32
    [n_atoms]; pred: device float32 [J]; budget: number M of draws.  Returns
    (bpmf [K] numpy, drawn indices, q of the draws)."""
    import torch
    J, n_atoms = coords.shape[0], coords.shape[1]
    K = len(recs)
    dev = coords.device
    if n_tot is None:
        lh = lig_full if lig_full is not None else bpmf_ligand_batch(ctx, [n_atoms], [J], coords.reshape(-1, 3),
                                                                       *params, stream=stream)
        n_tot = bpmf_valid_counts(ctx, lh, recs, J).sum(axis=0)
        if lig_full is None:
            bpmf_ligand_free(lh)
    u = torch.from_numpy(np.random.default_rng(seed).random(budget)).to(dev)
    idx = torch.empty(budget, dtype=torch.int32, device=dev)
    q_s = torch.empty(budget, dtype=torch.float64, device=dev)
    bpmf_proposal_sample(ctx, pred, mix, u, idx, q_s, stream)
    sub = coords.index_select(0, idx.long()).reshape(-1, 3).contiguous()
    lh = bpmf_ligand_batch(ctx, [n_atoms], [budget], sub, *params, stream=stream)
    try:
        logZ = torch.empty((budget, K), dtype=torch.float64, device=dev)
        nv = torch.empty((budget, K), dtype=torch.int64, device=dev)
        bpmf_eval(ctx, lh, recs, kT, mode, logZ, nv, None, None, stream)
    finally:
        bpmf_ligand_free(lh)
    out = torch.empty(K, dtype=torch.float64, device=dev)
    bpmf_proposal_bpmf(ctx, logZ, nv, q_s, torch.from_numpy(np.asarray(n_tot, dtype=np.int64)).to(dev), kT, out,
                       stream)
    return out.cpu().numpy(), idx.cpu().numpy(), q_s.cpu().numpy()
