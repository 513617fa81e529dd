"""Learned-proposal workflow over the C entry points (argument marshalling and
loops only; features, the MLP, sampling and the estimator run in the library's
kernels).

Flow for one ligand with J configurations against K receptors:
  features (bpmf_features) -> prediction (bpmf_mlp_forward) ->
  q = mix softmax(pred / tau) + (1 - mix)/J and M draws (bpmf_proposal_sample,
  on uniforms from a seeded numpy generator) -> bpmf_eval on the drawn
  configurations -> importance-weighted BPMF (bpmf_proposal_bpmf) with the
  valid-translation totals of all J configurations (bpmf_valid_counts).
Training: fully enumerated ligands give each configuration's log weight
relative to its ligand's largest, clipped below (bpmf_config_targets); the
temperature tau is the one whose exact importance-sampling variance
(bpmf_proposal_chi2) is lowest on held-out, fully enumerated ligands.
"""
from __future__ import annotations

import numpy as np

from . import (BPMF_MODE_FF, BPMF_N_FEATURES, bpmf_config_targets, bpmf_eval, bpmf_features, bpmf_ligand_batch,
               bpmf_ligand_free, bpmf_mlp_create, bpmf_mlp_forward, bpmf_mlp_free, bpmf_mlp_param_count,
               bpmf_mlp_train_step, bpmf_proposal_bpmf, bpmf_proposal_chi2, bpmf_proposal_sample, bpmf_valid_counts)

TARGET_CLIP = 50.0  # training targets: log weight relative to the ligand's largest, clipped at -50
TAUS = (0.25, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0)


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


def config_targets(ctx, logZ, n_valid, clip=TARGET_CLIP):
    """One ligand's (ls, t) on the device: ls [J] float64, each configuration's
    log weight ln sum_k S_jk; t [J] float32, the training target
    max(ls - max ls, -clip) (bpmf_config_targets)."""
    import torch
    lz = torch.as_tensor(logZ, dtype=torch.float64).cuda().contiguous()
    nv = torch.as_tensor(n_valid, dtype=torch.int64).cuda().contiguous()
    J = lz.shape[0]
    ls = torch.empty(J, dtype=torch.float64, device="cuda")
    t = torch.empty(J, dtype=torch.float32, device="cuda")
    bpmf_config_targets(ctx, lz, nv, clip, ls, t)
    return ls, t


def proposal_chi2(ctx, pred, ls, mix, tau) -> float:
    """Exact relative variance of one importance-sampling draw (bpmf_proposal_chi2)."""
    import torch
    out = torch.empty(1, dtype=torch.float64, device=pred.device)
    bpmf_proposal_chi2(ctx, pred, ls, mix, tau, out)
    return float(out.item())


def choose_tau(ctx, preds, lss, mix=0.8, taus=TAUS):
    """The temperature with the lowest mean log(1 + chi2) over fully
    enumerated validation ligands (preds, lss: per-ligand device tensors)."""
    best = None
    for tau in taus:
        v = float(np.mean([np.log1p(proposal_chi2(ctx, p, l, mix, tau)) for p, l in zip(preds, lss)]))
        if best is None or v < best[0]:
            best = (v, tau)
    return best[1]


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
                  n_tot=None, lig_full=None, stream=None, tau=1.0):
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
    bpmf_proposal_sample(ctx, pred, mix, u, idx, q_s, stream, tau=tau)
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
