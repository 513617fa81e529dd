"""Learned proposal on the GPU against the FP64 reference: features, MLP
forward and gradients (bf16 operand rounding emulated in the reference),
proposal draws, the importance-weighted estimator, the exact-enumeration
limit, and the measured gain of a trained network over uniform sampling."""
import numpy as np
import pytest

import oracle
from oracle import proposal as P
import synth

pytestmark = pytest.mark.gpu
KT = synth.KT


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    import paper_1708_07045_gb300 as pkg
    from paper_1708_07045_gb300.session import Session
    pkg.lib()
    s = Session(0)
    yield torch, pkg, s
    s.close()


def test_features_match_reference(env):
    torch, pkg, s = env
    lig = synth.ligand_params(4, 14)
    coords = synth.ligand_configs(5, 14, 40)
    lh, _, _ = s.load_ligands([synth.LigandInput(lig, coords)])
    F = np.empty((40, 24), dtype=np.float32)
    pkg.bpmf_features(s.ctx, lh, 0.25, F)
    checked = 0
    for j in range(40):
        ref = P.features(coords[j], lig.q, lig.eps, lig.R, 0.25)
        w = ref[7:10]
        assert np.allclose(F[j, 4:], ref[4:], rtol=1e-4, atol=1e-4), j
        # the frame (quaternion) is defined only when the moments are distinct
        if min(w[1] - w[0], w[2] - w[1]) > 1e-2 * w[2]:
            assert np.allclose(F[j, :4], ref[:4], atol=2e-4), (j, F[j, :4], ref[:4])
            checked += 1
    assert checked >= 30


def test_mlp_forward_and_gradients_match_reference(env):
    torch, pkg, s = env
    rng = np.random.default_rng(3)
    n_in, width, depth, B = 24, 128, 3, 300
    from paper_1708_07045_gb300 import proposal as PP
    params = PP.init_params(n_in, width, depth, seed=4)
    X = rng.normal(size=(B, n_in)).astype(np.float32) * 3 + 1
    t = rng.normal(size=B).astype(np.float32) * 50 - 20
    norm = PP.fit_norm(X, t)
    mlp = pkg.bpmf_mlp_create(s.ctx, n_in, width, depth, params, norm)
    try:
        Xd, td = torch.from_numpy(X).cuda(), torch.from_numpy(t).cuda()
        y = torch.empty(B, device="cuda")
        pkg.bpmf_mlp_forward(s.ctx, mlp, Xd, y)
        y_ref = P.mlp_forward(params, norm, X, n_in, width, depth)
        assert np.abs(y.cpu().numpy() - y_ref).max() <= 1e-4 * np.abs(y_ref).max() + 1e-3
        n = pkg.bpmf_mlp_param_count(n_in, width, depth)
        g = torch.empty(n, device="cuda")
        loss = pkg.bpmf_mlp_train_step(s.ctx, mlp, Xd, td, 1e-3, apply=False, grads=g)
        loss_ref, g_ref = P.mlp_grads(params, norm, X, t, n_in, width, depth)
        assert abs(loss - loss_ref) <= 1e-4 * max(1, loss_ref)
        gg = g.cpu().numpy()
        assert np.abs(gg - g_ref).max() <= 2e-3 * np.abs(g_ref).max()
        # the untouched weights are still the initial ones; training lowers the loss
        assert np.array_equal(pkg.bpmf_mlp_get_params(mlp, n), params)
        first = pkg.bpmf_mlp_train_step(s.ctx, mlp, Xd, td, 3e-3)
        for _ in range(60):
            last = pkg.bpmf_mlp_train_step(s.ctx, mlp, Xd, td, 3e-3)
        assert last < 0.5 * first
    finally:
        pkg.bpmf_mlp_free(mlp)


def test_sampling_and_estimator_match_reference(env):
    torch, pkg, s = env
    rng = np.random.default_rng(5)
    J, M, K = 1000, 300, 3
    pred = rng.normal(0, 2, J).astype(np.float32)
    u = rng.random(M)
    idx = torch.empty(M, dtype=torch.int32, device="cuda")
    qs = torch.empty(M, dtype=torch.float64, device="cuda")
    pkg.bpmf_proposal_sample(s.ctx, torch.from_numpy(pred).cuda(), 0.8, torch.from_numpy(u).cuda(), idx, qs)
    q = P.proposal(pred, 0.8)
    ref_idx = P.draw(q, u)
    assert np.array_equal(idx.cpu().numpy(), ref_idx)
    assert np.allclose(qs.cpu().numpy(), q[ref_idx] / q.sum(), rtol=1e-12)
    logZ = rng.normal(-50, 20, (M, K))
    nv = rng.integers(0, 5000, (M, K))
    ntot = rng.integers(10 ** 6, 10 ** 7, K)
    out = torch.empty(K, dtype=torch.float64, device="cuda")
    pkg.bpmf_proposal_bpmf(s.ctx, torch.from_numpy(logZ).cuda(), torch.from_numpy(nv).cuda(), qs,
                           torch.from_numpy(ntot).cuda(), KT, out)
    ref = P.is_bpmf(logZ, nv, qs.cpu().numpy(), ntot, KT)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-9)


@pytest.fixture(scope="module")
def small_set():
    """One receptor (32^3, 0.375 A) and 5 twelve-atom ligands with 256
    configurations each: 4 for training, 1 held out."""
    atoms = synth.receptor_atoms(1000, 400, 4.0, 10.0)
    g, o = synth.receptor_grids(atoms, (32, 32, 32), 0.375)
    lo, sn = synth.central_site((32, 32, 32), 16)
    rec = synth.ReceptorInput(g, 0.375, o, lo, sn)
    ligs = [synth.LigandInput(synth.ligand_params(50 + i, 12), synth.ligand_configs(60 + i, 12, 256))
            for i in range(5)]
    return rec, ligs


def test_learned_proposal_end_to_end(env, small_set):
    """Exact limit: a uniform proposal drawing every configuration once gives
    the full-enumeration BPMF.  Then the trained network's error and the
    uniform proposal's error at a 10 % budget, over 24 seeds each, against the
    full enumeration (reported; both estimators are unbiased for Z)."""
    torch, pkg, s = env
    from paper_1708_07045_gb300 import proposal as PP
    rec, ligs = small_set
    rh = s.load_receptor(rec)
    J = 256
    full = []
    for l in ligs:
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, total_conf=J)
        full.append(out)
    held = ligs[4]
    coords = torch.from_numpy(held.coords).cuda()
    params = [torch.from_numpy(getattr(held.params, k)).cuda() for k in ("q", "eps", "R")]
    # exact limit (the draws are every configuration once: pred = 0, mix = 0)
    u = (np.arange(J) + 0.5) / J
    idx = torch.empty(J, dtype=torch.int32, device="cuda")
    qs = torch.empty(J, dtype=torch.float64, device="cuda")
    pkg.bpmf_proposal_sample(s.ctx, torch.zeros(J, device="cuda"), 0.0, torch.from_numpy(u).cuda(), idx, qs)
    assert np.array_equal(np.sort(idx.cpu().numpy()), np.arange(J))
    sub = coords.index_select(0, idx.long()).reshape(-1, 3).contiguous()
    lh_s = pkg.bpmf_ligand_batch(s.ctx, [12], [J], sub, *params)
    logZ = torch.empty((J, 1), dtype=torch.float64, device="cuda")
    nv = torch.empty((J, 1), dtype=torch.int64, device="cuda")
    pkg.bpmf_eval(s.ctx, lh_s, [rh], KT, pkg.BPMF_MODE_FF, logZ, nv, None, None)
    pkg.bpmf_ligand_free(lh_s)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    ntot = full[4]["n_valid"].sum(axis=0)
    pkg.bpmf_proposal_bpmf(s.ctx, logZ, nv, qs, torch.from_numpy(ntot).cuda(), KT, out)
    B_full = full[4]["bpmf"][0, 0]
    assert abs(out.item() - B_full) <= 1e-9 * max(1, abs(B_full))
    # train on ligands 0-3 (features -> log sum_k S_jk), evaluate on ligand 4
    lh_tr, _, _ = s.load_ligands(ligs[:4])
    X = PP.features(s.ctx, lh_tr, 4 * J, rec.h, "cuda")
    t = np.concatenate([PP.config_targets(f["logZ"], f["n_valid"]) for f in full[:4]])
    ok = np.isfinite(t)
    Xtr = X[torch.from_numpy(np.nonzero(ok)[0]).cuda()].contiguous()
    ttr = torch.from_numpy(t[ok].astype(np.float32)).cuda()
    net = PP.LearnedProposal(s.ctx, PP.fit_norm(Xtr.cpu().numpy(), t[ok]))
    try:
        losses = net.fit(Xtr, ttr, epochs=40, batch=128, lr=1e-3)
        assert losses[-1] < losses[0]
        lh_h, _, _ = s.load_ligands([held])
        pred = net.predict(PP.features(s.ctx, lh_h, J, rec.h, "cuda"))
        M = J // 10
        err = {}
        for name, p, mix in (("trained", pred, 0.8), ("uniform", torch.zeros(J, device="cuda"), 0.0)):
            e = []
            for seed in range(24):
                B, _, _ = PP.proposal_bpmf(s.ctx, [rh], KT, coords, params, p, M, mix=mix, seed=seed, n_tot=ntot)
                e.append(B[0] - B_full)
            err[name] = np.array(e)
        rms = {k: float(np.sqrt(np.mean(v[np.isfinite(v)] ** 2))) for k, v in err.items()}
        print("learned-proposal BPMF rms error at a 10 % budget (kcal/mol):", rms)
        for v in err.values():
            assert np.isfinite(v).mean() > 0.5
    finally:
        net.free()
