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
    # tempered: q = mix softmax(pred / tau) + (1 - mix) / J
    idx_t = torch.empty(M, dtype=torch.int32, device="cuda")
    qs_t = torch.empty(M, dtype=torch.float64, device="cuda")
    pkg.bpmf_proposal_sample(s.ctx, torch.from_numpy(pred).cuda(), 0.8, torch.from_numpy(u).cuda(), idx_t, qs_t,
                             tau=3.5)
    q_t = P.proposal(pred, 0.8, 3.5)
    ref_t = P.draw(q_t, u)
    # the same draws wherever u is not at a CDF boundary (FP64 sums in another order)
    cdf = np.cumsum(q_t) / q_t.sum()
    away = np.min(np.abs(u[:, None] - cdf[None, :]), axis=1) > 1e-12
    assert np.array_equal(idx_t.cpu().numpy()[away], ref_t[away])
    assert np.allclose(qs_t.cpu().numpy()[away], (q_t[ref_t] / q_t.sum())[away], rtol=1e-12)
    logZ = rng.normal(-50, 20, (M, K))
    nv = rng.integers(0, 5000, (M, K))
    ntot = rng.integers(10 ** 6, 10 ** 7, K)
    out = torch.empty(K, dtype=torch.float64, device="cuda")
    pkg.bpmf_proposal_bpmf(s.ctx, torch.from_numpy(logZ).cuda(), torch.from_numpy(nv).cuda(), qs,
                           torch.from_numpy(ntot).cuda(), KT, out)
    ref = P.is_bpmf(logZ, nv, qs.cpu().numpy(), ntot, KT)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-9)


def test_config_targets_and_chi2_match_reference(env):
    torch, pkg, s = env
    from paper_1708_07045_gb300 import proposal as PP
    rng = np.random.default_rng(11)
    J, K = 700, 3
    logZ = rng.normal(-300, 120, (J, K))
    nv = rng.integers(0, 4000, (J, K))
    nv[17] = 0  # no valid translation against any receptor
    ls, t = PP.config_targets(s.ctx, logZ, nv, 50.0)
    ls_ref, t_ref = P.config_targets(logZ, nv, 50.0)
    lsv = ls.cpu().numpy()
    assert np.array_equal(np.isfinite(lsv), np.isfinite(ls_ref))
    fin = np.isfinite(ls_ref)
    assert np.allclose(lsv[fin], ls_ref[fin], rtol=1e-13, atol=1e-10)
    assert np.allclose(t.cpu().numpy(), t_ref.astype(np.float32), rtol=1e-6, atol=1e-5)
    pred = (ls_ref + rng.normal(0, 20, J)).astype(np.float32)
    pred[~fin] = 0.0
    pd = torch.from_numpy(pred).cuda()
    for mix, tau in ((0.8, 1.0), (0.8, 7.0), (0.5, 0.3), (0.0, 1.0)):
        got = PP.proposal_chi2(s.ctx, pd, ls, mix, tau)
        want = P.chi2(pred, ls_ref, mix, tau)
        assert abs(got - want) <= 1e-9 * max(1.0, abs(want)), (mix, tau, got, want)


@pytest.fixture(scope="module")
def small_set():
    """One receptor (32^3, 0.375 A) and ten twelve-atom ligands with 512
    configurations each: 6 to train on, 2 to choose the temperature, 2 held out."""
    atoms = synth.receptor_atoms(1000, 400, 4.0, 10.0)
    g, o = synth.receptor_grids(atoms, (32, 32, 32), 0.375)
    lo, sn = synth.central_site((32, 32, 32), 16)
    rec = synth.ReceptorInput(g, 0.375, o, lo, sn)
    ligs = [synth.LigandInput(synth.ligand_params(50 + i, 12), synth.ligand_configs(60 + i, 12, 512))
            for i in range(10)]
    return rec, ligs


def test_learned_proposal_end_to_end(env, small_set):
    """Exact limit: a uniform proposal drawing every configuration once gives
    the full-enumeration BPMF.  Then the trained, tempered proposal against
    uniform sampling on two held-out ligands, judged by the exact variance of
    the importance-sampling estimate (chi2 from the full enumeration, no
    sampling noise): on this workload the configurations' weights span
    hundreds of kT and one configuration carries nearly all of Z, so the gain
    is the network's ability to rank that configuration high.  The trained
    proposal must lower chi2 (geometric mean over the held-out ligands) below
    uniform's; the sampled BPMF errors at a 10 % budget are reported."""
    torch, pkg, s = env
    from paper_1708_07045_gb300 import proposal as PP
    rec, ligs = small_set
    rh = s.load_receptor(rec)
    J = 512
    full = []
    for l in ligs:
        lh, _, _ = s.load_ligands([l])
        _, out = s.eval(lh, [rh], KT, pkg.BPMF_MODE_FF, total_conf=J)
        full.append(out)
    held = ligs[9]
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
    ntot = full[9]["n_valid"].sum(axis=0)
    pkg.bpmf_proposal_bpmf(s.ctx, logZ, nv, qs, torch.from_numpy(ntot).cuda(), KT, out)
    B_full = full[9]["bpmf"][0, 0]
    assert abs(out.item() - B_full) <= 1e-9 * max(1, abs(B_full))
    # targets of every ligand, features, training on ligands 0-5
    tg = [PP.config_targets(s.ctx, f["logZ"], f["n_valid"]) for f in full]
    feats = []
    for l in ligs:
        lh, _, _ = s.load_ligands([l])
        feats.append(PP.features(s.ctx, lh, J, rec.h, "cuda"))
    Xtr = torch.cat(feats[:6]).contiguous()
    ttr = torch.cat([t for _, t in tg[:6]]).contiguous()
    net = PP.LearnedProposal(s.ctx, PP.fit_norm(Xtr.cpu().numpy(), ttr.cpu().numpy()))
    try:
        losses = net.fit(Xtr, ttr, epochs=60, batch=128, lr=1e-3)
        assert losses[-1] < losses[0]
        preds = [net.predict(f) for f in feats]
        tau = PP.choose_tau(s.ctx, preds[6:8], [ls for ls, _ in tg[6:8]])
        zero = torch.zeros(J, device="cuda")
        c_tr = [PP.proposal_chi2(s.ctx, preds[i], tg[i][0], 0.8, tau) for i in (8, 9)]
        c_un = [PP.proposal_chi2(s.ctx, zero, tg[i][0], 0.8, tau) for i in (8, 9)]
        gm = lambda v: float(np.exp(np.mean(np.log1p(v))))
        # sampled BPMF errors at a 10 % budget (reported)
        M = J // 10
        err = {}
        for name, p, mix in (("trained", preds[9], 0.8), ("uniform", zero, 0.0)):
            e = [PP.proposal_bpmf(s.ctx, [rh], KT, coords, params, p, M, mix=mix, seed=seed, n_tot=ntot,
                                  tau=tau)[0][0] - B_full for seed in range(16)]
            err[name] = float(np.median(np.abs(e)))
        print(f"learned proposal: tau {tau}, chi2 trained {c_tr} vs uniform {c_un}; "
              f"median |dB| at a 10 % budget trained {err['trained']:.3g} vs uniform {err['uniform']:.3g} kcal/mol")
        assert gm(c_tr) < gm(c_un)
    finally:
        net.free()
