"""Dominant-state outputs and pose resampling on the GPU against the FP64
oracle, through the C ABI.

* psi_min (minimum energy over the valid translations of every configuration
  and receptor) and psi_dom (per receptor minimum, minimum over receptors,
  exponential average): 1e-3 kcal/mol, the energy tolerance (a minimum lies
  inside every 20 kT window);
* bpmf_eval_dominant leaves logZ, n_valid, BPMF and dG bit-identical to
  bpmf_eval;
* resampled poses: with the same FP64 inputs (the library's log Z and
  energies) the draws equal the oracle's wherever the uniform is not within
  1e-9 of a cumulative-weight boundary (summation order differs); against the
  oracle's own energies they agree wherever the uniform is further from a
  boundary than the weight error that 1e-3 kcal/mol allows.
"""
import numpy as np
import pytest

import oracle
from oracle import sampling as S
import synth

pytestmark = pytest.mark.gpu

KT = synth.KT
E_TOL = 1e-3


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


@pytest.fixture(scope="module")
def case():
    """Two receptors on the 32^3 grid (the second with scaled grids) and two
    twelve-atom ligands of 48 and 40 configurations."""
    w = synth.plain_small(n_conf=48)
    r0 = w.receptors[0]
    r1 = synth.ReceptorInput((r0.grids * np.float32(0.7)).astype(np.float32), r0.h, r0.origin, r0.site_lo,
                             r0.site_n)
    ligs = [w.ligands[0], synth.LigandInput(synth.ligand_params(77, 12), synth.ligand_configs(78, 12, 40))]
    refs = [oracle.evaluate([r0, r1], l.coords, l.params.q, l.params.eps, l.params.R, KT) for l in ligs]
    return [r0, r1], ligs, refs


def _margin(p, u):
    """Distance of each u from the nearest boundary of the cumulative
    probabilities p (normalised)."""
    c = np.concatenate([[0.0], np.cumsum(p)])
    c /= c[-1]
    return np.min(np.abs(np.asarray(u)[:, None] - c[None, :]), axis=1)


def test_dominant_outputs_match_oracle(env, case):
    torch, pkg, s = env
    recs, ligs, refs = case
    rh = [s.load_receptor(r) for r in recs]
    lh, _, n_conf = s.load_ligands(ligs)
    T = sum(n_conf)
    _, base = s.eval(lh, rh, KT, pkg.BPMF_MODE_FF, n_lig=2, total_conf=T)
    out = {"logZ": np.empty((T, 2)), "n_valid": np.empty((T, 2), dtype=np.int64), "bpmf": np.empty((2, 2)),
           "dG": np.empty(2)}
    pmin = np.empty((T, 2))
    pdom = np.empty((2, 4))
    pkg.bpmf_eval_dominant(s.ctx, lh, rh, KT, pkg.BPMF_MODE_FF, out["logZ"], out["n_valid"], out["bpmf"],
                           out["dG"], pmin, pdom)
    for k in base:
        assert np.array_equal(out[k], base[k]), k
    o = 0
    for li, ref in enumerate(refs):
        J = n_conf[li]
        got = pmin[o:o + J]
        fin = np.isfinite(ref["Emin"])
        assert np.array_equal(np.isfinite(got), fin)
        assert np.abs(got[fin] - ref["Emin"][fin]).max() <= E_TOL
        d_ref = S.dominant(ref["Emin"], KT)
        assert np.abs(pdom[li] - d_ref).max() <= E_TOL, (pdom[li], d_ref)
        o += J
    # psi_dom alone, in device memory
    pd = torch.empty((2, 4), dtype=torch.float64, device="cuda")
    lz = torch.empty((T, 2), dtype=torch.float64, device="cuda")
    pkg.bpmf_eval_dominant(s.ctx, lh, rh, KT, pkg.BPMF_MODE_FF, lz, None, None, None, None, pd)
    torch.cuda.synchronize()
    assert np.array_equal(pd.cpu().numpy(), pdom)
    with pytest.raises(pkg.BpmfError):
        pkg.bpmf_eval_dominant(s.ctx, lh, rh, KT, pkg.BPMF_MODE_FF, lz, None, None, None, None, None)


def _sir(torch, pkg, s, lh, li, rh_k, K, k, logZ, nv, u1, u2):
    M = len(u1)
    conf = torch.empty(M, dtype=torch.int32, device="cuda")
    pose = torch.empty(M, dtype=torch.int32, device="cuda")
    pkg.bpmf_sir_poses(s.ctx, lh, li, rh_k, k, KT, pkg.BPMF_MODE_FF, logZ, nv, torch.from_numpy(u1).cuda(),
                       torch.from_numpy(u2).cuda(), conf, pose)
    return conf.cpu().numpy(), pose.cpu().numpy()


def test_sir_draws_match_oracle(env, case):
    torch, pkg, s = env
    recs, ligs, refs = case
    rh = [s.load_receptor(r) for r in recs]
    lig, ref = ligs[0], refs[0]
    lh, _, _ = s.load_ligands([lig])
    J, K, M = lig.coords.shape[0], 2, 300
    logZ = torch.empty((J, K), dtype=torch.float64, device="cuda")
    nv = torch.empty((J, K), dtype=torch.int64, device="cuda")
    pkg.bpmf_eval(s.ctx, lh, rh, KT, pkg.BPMF_MODE_FF, logZ, nv, None, None)
    lz, n = logZ.cpu().numpy(), nv.cpu().numpy()
    rng = np.random.default_rng(11)
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    for k in range(K):
        u1, u2 = rng.random(M), rng.random(M)
        conf, pose = _sir(torch, pkg, s, lh, 0, rh[k], K, k, logZ, nv, u1, u2)
        assert np.all(conf >= 0) and np.all(pose >= 0)
        # (1) the same FP64 inputs: the library's log S and energies
        with np.errstate(divide="ignore"):
            logS_gpu = np.where(n[:, k] > 0, lz[:, k] + np.log(np.maximum(n[:, k], 1)), -np.inf)
        c_ref = S.sir_configs(logS_gpu, u1)
        far = _margin(S.config_weights(logS_gpu), u1) > 1e-9
        assert np.array_equal(conf[far], c_ref[far])
        E_gpu = {}
        for j in np.unique(conf):
            E_gpu[j] = s.export_energies(lh, rh[k], 0, int(j), recs[k].site_n).ravel()
            sel = conf == j
            t_ref = S.sir_translations(E_gpu[j], KT, u2[sel])
            far_t = _margin(S.translation_weights(E_gpu[j], KT), u2[sel]) > 1e-9
            assert np.array_equal(pose[sel][far_t], t_ref[far_t])
            assert np.all(np.isfinite(E_gpu[j][pose[sel]]))
        # (2) the oracle's own FP64 log S and pose energies
        w_tol = 4 * E_TOL / KT  # relative weight error bound, summed
        c_or = S.sir_configs(ref["logS"][:, k], u1)
        far = _margin(S.config_weights(ref["logS"][:, k]), u1) > w_tol
        assert far.mean() > 0.5
        assert np.array_equal(conf[far], c_or[far])
        for j in np.unique(conf[far]):
            E_or, _ = oracle.pose_energies(recs[k].grids, recs[k].h, recs[k].site_lo, recs[k].site_n,
                                           lig.coords[j], gam)
            E_or = E_or.ravel()
            sel = far & (conf == j)
            t_or = S.sir_translations(E_or, KT, u2[sel])
            far_t = _margin(S.translation_weights(E_or, KT), u2[sel]) > w_tol
            assert np.array_equal(pose[sel][far_t], t_or[far_t])
            assert np.all(np.isfinite(E_or[pose[sel]]))


def test_sir_stratified_draws_follow_weights(env, case):
    """Stratified uniforms: every configuration is drawn within one of M p_j
    times, p_j = S_j / sum S from the library's log Z."""
    torch, pkg, s = env
    recs, ligs, _ = case
    rh = s.load_receptor(recs[0])
    lh, _, _ = s.load_ligands([ligs[1]])
    J, M = ligs[1].coords.shape[0], 4000
    logZ = torch.empty((J, 1), dtype=torch.float64, device="cuda")
    nv = torch.empty((J, 1), dtype=torch.int64, device="cuda")
    pkg.bpmf_eval(s.ctx, lh, [rh], KT, pkg.BPMF_MODE_FF, logZ, nv, None, None)
    lz, n = logZ.cpu().numpy()[:, 0], nv.cpu().numpy()[:, 0]
    u1 = (np.arange(M) + 0.5) / M
    conf, pose = _sir(torch, pkg, s, lh, 0, rh, 1, 0, logZ, nv, u1, np.random.default_rng(2).random(M))
    p = S.config_weights(np.where(n > 0, lz + np.log(np.maximum(n, 1)), -np.inf))
    assert np.all(np.abs(np.bincount(conf, minlength=J) - M * p) <= 1.0 + 1e-6)


def test_sir_no_valid_pose_and_bad_arguments(env, case):
    torch, pkg, s = env
    recs, ligs, _ = case
    rh = s.load_receptor(recs[0])
    big = synth.LigandInput(ligs[0].params, (ligs[0].coords[:4] * 8.0).astype(np.float32))
    lh, _, _ = s.load_ligands([big])
    logZ = torch.empty((4, 1), dtype=torch.float64, device="cuda")
    nv = torch.empty((4, 1), dtype=torch.int64, device="cuda")
    rc = pkg.bpmf_eval(s.ctx, lh, [rh], KT, pkg.BPMF_MODE_FF, logZ, nv, None, None)
    assert rc == pkg.BPMF_WARN_NO_VALID and int(nv.sum()) == 0
    conf, pose = _sir(torch, pkg, s, lh, 0, rh, 1, 0, logZ, nv, np.array([0.1, 0.9]), np.array([0.5, 0.5]))
    assert np.all(conf == -1) and np.all(pose == -1)
    with pytest.raises(pkg.BpmfError):  # host memory is refused
        pkg.bpmf_sir_poses(s.ctx, lh, 0, rh, 0, KT, pkg.BPMF_MODE_FF, logZ.cpu(), nv, torch.zeros(2).double().cuda(),
                           torch.zeros(2).double().cuda(), torch.empty(2, dtype=torch.int32, device="cuda"),
                           torch.empty(2, dtype=torch.int32, device="cuda"))
    with pytest.raises(pkg.BpmfError):  # receptor column out of range
        pkg.bpmf_sir_poses(s.ctx, lh, 0, rh, 1, KT, pkg.BPMF_MODE_FF, logZ, nv, torch.zeros(2).double().cuda(),
                           torch.zeros(2).double().cuda(), torch.empty(2, dtype=torch.int32, device="cuda"),
                           torch.empty(2, dtype=torch.int32, device="cuda"))


def test_bootstrap_matches_oracle(env, case):
    """Bootstrap replicates of B_k and dG: with the library's own log Z the
    replicates equal the FP64 reference to rounding; against the oracle's log
    S they stay within the BPMF tolerance; the identity replicate reproduces
    bpmf_eval's BPMF and dG."""
    torch, pkg, s = env
    recs, ligs, refs = case
    rh = [s.load_receptor(r) for r in recs]
    lig, ref = ligs[0], refs[0]
    lh, _, _ = s.load_ligands([lig])
    J, K, R = lig.coords.shape[0], 2, 200
    logZ = torch.empty((J, K), dtype=torch.float64, device="cuda")
    nv = torch.empty((J, K), dtype=torch.int64, device="cuda")
    B = torch.empty((1, K), dtype=torch.float64, device="cuda")
    dG = torch.empty(1, dtype=torch.float64, device="cuda")
    pkg.bpmf_eval(s.ctx, lh, rh, KT, pkg.BPMF_MODE_FF, logZ, nv, B, dG)
    u = np.random.default_rng(21).random((R, J))
    u[0] = (np.arange(J) + 0.5) / J  # identity replicate
    rep = torch.empty((R, K + 1), dtype=torch.float64, device="cuda")
    stats = torch.empty((2, K + 1), dtype=torch.float64, device="cuda")
    pkg.bpmf_bootstrap(s.ctx, logZ, nv, KT, recs[0].h, torch.from_numpy(u).cuda(), rep, stats)
    rep_, stats_ = rep.cpu().numpy(), stats.cpu().numpy()
    lz, n = logZ.cpu().numpy(), nv.cpu().numpy()
    with np.errstate(divide="ignore"):
        logS = np.where(n > 0, lz + np.log(np.maximum(n, 1)), -np.inf)
    r_ref, s_ref = S.bootstrap(logS, n, KT, recs[0].h, u)
    assert np.allclose(rep_, r_ref, rtol=1e-12, atol=1e-9)
    assert np.allclose(stats_, s_ref, rtol=1e-9, atol=1e-9)
    assert np.allclose(rep_[0, :K], B.cpu().numpy()[0], rtol=1e-12, atol=1e-9)
    assert abs(rep_[0, K] - dG.item()) <= 1e-9
    r_or, s_or = S.bootstrap(ref["logS"], ref["n_valid"], KT, recs[0].h, u)
    assert np.abs(rep_ - r_or).max() <= 1e-2
    assert np.all(stats_[1] > 0)
