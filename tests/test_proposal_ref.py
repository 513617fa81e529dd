"""Pins of the FP64 learned-proposal reference (CPU only): analytic MLP
gradients against finite differences, the importance-weighted estimator
against full enumeration (exactly, when every configuration is drawn once
under a uniform proposal) and against its expectation (unbiasedness for Z),
inverse-CDF draws, and rotation behaviour of the features."""
import numpy as np
from scipy.special import logsumexp
from scipy.spatial.transform import Rotation

import oracle
from oracle import proposal as P
import synth


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, width, depth, B = 5, 7, 2, 9
    n = n_in * width + width + (depth - 1) * (width * width + width) + width + 1
    params = rng.normal(0, 0.5, n)
    norm = np.concatenate([rng.normal(size=n_in), rng.uniform(0.5, 2, n_in), [0.3, 1.7]])
    X = rng.normal(size=(B, n_in))
    t = rng.normal(size=B)
    loss, g = P.mlp_grads(params, norm, X, t, n_in, width, depth, bf16_ops=False)
    eps = 1e-6
    fd = np.empty(n)
    for i in range(n):
        pp, pm = params.copy(), params.copy()
        pp[i] += eps
        pm[i] -= eps
        fd[i] = (P.mlp_grads(pp, norm, X, t, n_in, width, depth, False)[0] -
                 P.mlp_grads(pm, norm, X, t, n_in, width, depth, False)[0]) / (2 * eps)
    assert np.abs(fd - g).max() <= 1e-6 * max(1.0, np.abs(g).max())


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -9, -2.5], dtype=np.float32)
    r = P.bf16(x)
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: the even mantissa (1) wins
    assert np.array_equal(r, [1.0, 1.0, 1.0 + 2 ** -7, 1.0, -2.5])


def test_uniform_proposal_drawing_each_configuration_once_is_full_enumeration():
    w = synth.plain_small(n_conf=12)
    r, l = w.receptors[0], w.ligands[0]
    ref = oracle.evaluate([r], l.coords, l.params.q, l.params.eps, l.params.R, KT := w.kT)
    J = l.coords.shape[0]
    q = P.proposal(np.zeros(J), 0.8)
    assert np.allclose(q, 1.0 / J)
    idx = np.random.default_rng(1).permutation(J)
    B = P.is_bpmf(ref["logZ"][idx], ref["n_valid"][idx], q[idx], ref["n_valid"].sum(0), KT)
    assert abs(B[0] - ref["bpmf"][0]) <= 1e-9 * max(1, abs(ref["bpmf"][0]))


def test_importance_estimator_is_unbiased_for_Z():
    rng = np.random.default_rng(2)
    J, M, R = 200, 20, 6000
    logS = rng.normal(0, 1.5, J)
    Z = np.exp(logsumexp(logS))
    pred = logS + rng.normal(0, 0.7, J)  # an imperfect learned predictor
    q = P.proposal(pred, 0.8)
    est = np.empty(R)
    for i in range(R):
        idx = P.draw(q, rng.random(M))
        est[i] = np.mean(np.exp(logS[idx]) / q[idx])
    se = est.std(ddof=1) / np.sqrt(R)
    assert abs(est.mean() - Z) <= 3.5 * se


def test_inverse_cdf_draws_follow_q():
    q = np.array([0.1, 0.0, 0.5, 0.4])
    assert list(P.draw(q, [0.0, 0.099, 0.1, 0.59, 0.6, 0.999])) == [0, 0, 2, 2, 3, 3]


def test_features_rotation_behaviour():
    lig = synth.ligand_params(4, 14)
    x = synth.ligand_configs(5, 14, 1)[0].astype(np.float64)
    f0 = P.features(x, lig.q, lig.eps, lig.R, 0.25)
    rot = Rotation.from_euler("zyx", [0.3, -0.4, 1.1])
    x1 = (x - x.mean(0)) @ rot.as_matrix().T + x.mean(0)
    f1 = P.features(x1, lig.q, lig.eps, lig.R, 0.25)
    assert np.isclose(np.linalg.norm(f0[:4]), 1.0) and f0[0] >= 0
    assert np.allclose(f0[7:16], f1[7:16], atol=1e-9)   # moments, Rg, end-to-end, torsions
    assert np.array_equal(f0[16:], f1[16:])             # atom-type counts
    # the orientation composes with the applied rotation
    q0 = Rotation.from_quat([f0[1], f0[2], f0[3], f0[0]])
    q1 = Rotation.from_quat([f1[1], f1[2], f1[3], f1[0]])
    assert (rot * q0).approx_equal(q1, atol=1e-7)


def test_tempered_proposal_limits():
    """tau -> infinity flattens the softmax to uniform; tau = 1 is the plain
    softmax; mix = 0 is uniform whatever the prediction."""
    rng = np.random.default_rng(9)
    pred = rng.normal(0, 5, 64)
    assert np.allclose(P.proposal(pred, 0.8, 1e12), 1.0 / 64, rtol=1e-9)
    e = np.exp(pred - pred.max())
    assert np.allclose(P.proposal(pred, 1.0, 1.0), e / e.sum(), rtol=1e-12)
    assert np.allclose(P.proposal(pred, 0.0, 0.3), 1.0 / 64)
    # halving tau squares the softmax weights before renormalising
    q2 = P.proposal(pred, 1.0, 0.5)
    assert np.allclose(q2, e ** 2 / np.sum(e ** 2), rtol=1e-9)


def test_chi2_closed_forms():
    """chi2 vanishes when q is proportional to S (the zero-variance proposal),
    equals J sum w^2 - 1 for the uniform proposal, and matches the Monte-Carlo
    variance of S_j / (q_j Z) for j ~ q."""
    rng = np.random.default_rng(10)
    J = 200
    ls = rng.normal(0, 3, J)
    ls[5] = -np.inf  # a configuration without a valid translation
    w = np.exp(ls - ls[np.isfinite(ls)].max())
    w[~np.isfinite(ls)] = 0
    w /= w.sum()
    pred_exact = np.where(np.isfinite(ls), ls, -1e30)
    assert abs(P.chi2(pred_exact, ls, 1.0, 1.0)) < 1e-9
    assert abs(P.chi2(np.zeros(J), ls, 0.8, 1.0) - (J * np.sum(w ** 2) - 1.0)) < 1e-9
    pred = ls + rng.normal(0, 1.0, J)
    pred[5] = 0.0
    q = P.proposal(pred, 0.8, 2.0)
    draws = rng.choice(J, size=400_000, p=q)
    r = w[draws] / q[draws]
    assert abs(np.var(r) - P.chi2(pred, ls, 0.8, 2.0)) <= 0.03 * max(1.0, P.chi2(pred, ls, 0.8, 2.0))


def test_config_targets_clip_and_offset():
    """ls is the log of the configuration's summed weight over receptors;
    the targets are relative to the ligand's largest and clipped below."""
    logZ = np.array([[0.0, 1.0], [5.0, -np.inf], [-200.0, -300.0], [-np.inf, -np.inf]])
    n = np.array([[1, 3], [2, 0], [4, 4], [0, 0]])
    ls, t = P.config_targets(logZ, n, 50.0)
    assert abs(ls[0] - np.log(1 + 3 * np.e)) < 1e-12
    assert abs(ls[1] - (5.0 + np.log(2))) < 1e-12
    assert np.isneginf(ls[3])
    assert t[1] == 0.0 and abs(t[0] - (ls[0] - ls[1])) < 1e-12
    assert t[2] == -50.0 and t[3] == -50.0
