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
