"""Pins of the dominant-state and pose-resampling oracle (``oracle.sampling``)
to brute force, closed forms and exact identities (CPU only)."""
import itertools

import numpy as np
from scipy.special import logsumexp

import oracle
from oracle import sampling as S
import synth

KT = 0.5925


def _single_atom_case():
    w = synth.plain_small(n_conf=1)
    r = w.receptors[0]
    xyz = np.array([[1.234, -0.5, 2.0]], dtype=np.float32)
    lig = synth.ligand_params(7, 1)
    gam = oracle.gamma(lig.q, lig.eps, lig.R)
    return r, xyz, gam


def test_emin_is_brute_force_minimum_and_bounds_logS():
    """One atom on the nodes: the minimum over valid translations is the
    minimum of the summed grid values over the nodes the atom can occupy."""
    r, xyz, gam = _single_atom_case()
    logS, n, emin = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, xyz[None], gam, KT)
    N = np.array(r.shape)
    vals = []
    for m in itertools.product(*[range(v) for v in N]):
        m = np.array(m)
        if np.all(m + 4 <= N - 1) and np.all(m + 2 >= r.site_lo) and np.all(m + 2 < np.array(r.site_lo) + r.site_n):
            vals.append(sum(gam[t, 0] * float(r.grids[(t,) + tuple(m + 2)]) for t in range(3)))
    assert abs(emin[0] - min(vals)) <= 1e-9 * max(1, abs(min(vals)))
    # exp(-E_min/kT) <= S <= n exp(-E_min/kT)
    assert -emin[0] / KT - 1e-9 <= logS[0] <= -emin[0] / KT + np.log(n[0]) + 1e-9


def test_emin_of_many_atoms_matches_pose_energies():
    w = synth.plain_small(n_conf=3)
    r, lig = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    _, _, emin = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, lig.coords, gam, KT)
    for j in range(3):
        E, _ = oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, lig.coords[j], gam)
        assert emin[j] == E[np.isfinite(E)].min()


def test_dominant_combinations_closed_forms():
    rng = np.random.default_rng(0)
    E = rng.normal(-5, 3, (7, 4))
    E[2, 1] = np.inf
    d = S.dominant(E, KT)
    per = d[:4]
    # per-receptor minimum over configurations, brute force
    for k in range(4):
        assert per[k] == min(E[j, k] for j in range(7))
    assert d[4] == per.min()
    # exponential average: between the minimum and minimum + kT ln K, shifts
    # with a constant offset, equals the common value when all agree
    assert d[4] <= d[5] <= d[4] + KT * np.log(4) + 1e-12
    assert abs(S.dominant(E + 3.0, KT)[5] - (d[5] + 3.0)) <= 1e-12
    same = np.full((3, 5), -2.5)
    assert abs(S.dominant(same, KT)[5] + 2.5) <= 1e-12
    assert S.dominant(E[:, :1], KT)[2] == per[0]
    assert np.all(np.isinf(S.dominant(np.full((2, 3), np.inf), KT)))
    # K = 2 against the two-term log-sum-exp
    a, b = -3.0, -1.0
    ref = -KT * (logsumexp([-a / KT, -b / KT]) - np.log(2))
    assert abs(S.dominant(np.array([[a, b]]), KT)[3] - ref) <= 1e-12


def test_inverse_cdf_stratified_counts_follow_weights():
    """With stratified uniforms u_i = (i + 1/2)/N the inverse CDF draws index
    t within one of N p_t times; zero weights are never
    drawn; lower energies are drawn more often (the sign of the exponent)."""
    rng = np.random.default_rng(1)
    E = rng.normal(0, 1.0, 40)
    E[[3, 17, 30]] = np.inf
    p = np.where(np.isfinite(E), np.exp(-E / KT), 0.0)
    p /= p.sum()
    N = 100000
    u = (np.arange(N) + 0.5) / N
    idx = S.sir_translations(E, KT, u)
    cnt = np.bincount(idx, minlength=40)
    assert np.all(cnt[[3, 17, 30]] == 0)
    assert np.all(np.abs(cnt - N * p) <= 1.0 + 1e-9)
    fin = np.isfinite(E)
    assert np.argmax(cnt) == np.argmin(np.where(fin, E, np.inf))


def test_inverse_cdf_edges():
    w_E = np.array([np.inf, 1.0, np.inf, 2.0, np.inf])
    assert S.sir_translations(w_E, KT, [0.0])[0] == 1
    assert S.sir_translations(w_E, KT, [np.nextafter(1.0, 0.0)])[0] == 3
    assert np.all(S.sir_translations(np.full(4, np.inf), KT, [0.2, 0.7]) == -1)
    assert np.all(S.sir_configs(np.full(3, -np.inf), [0.5]) == -1)
    # u = 0 skips leading zero weights of configurations too
    assert S.sir_configs(np.array([-np.inf, -np.inf, 0.0, 1.0]), [0.0])[0] == 2


def test_two_stage_draw_is_the_flat_pose_distribution():
    """P(configuration j) P(translation t | j) from log S and the pose
    energies equals exp(-E_jt/kT) / sum over every valid pose, which links
    the per-configuration log S of the oracle to its pose energies."""
    w = synth.plain_small(n_conf=4)
    r, lig = w.receptors[0], w.ligands[0]
    gam = oracle.gamma(lig.params.q, lig.params.eps, lig.params.R)
    logS, _, _ = oracle.logS_batch(r.grids, r.h, r.site_lo, r.site_n, lig.coords, gam, KT)
    Es = [oracle.pose_energies(r.grids, r.h, r.site_lo, r.site_n, lig.coords[j], gam)[0].ravel()
          for j in range(4)]
    flat = np.concatenate(Es)
    fin = np.isfinite(flat)
    lw = np.where(fin, -flat / KT, -np.inf)
    p_flat = np.exp(lw - logsumexp(lw[fin]))
    pj = S.config_weights(logS)
    p_two = np.concatenate([pj[j] * S.translation_weights(Es[j], KT) for j in range(4)])
    assert np.allclose(p_two, p_flat, rtol=1e-10, atol=1e-300)
    # the flat inverse CDF and the two-stage draw agree in distribution: the
    # stratified counts of both follow the same probabilities
    N = 20000
    u = (np.arange(N) + 0.5) / N
    flat_idx = S._inverse_cdf(p_flat, u)
    assert np.all(np.abs(np.bincount(flat_idx, minlength=flat.size) - N * p_flat) <= 1.0 + 1e-9)


def _logS_table(J=5, K=3, seed=4):
    rng = np.random.default_rng(seed)
    n = rng.integers(1, 500, (J, K))
    logZ = rng.normal(-20, 6, (J, K))
    return logZ + np.log(n), n


def test_bootstrap_identity_and_single_configuration():
    """A replicate that draws every configuration once is the full estimate;
    one that draws a single configuration J times is that configuration's
    own B = -kT log Z and dG with its own site volume."""
    logS, n = _logS_table()
    J, K = logS.shape
    h = 0.25
    u = np.vstack([(np.arange(J) + 0.5) / J, np.zeros(J)])
    reps, _ = S.bootstrap(logS, n, KT, h, u)
    B = oracle.bpmf(logS, n, KT)
    assert np.allclose(reps[0, :K], B, rtol=1e-13, atol=1e-10)
    assert abs(reps[0, K] - oracle.dG(B, KT, oracle.site_volume(n, h))) <= 1e-10
    own = -KT * (logS[0] - np.log(n[0]))
    assert np.allclose(reps[1, :K], own, rtol=1e-13, atol=1e-10)
    # closed form of dG for one configuration: -kT ln mean_k exp(-B_k/kT) - kT ln(h^3 mean_k n_k C)
    ref = -KT * logsumexp(-own / KT, b=np.full(K, 1.0 / K)) - KT * np.log(h ** 3 * n[0].mean() * oracle.C_STANDARD)
    assert abs(reps[1, K] - ref) <= 1e-10


def test_bootstrap_two_configurations_exact_distribution():
    """Two configurations: a replicate of two slots is one of four equally
    likely ordered draws; the bootstrap mean and variance over stratified
    uniforms converge to the exact moments of those four outcomes."""
    logS, n = _logS_table(J=2, K=2, seed=9)
    h = 0.375
    outcomes = []
    for a in range(2):
        for b in range(2):
            idx = np.array([a, b])
            Bk = oracle.bpmf(logS[idx], n[idx], KT)
            outcomes.append(np.append(Bk, oracle.dG(Bk, KT, oracle.site_volume(n[idx], h))))
    outcomes = np.array(outcomes)
    # stratified: every ordered pair equally often
    u = np.array([[x, y] for x in (0.25, 0.75) for y in (0.25, 0.75)] * 25)
    reps, stats = S.bootstrap(logS, n, KT, h, u)
    assert np.allclose(stats[0], outcomes.mean(axis=0), rtol=1e-12, atol=1e-9)
    R = u.shape[0]
    var = outcomes.var(axis=0) * R / (R - 1)
    assert np.allclose(stats[1] ** 2, var, rtol=1e-9, atol=1e-12)


def test_bootstrap_constant_replicates_have_zero_spread():
    logS, n = _logS_table()
    u = np.tile((np.arange(5) + 0.5) / 5, (6, 1))
    reps, stats = S.bootstrap(logS, n, KT, 0.25, u)
    assert np.all(reps == reps[0]) and np.all(stats[1] <= 1e-12 * np.abs(stats[0]))
