"""Pins of the learned-proposal reference: finite-difference gradients of the
FP64 network, the walker features as the gradient of log|<Phi(x)|phi>| at
x = 0, and exact Metropolis-Hastings with the random-walk and learned
proposals on the closed-form target N(c, I) (commuting U_k)."""

import math

import numpy as np

import afqmc_inputs as ai
from oracle import afqmc as oa
from oracle import mlp as om
from oracle import philox as px


def test_gradient_matches_finite_differences():
    K, H = 5, 8
    rng = np.random.default_rng(0)
    theta = 0.4 * rng.normal(size=om.n_params(K, H))
    f = rng.normal(size=(3, K))
    x = rng.normal(size=(3, 4, K))
    loss, g = om.loss_and_grad(theta, f, x, K, H)
    for idx in rng.choice(theta.size, 25, replace=False):
        e = np.zeros_like(theta)
        e[idx] = 1e-6
        num = (om.loss_and_grad(theta + e, f, x, K, H)[0] - om.loss_and_grad(theta - e, f, x, K, H)[0]) / 2e-6
        assert abs(num - g[idx]) < 1e-7 * max(1.0, abs(num)), idx


def test_features_are_the_log_overlap_gradient():
    s = ai.make_system(ai.SystemSpec(9, 3, 2, 6, 4, False, 5))
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, 3, 2, 0.01)
    rng = np.random.default_rng(1)
    phu = rng.normal(size=(2, 9, 3)) + 1j * rng.normal(size=(2, 9, 3))
    phd = rng.normal(size=(2, 9, 2)) + 1j * rng.normal(size=(2, 9, 2))
    f = om.features(s.Phi0, s.U, phu, phd)
    h = 1e-5
    for w in range(2):
        for k in range(4):
            e = np.zeros(4)
            e[k] = h
            lp = oa.log_overlap(ham, oa.trial_orbitals(ham, e), phu[w], phd[w]).real
            lm = oa.log_overlap(ham, oa.trial_orbitals(ham, -e), phu[w], phd[w]).real
            assert abs((lp - lm) / (2 * h) - f[w, k]) < 1e-6


def _commuting_setup():
    s = ai.make_system(ai.SystemSpec(6, 2, 2, 10, 3, False, 12))
    rng = np.random.default_rng(4)
    _, Q = np.linalg.eigh(s.h)
    d = rng.normal(0.0, 0.2, size=(3, 6))
    U = np.einsum("ia,ka,ja->kij", Q, d, Q)
    ham = oa.prepare(s.h, s.L, s.Phi0, U, 2, 2, 0.01)
    c = 2.0 * d[:, :2].sum(axis=1)
    return ham, c


def _sample(ham, cfg, mlp=None, sweeps=120):
    st = oa.init(ham, cfg)
    W, P = cfg.n_walkers, cfg.n_paths
    logov = np.array([[oa.log_overlap(ham, st.Phi[w, p], st.phi_up[w], st.phi_dn[w]) for p in range(P)]
                      for w in range(W)])
    alive = np.ones(W, dtype=bool)
    xs, acc = [], 0
    for sweep in range(sweeps):
        a = oa.mcmc_sweep(ham, cfg, st, logov, alive, 0, sweep, px.TAG_BURN_PROPOSE, px.TAG_BURN_ACCEPT, mlp)
        if sweep >= 20:
            xs.append(st.x.reshape(-1, 3).copy())
            acc += a
    return np.concatenate(xs), acc / ((sweeps - 20) * W * P)


def test_random_walk_and_learned_proposals_sample_the_closed_form_target():
    ham, c = _commuting_setup()
    for proposal, mlp in (("rw", None), ("mlp", (np.tile(c + 0.3, (4, 1)), np.full((4, 3), math.log(1.5))))):
        cfg = oa.OracleConfig(dtau=0.01, n_walkers=4, n_paths=64, seed=23, n_burn=0, proposal=proposal, rw_step=0.9,
                              mlp_mix=0.2)
        X, acc = _sample(ham, cfg, mlp)
        n_eff = X.shape[0] * 0.05
        assert np.all(np.abs(X.mean(axis=0) - c) < 5.0 / math.sqrt(n_eff)), proposal
        assert np.allclose(np.cov(X.T), np.eye(3), atol=0.1), proposal
        assert 0.05 < acc < 0.98
