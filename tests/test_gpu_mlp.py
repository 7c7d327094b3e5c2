"""The learned Metropolis proposal on the GPU: the BF16 network's output,
loss and gradients against the FP64 oracle network, random-walk and learned
proposal steps against the oracle step, and what online training gains over
the prior proposal (acceptance rate and integrated autocorrelation time)."""

import math

import numpy as np
import pytest

import afqmc_inputs as ai
from oracle import afqmc as oa
from oracle import mlp as om

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2505_18519_gb300 import afqmc as lib  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2505_18519_gb300 import build
    build.build()
    lib.load_library()


def _ctx(spec, W, P, dtau, seed, **kw):
    s = ai.make_system(spec)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, **kw)
    return s, lib.Context(cfg, s.h, s.L, s.Phi0, s.U)


def test_network_output_loss_and_gradient_match_the_oracle():
    spec = ai.SystemSpec(8, 4, 4, 12, 11, False, 1000)
    s, ctx = _ctx(spec, 20, 6, 0.01, 5, proposal="mlp", n_burn=0)
    K = spec.K
    rng = np.random.default_rng(3)
    theta = (0.15 * rng.normal(size=om.n_params(K))).astype(np.float32)
    ctx.mlp_params(theta)
    assert np.array_equal(ctx.mlp_params(), theta)
    f = rng.normal(size=(20, K)).astype(np.float32)
    x = rng.normal(size=(20, 6, K))
    g = ctx.mlp_eval(f, x)
    ref = om.forward(theta.astype(np.float64), f.astype(np.float64), K)
    loss, grad = om.loss_and_grad(theta.astype(np.float64), f.astype(np.float64), x, K)
    # BF16 weights and activations: about 2^-9 relative per rounding, a few layers deep
    assert np.max(np.abs(g["mu"] - ref["mu"])) < 3e-2 * np.max(np.abs(ref["mu"]))
    assert np.max(np.abs(g["logv"] - ref["logv"])) < 3e-2
    assert abs(g["loss"] - loss) < 2e-2 * abs(loss)
    assert np.linalg.norm(g["grad"] - grad) < 5e-2 * np.linalg.norm(grad)
    ctx.close()


def _oracle_state(ham, ocfg):
    st = oa.init(ham, ocfg)
    st, _ = oa.step(ham, ocfg, st)
    return st


def _as_dict(st):
    return dict(step=st.step, phi_up=st.phi_up, phi_dn=st.phi_dn, weight=st.weight, x=st.x, Phi=st.Phi)


@pytest.mark.parametrize("proposal", ["rw", "mlp"])
def test_random_walk_and_learned_steps_match_the_oracle(proposal):
    spec = ai.SystemSpec(10, 4, 3, 16, 7, False, 80)
    W, P, dtau = 6, 5, 0.01
    s, ctx = _ctx(spec, W, P, dtau, 41, proposal=proposal, n_burn=2, rw_step=0.7, mlp_mix=0.3, n_sweeps=2)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=41, n_burn=2, proposal="rw", rw_step=0.7,
                           mlp_mix=0.3, n_sweeps=2)
    ost = _oracle_state(ham, ocfg)
    ctx.load_state_arrays(_as_dict(ost))
    ctx.step(1)
    g = ctx.state_arrays()
    mlp = None
    if proposal == "mlp":
        ms = ctx.mlp_state()
        # the features are the oracle's, computed at the propagated walkers
        st_prop = ost.copy()
        ocfg_m = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=41, proposal="mlp", rw_step=0.7, mlp_mix=0.3,
                                 n_sweeps=2)
        mlp = (ms["mu"].astype(np.float64), ms["logv"].astype(np.float64))
        ost2, d = oa.step(ham, ocfg_m, st_prop, mlp_mu_logv=mlp)
    else:
        ost2, d = oa.step(ham, ocfg, ost)
    assert np.allclose(g["weight"], ost2.weight, rtol=1e-9, atol=0)
    assert np.max(np.abs(g["x"] - ost2.x)) < 1e-9
    assert np.max(np.abs(g["phi_up"] - ost2.phi_up)) < 1e-9
    assert ctx.history(1)[0][3] == d["n_accept"]
    if proposal == "mlp":
        phi_new = [oa.propagate_walker(ham, ost.phi_up[w], d["xi"][w] + 1j * np.sqrt(dtau) * d["v_bar"][w], dtau, 6)
                   for w in range(W)]
        f_ref = om.features(s.Phi0, s.U, np.array(phi_new),
                            np.array([oa.propagate_walker(ham, ost.phi_dn[w], d["xi"][w] + 1j * np.sqrt(dtau) * d["v_bar"][w],
                                                          dtau, 6) for w in range(W)]))
        assert np.allclose(ms["features"], f_ref, rtol=1e-5, atol=1e-5)
    ctx.close()


def _tau_int(series):
    """Integrated autocorrelation time with Sokal's self-consistent window (c = 5)."""
    x = np.asarray(series, dtype=np.float64)
    x = x - x.mean()
    n = x.size
    var = np.dot(x, x) / n
    if var == 0:
        return 1.0
    tau = 1.0
    for t in range(1, n // 2):
        rho = np.dot(x[:-t], x[t:]) / (n * var)
        tau += 2.0 * rho
        if t >= 5 * tau:
            break
    return max(tau, 1.0)


def test_trained_network_gains_over_the_prior_proposal():
    """Online training on the medium system's chains (16 x 16 paths), then the
    frozen network against the prior proposal from the same state: higher
    acceptance and shorter integrated autocorrelation of the paths' x."""
    spec = ai.SystemSpec(30, 6, 6, 60, 30, True, 4040)
    W, P, dtau = 16, 16, 0.005
    s, ctx = _ctx(spec, W, P, dtau, 9, proposal="mlp", mlp_train=True, mlp_lr=2e-3, n_burn=10, mlp_mix=0.1,
                  e_shift=20.0)
    theta0 = ctx.mlp_params()
    ctx.step(60)
    theta = ctx.mlp_params()
    # the fit on the chains' latest states: initial network against trained network
    st, ms = ctx.state_arrays(), ctx.mlp_state()
    loss_trained = ctx.mlp_eval(ms["features"], st["x"])["loss"]
    ctx.mlp_params(theta0)
    loss_initial = ctx.mlp_eval(ms["features"], st["x"])["loss"]
    ctx.mlp_params(theta)
    print("proposal loss on the last states: initial %.4f, trained %.4f" % (loss_initial, loss_trained))
    assert loss_trained < loss_initial
    start = ctx.save_state()
    ctx.close()
    res = {}
    for prop in ("prior", "mlp"):
        s, c = _ctx(spec, W, P, dtau, 9, proposal=prop, mlp_train=False, mlp_mix=0.1, n_burn=0, e_shift=20.0)
        if prop == "mlp":
            c.mlp_params(theta)
        c.load_state(start)
        xs, acc = [], []
        for _ in range(40):
            c.step(1)
            xs.append(c.state_arrays()["x"][:, :, 0].ravel().copy())
            acc.append(c.history(1)[0][3] / (W * P))
        X = np.array(xs)
        res[prop] = (float(np.mean(acc)), float(np.mean([_tau_int(X[:, j]) for j in range(X.shape[1])])))
        c.close()
    print("acceptance, tau_int:", res)
    assert res["mlp"][0] > res["prior"][0]
    assert res["mlp"][1] < res["prior"][1]
