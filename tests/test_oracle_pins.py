"""Pins of the CPU oracle against things other than itself.

Brute force in determinant space (a literal second-quantised Hamiltonian),
library matrix functions, closed forms of exactly solvable limits, invariances
and statistical laws.  A dropped term, a wrong sign or index, or a transposed
operand anywhere in the oracle's local energy, force bias, overlaps,
propagator, Metropolis step or weight update fails at least one of them.
"""

import dataclasses
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as ssla
import scipy.stats as stats

import afqmc_inputs as ai
from fock_space import FockSpace
from oracle import afqmc as oa
from oracle import philox as px


def _rand_walker(rng, N, n):
    return rng.normal(size=(N, n)) + 1j * rng.normal(size=(N, n))


def _ham(sysobj, n_up, n_dn, dtau=0.01, U=None, L=None, Phi0=None):
    return oa.prepare(sysobj.h, sysobj.L if L is None else L, sysobj.Phi0 if Phi0 is None else Phi0,
                      sysobj.U if U is None else U, n_up, n_dn, dtau)


def _small_system(N=6, n_up=3, n_dn=3, G=10, K=5, seed=7):
    return ai.make_system(ai.SystemSpec(N, max(n_up, n_dn), max(n_up, n_dn), G, K, False, seed))


def _commuting_U(h, K, n_up, rng, scale=0.3):
    """U_k = Q diag(d_k) Q^T with Q the eigenvectors of h (so [U_k, h] = 0)."""
    _, Q = np.linalg.eigh(h)
    d = rng.normal(0.0, scale, size=(K, h.shape[0]))
    return np.einsum("ia,ka,ja->kij", Q, d, Q), d


@pytest.fixture(scope="module")
def c0():
    s, run = ai.make_config("small_n8")
    fs = FockSpace(8, 4, 4)
    H = fs.hamiltonian(s.h, s.L)
    return s, run, fs, H


# ---------------------------------------------------------------- determinant space

def test_local_energy_and_overlap_match_determinant_space_c0(c0):
    s, run, fs, H = c0
    ham = _ham(s, 4, 4, run.dtau)
    rng = np.random.default_rng(11)
    for trial in range(3):
        x = rng.normal(size=ham.U.shape[0])
        Phi = oa.trial_orbitals(ham, x)
        phu, phd = _rand_walker(rng, 8, 4), _rand_walker(rng, 8, 4)
        cP = fs.determinant(Phi, Phi)
        cp = fs.determinant(phu, phd)
        ov = cP @ cp
        e_fs = (cP @ (H @ cp)) / ov
        e, v = oa.local_energy_force_bias(ham, Phi, phu, phd)
        assert abs(e - e_fs) < 1e-10 * max(1.0, abs(e_fs))
        assert abs(np.exp(oa.log_overlap(ham, Phi, phu, phd)) - ov) < 1e-10 * abs(ov)
        # force bias values: <Phi|L_g|phi>/<Phi|phi> with L_g = sum_s sum_ij L_g,ij c+_is c_js
        for g in (0, 5, 31):
            Lg = fs.one_body(s.L[g], 4, 4)
            vg = (cP @ (Lg @ cp)) / ov
            assert abs(v[g] - vg) < 1e-11 * max(1.0, abs(vg))


@pytest.mark.parametrize("n_up,n_dn", [(3, 2), (2, 0), (1, 1)])
def test_local_energy_unequal_spins(n_up, n_dn):
    s = _small_system(6, n_up, n_dn, G=7, K=4, seed=3)
    fs = FockSpace(6, n_up, n_dn)
    H = fs.hamiltonian(s.h, s.L)
    ham = _ham(s, n_up, n_dn)
    rng = np.random.default_rng(5)
    Phi = oa.trial_orbitals(ham, rng.normal(size=4))
    phu, phd = _rand_walker(rng, 6, n_up), _rand_walker(rng, 6, n_dn)
    cP = fs.determinant(Phi, Phi[:, :n_dn])
    cp = fs.determinant(phu, phd)
    ov = cP @ cp
    e, v = oa.local_energy_force_bias(ham, Phi, phu, phd)
    assert abs(e - (cP @ (H @ cp)) / ov) < 1e-10
    assert abs(np.exp(oa.log_overlap(ham, Phi, phu, phd)) - ov) < 1e-10 * abs(ov)


def test_fci_ground_state_below_trial_energy(c0):
    s, run, fs, H = c0
    e0 = ssla.eigsh(H, k=1, which="SA")[0][0]
    ham = _ham(s, 4, 4, run.dtau)
    e_trial, _ = oa.local_energy_force_bias(ham, s.Phi0, s.Phi0.astype(complex), s.Phi0.astype(complex))
    cP = fs.determinant(s.Phi0, s.Phi0)
    assert abs(e_trial - (cP @ (H @ cP)) / (cP @ cP)) < 1e-10
    assert e0 < e_trial.real - 1e-3


# ---------------------------------------------------------------- Green's function and ratios

def test_green_idempotent_and_trace():
    s = _small_system(8, 4, 4)
    ham = _ham(s, 4, 4)
    rng = np.random.default_rng(2)
    Phi = oa.trial_orbitals(ham, rng.normal(size=5))
    phi = _rand_walker(rng, 8, 4)
    G = oa.green(Phi, phi)
    assert np.allclose(G @ G, G, atol=1e-12)
    assert abs(np.trace(G) - 4) < 1e-12
    # G^T acts as the identity on the walker's column space
    assert np.allclose(G.T @ phi, phi, atol=1e-12)


def test_ratio_from_inverse_equals_full_recomputation():
    s = _small_system(8, 4, 4)
    ham = _ham(s, 4, 4)
    rng = np.random.default_rng(3)
    Phi = oa.trial_orbitals(ham, rng.normal(size=5))
    phi, phi2 = _rand_walker(rng, 8, 4), _rand_walker(rng, 8, 4)
    A = Phi.T @ phi
    via_inverse = np.linalg.det(np.linalg.inv(A) @ (Phi.T @ phi2))
    lo1 = oa.log_overlap(ham, Phi, phi, np.zeros((8, 4)) + phi)
    lo2 = oa.log_overlap(ham, Phi, phi2, np.zeros((8, 4)) + phi)
    assert abs(np.exp(lo2 - lo1) - via_inverse) < 1e-11 * abs(via_inverse)


def test_invariance_under_right_multiplication():
    s = _small_system(8, 4, 4)
    ham = _ham(s, 4, 4)
    rng = np.random.default_rng(4)
    Phi = oa.trial_orbitals(ham, rng.normal(size=5))
    phu, phd = _rand_walker(rng, 8, 4), _rand_walker(rng, 8, 4)
    R = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    e1, v1 = oa.local_energy_force_bias(ham, Phi, phu, phd)
    e2, v2 = oa.local_energy_force_bias(ham, Phi, phu @ R, phd)
    assert abs(e1 - e2) < 1e-11 * abs(e1)
    assert np.allclose(v1, v2, atol=1e-12)
    Q = oa.reorthonormalise(phu)
    assert np.allclose(Q.conj().T @ Q, np.eye(4), atol=1e-12)
    e3, _ = oa.local_energy_force_bias(ham, Phi, Q, phd)
    assert abs(e1 - e3) < 1e-11 * abs(e1)
    Rm = Q.conj().T @ phu                       # upper triangular with positive real diagonal
    assert np.allclose(np.tril(Rm, -1), 0, atol=1e-12)
    assert np.all(np.diag(Rm).real > 0) and np.allclose(np.diag(Rm).imag, 0, atol=1e-12)


# ---------------------------------------------------------------- matrix functions

def test_matrix_functions_against_scipy():
    s = _small_system(8, 4, 4)
    ham = _ham(s, 4, 4, dtau=0.05)
    assert np.allclose(ham.expT_half, sla.expm(-0.025 * ham.T), atol=1e-13)
    T_direct = s.h - 0.5 * sum(s.L[g] @ s.L[g] for g in range(s.L.shape[0]))
    assert np.allclose(ham.T, T_direct, atol=1e-14)
    x = np.random.default_rng(1).normal(size=5)
    S = sum(x[k] * s.U[k] for k in range(5))
    assert np.allclose(oa.trial_orbitals(ham, x), sla.expm(S) @ s.Phi0, atol=1e-12)


def test_taylor_propagator_within_truncation_bound():
    s = _small_system(8, 4, 4)
    tau = 0.01
    ham = _ham(s, 4, 4, dtau=tau)
    rng = np.random.default_rng(9)
    y = rng.normal(size=s.L.shape[0]) + 0.3j * rng.normal(size=s.L.shape[0])
    phi = _rand_walker(rng, 8, 4)
    A = 1j * math.sqrt(tau) * np.einsum("g,gij->ij", y, s.L)
    exact = ham.expT_half @ sla.expm(A) @ ham.expT_half @ phi
    got = oa.propagate_walker(ham, phi, y, tau, 6)
    a = np.linalg.norm(A, 2)
    bound = a ** 7 / math.factorial(7) * math.exp(a) * np.linalg.norm(phi, 2)
    assert np.linalg.norm(got - exact, 2) <= bound * 1.01 + 1e-13
    # and the sixth-order truncation is actually what is computed: order 12 is closer to exact
    got12 = oa.propagate_walker(ham, phi, y, tau, 12)
    assert np.linalg.norm(got12 - exact, 2) < 1e-12


# ---------------------------------------------------------------- exactly solvable limits

def test_exact_eigenstate_one_body_hamiltonian():
    """L = 0 and U commuting with h: every Phi(x) is the exact ground state,
    so every local energy equals 2 * sum of the lowest n eigenvalues of h."""
    s = _small_system(8, 3, 3, K=4, seed=21)
    rng = np.random.default_rng(0)
    U, _ = _commuting_U(s.h, 4, 3, rng)
    L0 = np.zeros((2, 8, 8))
    ham = _ham(s, 3, 3, dtau=0.02, U=U, L=L0)
    e_exact = 2.0 * np.sum(np.linalg.eigvalsh(s.h)[:3])
    cfg = oa.OracleConfig(dtau=0.02, n_walkers=4, n_paths=3, seed=99, n_burn=2)
    st = oa.init(ham, cfg)
    for _ in range(3):
        st, d = oa.step(ham, cfg, st)
        assert np.allclose(d["measure"]["e_pair"], e_exact, atol=1e-11)
        num, den = d["mixed"]
        assert abs(num / den - e_exact) < 1e-11


def test_one_electron_local_energy_is_constant():
    """One electron, L != 0, Phi0 an eigenvector of h and U commuting with h:
    the two-body term cannot act on one particle, so E_L = eps_0 for every
    walker while the full auxiliary-field propagation runs."""
    s = _small_system(7, 1, 1, G=6, K=3, seed=5)
    rng = np.random.default_rng(1)
    U, _ = _commuting_U(s.h, 3, 1, rng)
    ham = _ham(s, 1, 0, dtau=0.02, U=U)
    eps0 = np.linalg.eigvalsh(s.h)[0]
    cfg = oa.OracleConfig(dtau=0.02, n_walkers=5, n_paths=2, seed=3, n_burn=1)
    st = oa.init(ham, cfg)
    for _ in range(3):
        st, d = oa.step(ham, cfg, st)
        assert np.allclose(d["measure"]["e_pair"], eps0, atol=1e-11)
        assert np.any(np.abs(d["v_bar"]) > 1e-3)          # the force bias is not trivial


def test_no_hidden_variables_reduces_to_single_determinant():
    """U = 0: Phi(x) = Phi0 for every path, so every path sign is equal, every
    proposal is accepted, the hand-off angle vanishes, the three constraint
    variants coincide, and the walk does not depend on the number of paths."""
    s = _small_system(8, 3, 3, K=4, seed=8)
    U0 = np.zeros_like(s.U[:4])
    ham = _ham(s, 3, 3, dtau=0.02, U=U0)
    results = {}
    for P in (1, 4):
        for c in oa.CONSTRAINTS:
            cfg = oa.OracleConfig(dtau=0.02, n_walkers=6, n_paths=P, seed=17, n_burn=1, constraint=c)
            st = oa.init(ham, cfg)
            for _ in range(3):
                st, d = oa.step(ham, cfg, st)
                S = d["measure"]["S"]
                assert np.allclose(S, S[:, :1], atol=1e-12)
                assert d["n_accept"] == d["n_proposed"]
                dth_T = np.angle(d["new_sum"]) - np.angle(d["old_sum"])
                assert np.allclose(np.angle(np.exp(1j * dth_T)), 0.0, atol=1e-10)
            results[(P, c)] = (st.weight.copy(), st.phi_up.copy())
    ref_w, ref_phi = results[(1, "combined")]
    for key, (w, phi) in results.items():
        assert np.allclose(w, ref_w, rtol=1e-11, atol=0), key
        assert np.allclose(phi, ref_phi, atol=1e-11), key


def test_combined_angle_identity():
    """Delta theta + Delta theta_T = Arg sum_p S'_p - Arg sum_p S_p (mod 2 pi)."""
    s, run = ai.make_config("small_n8")
    ham = _ham(s, 4, 4, run.dtau)
    cfg = oa.OracleConfig(dtau=run.dtau, n_walkers=8, n_paths=6, seed=5, n_burn=3)
    st0 = oa.init(ham, cfg)
    st, d = oa.step(ham, cfg, st0)
    lhs = np.angle(d["ratio"]) + np.angle(d["new_sum"]) - np.angle(d["old_sum"])
    rhs = np.angle(d["new_sum"]) - np.angle(d["measure"]["sumS"])
    assert np.allclose(np.exp(1j * lhs), np.exp(1j * rhs), atol=1e-12)
    # the combined-angle weight factor depends only on the path signs before and after
    factor = st.weight / (st0.weight * d["I_abs"])
    assert np.allclose(factor, np.maximum(0.0, np.cos(rhs)), atol=1e-12)
    assert np.any(np.abs(rhs) > 1e-3)


def test_metropolis_samples_closed_form_target():
    """U_k = Q diag(d_k) Q^T commuting with h: |<Phi(x)|phi>| is proportional to
    exp(c . x), c_k = sum over occupied a of d_k,a for each spin, so the path
    density of Eq. (23) is N(c, I) and the independence sampler from the prior
    accepts with probability 2 Phi_normal(-|c| / sqrt(2))."""
    s = _small_system(6, 2, 2, K=3, seed=12)
    rng = np.random.default_rng(4)
    U, d = _commuting_U(s.h, 3, 2, rng, scale=0.2)
    ham = _ham(s, 2, 2, U=U)
    c = 2.0 * d[:, :2].sum(axis=1)                 # both spins occupy the two lowest orbitals
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=4, n_paths=64, seed=23, n_burn=0)
    st = oa.init(ham, cfg)
    W, P = 4, 64
    logov = np.array([[oa.log_overlap(ham, st.Phi[w, p], st.phi_up[w], st.phi_dn[w]) for p in range(P)]
                      for w in range(W)])
    alive = np.ones(W, dtype=bool)
    xs, acc, tot = [], 0, 0
    for sweep in range(120):
        a = oa.mcmc_sweep(ham, cfg, st, logov, alive, 0, sweep, px.TAG_BURN_PROPOSE, px.TAG_BURN_ACCEPT)
        if sweep >= 20:
            xs.append(st.x.reshape(-1, 3).copy())
            acc += a
            tot += W * P
    X = np.concatenate(xs)
    # independence sampler: integrated autocorrelation ~ 1/acceptance; be generous
    n_eff = X.shape[0] * 0.2
    assert np.all(np.abs(X.mean(axis=0) - c) < 5.0 / math.sqrt(n_eff))
    assert np.allclose(np.cov(X.T), np.eye(3), atol=0.08)
    acc_exact = 2.0 * stats.norm.cdf(-np.linalg.norm(c) / math.sqrt(2.0))
    assert abs(acc / tot - acc_exact) < 0.02


# ---------------------------------------------------------------- counter-based random numbers

def test_philox_uniforms_and_normals_statistics():
    u = px.uniforms(0x1234, px.TAG_ACCEPT, 7, np.arange(2000), 0, 500).ravel()
    assert np.all((u >= 0) & (u < 1))
    assert stats.kstest(u, "uniform").pvalue > 1e-4
    hist, _ = np.histogram(u, bins=100, range=(0, 1))
    assert stats.chisquare(hist).pvalue > 1e-4
    z = px.normals(0x1234, px.TAG_FIELD, 3, np.arange(2000), 0, 500).ravel()
    assert stats.kstest(z, "norm").pvalue > 1e-4
    assert abs(z.mean()) < 5e-3 and abs(z.var() - 1) < 1e-2
    assert abs(stats.skew(z)) < 2e-2 and abs(stats.kurtosis(z)) < 4e-2


def test_philox_streams_are_distinct_and_deterministic():
    a = px.normals(5, px.TAG_FIELD, 0, np.arange(10), 0, 8)
    b = px.normals(5, px.TAG_FIELD, 0, np.arange(10), 0, 8)
    assert np.array_equal(a, b)
    for other in (px.normals(6, px.TAG_FIELD, 0, np.arange(10), 0, 8),
                  px.normals(5, px.TAG_PROPOSE, 0, np.arange(10), 0, 8),
                  px.normals(5, px.TAG_FIELD, 1, np.arange(10), 0, 8),
                  px.normals(5, px.TAG_FIELD, 0, np.arange(10), 1, 8)):
        assert not np.any(np.isclose(a, other))
    # an odd count is the prefix of the even one
    assert np.array_equal(px.normals(5, 3, 0, [4], 0, 7), px.normals(5, 3, 0, [4], 0, 8)[:, :7])
    # counter words: one changed input bit changes about half of the output bits
    c0 = np.array([[0, 0, 0, 0]], dtype=np.uint32)
    c1 = np.array([[1, 0, 0, 0]], dtype=np.uint32)
    o0, o1 = px.philox4x32_10(c0, (0, 0)), px.philox4x32_10(c1, (0, 0))
    flips = sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(o0[0], o1[0]))
    assert 40 < flips < 88


def test_force_bias_cancels_first_order_weight_fluctuation():
    """With the optimal shift of Eq. (15) the O(sqrt(tau)) field dependence of
    the importance function Eq. (14) cancels; at tau = 1e-6 every |log|I||
    stays O(tau), while a shift with the wrong sign or scale leaves O(sqrt(tau))."""
    s, run = ai.make_config("small_n8")
    tau = 1e-6
    ham = _ham(s, 4, 4, tau)
    cfg = oa.OracleConfig(dtau=tau, n_walkers=12, n_paths=4, seed=31, n_burn=2)
    st = oa.init(ham, cfg)
    rng = np.random.default_rng(6)
    for w in range(12):                                 # complex walkers: the test has teeth
        st.phi_up[w] = oa.reorthonormalise(st.phi_up[w] + 0.3j * _rand_walker(rng, 8, 4))
        st.phi_dn[w] = oa.reorthonormalise(st.phi_dn[w] + 0.3j * _rand_walker(rng, 8, 4))
    st, d = oa.step(ham, cfg, st)
    assert np.max(np.abs(d["v_bar"].imag)) > 1e-2
    assert np.max(np.abs(np.log(d["I_abs"]))) < 200 * tau


def test_sampled_trial_estimator_matches_quadrature():
    """K = 1: <Psi_T|O|phi>/<Psi_T|phi> with Psi_T = int dx p(x) Phi(x) is a
    one-dimensional integral; Gauss-Hermite quadrature gives it exactly, and
    the path-sign-weighted average of Eq. (27) over paths sampled from Eq. (23)
    must converge to it (O = H and O = L_g)."""
    N, n = 4, 2
    s = _small_system(N, n, n, G=3, K=1, seed=43)
    rng = np.random.default_rng(8)
    U = 2.0 * s.U[:1]
    ham = _ham(s, n, n, U=U)
    phu, phd = _rand_walker(rng, N, n), _rand_walker(rng, N, n)
    # quadrature: sum_j w_j ov(x_j) O_L(x_j) / sum_j w_j ov(x_j)
    xq, wq = np.polynomial.hermite_e.hermegauss(80)
    num_e = den = 0.0
    num_v = 0.0
    for xj, wj in zip(xq, wq):
        Phi = oa.trial_orbitals(ham, np.array([xj]))
        ov = np.exp(oa.log_overlap(ham, Phi, phu, phd))
        e, v = oa.local_energy_force_bias(ham, Phi, phu, phd)
        num_e, num_v, den = num_e + wj * ov * e, num_v + wj * ov * v, den + wj * ov
    e_exact, v_exact = num_e / den, num_v / den
    # sampled estimator: many walkers sharing phi, independent chains
    W, P = 16, 64
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=W, n_paths=P, seed=77, n_burn=0)
    st = oa.init(ham, cfg)
    st.phi_up[:] = phu
    st.phi_dn[:] = phd
    logov = np.array([[oa.log_overlap(ham, st.Phi[w, p], phu, phd) for p in range(P)] for w in range(W)])
    alive = np.ones(W, dtype=bool)
    se = sv = ss = 0.0
    for sweep in range(60):
        oa.mcmc_sweep(ham, cfg, st, logov, alive, 0, sweep, px.TAG_BURN_PROPOSE, px.TAG_BURN_ACCEPT)
        if sweep >= 10:
            m = oa.measure(ham, st)
            se += np.sum(m["S"] * m["e_pair"])
            sv += np.sum(m["S"][:, :, None] * m["v_pair"], axis=(0, 1))
            ss += np.sum(m["S"])
    mean_sign = abs(ss) / (50 * W * P)
    assert 0.05 < mean_sign < 0.95                      # the phases really vary
    assert abs(se / ss - e_exact) < 0.02 * abs(e_exact)
    assert np.allclose(sv / ss, v_exact, atol=0.02 * np.max(np.abs(v_exact)))


def test_importance_function_averages_to_exact_projection(c0):
    """Averaged over the auxiliary fields, the complex importance function of
    Eq. (14) (shifted Gaussian ratio times overlap ratio, Eq. (10)-(14)) equals
    <Phi0|exp(-tau H)|phi>/<Phi0|phi> up to O(tau^2) Trotter error; computed
    here with a literal determinant-space Hamiltonian.  U = 0 and one path, so
    the sampled trial is exactly Phi0."""
    s, run, fs, H = c0
    tau = 0.005
    ham = _ham(s, 4, 4, tau, U=np.zeros((1, 8, 8)))
    W = 3000
    cfg = oa.OracleConfig(dtau=tau, n_walkers=W, n_paths=1, seed=2024, n_burn=0)
    st = oa.init(ham, cfg)
    rng = np.random.default_rng(12)
    phu = oa.reorthonormalise(s.Phi0 + 0.4 * _rand_walker(rng, 8, 4))
    phd = oa.reorthonormalise(s.Phi0 + 0.4 * _rand_walker(rng, 8, 4))
    st.phi_up[:] = phu
    st.phi_dn[:] = phd
    st, d = oa.step(ham, cfg, st)
    I = d["I"]
    mean, err = I.mean(), I.std() / math.sqrt(W)
    cP, cp = fs.determinant(s.Phi0, s.Phi0), fs.determinant(phu, phd)
    exact = (cP @ ssla.expm_multiply(-tau * H, cp)) / (cP @ cp)
    shift = abs(exact - 1.0)
    assert shift > 0.03                                  # the projection is resolved
    assert abs(mean - exact) < 5 * err + 5e-4


# ---------------------------------------------------------------- importance function and population control
def test_local_energy_weights_of_an_exact_eigenstate():
    """L = 0 and U commuting with h make every trial sample an eigenstate of
    H = h: the hybrid |I| (the overlap ratio) and the local-energy |I| =
    exp(-tau E_L) both equal exp(-tau E0), the constraint factor is 1, and after
    k steps every weight is exp(-k tau (E0 - E_T)) under either form."""
    s = _small_system(8, 3, 3, K=4, seed=21)
    rng = np.random.default_rng(4)
    U, _ = _commuting_U(s.h, 4, 3, rng)
    tau = 0.02
    ham = _ham(s, 3, 3, dtau=tau, U=U, L=np.zeros((2, 8, 8)))
    e0 = 2.0 * np.sum(np.linalg.eigvalsh(s.h)[:3])
    e_t = e0 + 0.7
    for imp in oa.IMPORTANCE:
        cfg = oa.OracleConfig(dtau=tau, n_walkers=4, n_paths=3, seed=11, n_burn=2, importance=imp, e_shift=e_t)
        st = oa.init(ham, cfg)
        for k in range(1, 4):
            st, d = oa.step(ham, cfg, st)
            assert np.allclose(d["I_abs"], math.exp(-tau * e0), rtol=1e-12, atol=0), imp
            assert np.allclose(st.weight, math.exp(-k * tau * (e0 - e_t)), rtol=1e-11, atol=0), imp


def test_local_energy_importance_of_one_electron():
    """One electron with L != 0: the two-body term has nothing to act on, so
    E_L = eps_0 and the local-energy |I| is exp(-tau eps_0) for every live walker
    while the fields act (the hybrid |I| differs from walker to walker); the
    constraint factor W'/(W |I|) stays in [0, 1]."""
    s = _small_system(7, 1, 1, G=6, K=3, seed=5)
    rng = np.random.default_rng(1)
    U, _ = _commuting_U(s.h, 3, 1, rng)
    tau = 0.02
    ham = _ham(s, 1, 0, dtau=tau, U=U)
    eps0 = np.linalg.eigvalsh(s.h)[0]
    cfg = oa.OracleConfig(dtau=tau, n_walkers=5, n_paths=2, seed=3, n_burn=1, importance="local_energy")
    st = oa.init(ham, cfg)
    for _ in range(3):
        w0 = st.weight.copy()
        st, d = oa.step(ham, cfg, st)
        live = d["alive"]
        assert live.sum() >= 3
        assert np.allclose(d["I_abs"][live], math.exp(-tau * eps0), rtol=1e-11, atol=0)
        assert np.ptp(np.abs(d["I"][live])) > 1e-6
        f = st.weight[live] / (w0[live] * d["I_abs"][live])
        assert np.all((f >= 0.0) & (f <= 1.0 + 1e-12))


def test_comb_keeps_the_total_weight_and_copies_in_proportion():
    """A comb keeps the total weight, gives every new walker the mean weight,
    never copies a dead walker, gives walker w floor or ceil of W w_w / sum w
    copies, and leaves every walker that has a copy in its own slot."""
    rng = np.random.default_rng(12)
    W = 37
    weight = rng.exponential(size=W) * (rng.random(W) > 0.25)
    total = math.fsum(weight)
    expect = W * weight / total
    for u in (0.0, 0.31, 0.5, 1.0 - 2.0 ** -53):
        src, wn = oa.comb(weight, u)
        assert src.shape == (W,)
        assert np.all(weight[src] > 0.0)
        assert np.allclose(wn, total / W, rtol=1e-14, atol=0)
        assert abs(math.fsum(wn) - total) <= 1e-13 * total
        n = np.bincount(src, minlength=W)
        assert np.all(n >= np.floor(expect - 1e-9)) and np.all(n <= np.ceil(expect + 1e-9))
        moved = src != np.arange(W)
        assert np.all(src[n > 0] == np.arange(W)[n > 0]) and np.all(n[moved] == 0)
        assert np.all(~moved[src[moved]])      # every source is a walker that stays in place


def test_comb_of_equal_weights_is_the_identity():
    """Equal weights: tooth j falls in walker j's interval.  (With u within an
    ulp of 1, j + u rounds to j + 1 and the tooth lands on the next boundary;
    1 - 2^-40 stays clear of that.)"""
    weight = np.full(29, 2.5)
    for u in (0.0, 0.2, 0.75, 1.0 - 2.0 ** -40):
        src, wn = oa.comb(weight, u)
        np.testing.assert_array_equal(src, np.arange(29))
        assert np.all(wn == 2.5)


def test_comb_is_unbiased_over_its_uniform():
    """Averaged over u in [0, 1) (midpoint rule), walker w gets W w_w / sum w
    copies and the weighted sum of any per-walker quantity is unchanged: each
    walker's copy count jumps at most twice in u, so the rule errs by at most
    2 / M per walker."""
    rng = np.random.default_rng(3)
    W, M = 23, 20000
    weight = rng.gamma(0.5, size=W)
    weight[[4, 17]] = 0.0
    energy = rng.normal(size=W)
    copies = np.zeros(W)
    est = 0.0
    for u in (np.arange(M) + 0.5) / M:
        src, wn = oa.comb(weight, u)
        copies += np.bincount(src, minlength=W)
        est += np.sum(wn * energy[src])
    copies /= M
    est /= M
    assert np.allclose(copies, W * weight / weight.sum(), rtol=0, atol=2.5 / M)
    assert abs(est - np.sum(weight * energy)) <= 2.5 / M * np.sum(np.abs(energy)) * weight.sum() / W


def test_comb_step_resamples_the_walkers_of_the_plain_step():
    """With pop_period = 2 the first step leaves the population alone and the
    second combs, after the weight update and reorthonormalisation, with the
    uniform of its own Philox stream; every state array is gathered alike."""
    s, run = ai.make_config("small_n8")
    ham = _ham(s, 4, 4, run.dtau)
    base = oa.OracleConfig(dtau=run.dtau, n_walkers=8, n_paths=4, seed=9, n_burn=2)
    combing = dataclasses.replace(base, pop_period=2)
    st = oa.init(ham, base)
    st.weight = np.array([0.0, 3.0, 0.2, 1.0, 0.0, 0.5, 2.0, 0.3])
    st1, d1 = oa.step(ham, combing, st)
    assert d1["comb_src"] is None
    plain, _ = oa.step(ham, base, st1)
    combed, d2 = oa.step(ham, combing, st1)
    u = px.uniforms(base.seed, px.TAG_COMB, st1.step, [0], 0, 1)[0, 0]
    ref_src, ref_w = oa.comb(plain.weight, u)
    np.testing.assert_array_equal(d2["comb_src"], ref_src)
    assert np.array_equal(combed.weight, ref_w)
    for name in ("phi_up", "phi_dn", "x", "Phi"):
        np.testing.assert_array_equal(getattr(combed, name), getattr(plain, name)[ref_src])
    assert len(set(ref_src.tolist())) < 8 and plain.weight[0] == 0.0 and combed.weight[0] > 0.0


# ---------------------------------------------------------------- extra measurement paths
def test_measurement_paths_without_sweeps_are_the_plain_estimate():
    """One round and no sweep: the measurement paths are the propagation's, so
    R = 1, E'_w = E_w and the estimate is Eq. (16)'s; the state is untouched."""
    s, run = ai.make_config("small_n8")
    ham = _ham(s, 4, 4, run.dtau)
    cfg = oa.OracleConfig(dtau=run.dtau, n_walkers=6, n_paths=5, seed=14, n_burn=2)
    st, _ = oa.step(ham, cfg, oa.init(ham, cfg))
    st.weight[2] = 0.0
    before = st.copy()
    r = oa.measure_paths(ham, cfg, st, rounds=1, sweeps=0)
    m = oa.measure(ham, st)
    num, den = oa.mixed_energy(st.weight, m["e_bar"])
    assert abs(r["e_mix"] - num / den) < 1e-12
    assert np.allclose(r["R"][r["alive"]], 1.0, rtol=0, atol=1e-13)
    assert np.allclose(r["e_walker"], m["e_bar"], rtol=0, atol=1e-12)
    for name in ("x", "Phi", "weight", "phi_up"):
        assert np.array_equal(getattr(st, name), getattr(before, name))
    # with sweeps the paths move and the estimate changes
    r2 = oa.measure_paths(ham, cfg, st, rounds=2, sweeps=1)
    assert abs(r2["e_mix"] - r["e_mix"]) > 1e-8


def test_measurement_paths_in_the_exact_limits():
    """U = 0 (every path gives Phi0): R = 1 and the same estimate for any number
    of rounds; an exact-eigenstate trial (L = 0, [U_k, h] = 0): E' = E0."""
    s = _small_system(8, 3, 3, K=4, seed=8)
    ham0 = _ham(s, 3, 3, dtau=0.02, U=np.zeros_like(s.U[:4]))
    cfg = oa.OracleConfig(dtau=0.02, n_walkers=5, n_paths=3, seed=19, n_burn=1)
    st, _ = oa.step(ham0, cfg, oa.init(ham0, cfg))
    plain = oa.measure_paths(ham0, cfg, st, rounds=1, sweeps=0)
    more = oa.measure_paths(ham0, cfg, st, rounds=3, sweeps=2)
    assert np.allclose(more["R"], 1.0, rtol=0, atol=1e-12)
    assert abs(more["e_mix"] - plain["e_mix"]) < 1e-11
    rng = np.random.default_rng(3)
    U, _ = _commuting_U(s.h, 4, 3, rng)
    hame = _ham(s, 3, 3, dtau=0.02, U=U, L=np.zeros((2, 8, 8)))
    e0 = 2.0 * np.sum(np.linalg.eigvalsh(s.h)[:3])
    st, _ = oa.step(hame, cfg, oa.init(hame, cfg))
    r = oa.measure_paths(hame, cfg, st, rounds=3, sweeps=2)
    assert abs(r["e_mix"] - e0) < 1e-11 and np.allclose(r["e_walker"], e0, atol=1e-11)


def test_measurement_paths_converge_to_the_quadrature():
    """K = 1: with many measurement rounds at one walker, the sign-weighted
    average over the measurement paths, and the estimate weighted by R, tend
    to <Psi_T|H|phi>/<Psi_T|phi> given by Gauss-Hermite quadrature."""
    N, n = 4, 2
    s = _small_system(N, n, n, G=3, K=1, seed=43)
    rng = np.random.default_rng(8)
    ham = _ham(s, n, n, U=2.0 * s.U[:1])
    phu, phd = _rand_walker(rng, N, n), _rand_walker(rng, N, n)
    xq, wq = np.polynomial.hermite_e.hermegauss(80)
    num = den = dabs = 0.0
    for xj, wj in zip(xq, wq):
        Phi = oa.trial_orbitals(ham, np.array([xj]))
        ov = np.exp(oa.log_overlap(ham, Phi, phu, phd))
        e, _ = oa.local_energy_force_bias(ham, Phi, phu, phd)
        num, den, dabs = num + wj * ov * e, den + wj * ov, dabs + wj * abs(ov)
    e_exact = num / den
    sign_exact = den / dabs          # mean path sign under |ov| p(x)
    W, P = 8, 32
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=W, n_paths=P, seed=78, n_burn=10)
    st = oa.init(ham, cfg)
    st.phi_up[:] = phu
    st.phi_dn[:] = phd
    logov = np.array([[oa.log_overlap(ham, st.Phi[w, p], phu, phd) for p in range(P)] for w in range(W)])
    for b in range(10):   # equilibrate the paths at this walker
        oa.mcmc_sweep(ham, cfg, st, logov, np.ones(W, dtype=bool), 0, b, px.TAG_BURN_PROPOSE, px.TAG_BURN_ACCEPT)
    sumS = oa.measure(ham, st)["sumS"]
    r = oa.measure_paths(ham, cfg, st, rounds=60, sweeps=1)
    pooled = r["num"].sum() / r["den"].sum()
    assert abs(pooled - e_exact) < 0.02 * abs(e_exact)
    assert abs(r["e_mix"] - e_exact.real) < 0.03 * abs(e_exact)
    # R_w (sum_p S_p / P) is the measurement paths' mean sign, which tends to the exact one
    assert 0.05 < abs(sign_exact) < 0.95
    assert abs(np.mean(r["R"] * sumS / P) - sign_exact) < 0.05


# ---------------------------------------------------------------- complex trial samples
def test_complex_trial_local_energy_matches_determinant_space(c0):
    """Complex trial samples (R19, alpha = -i sqrt(s)): the bra <Phi| has the
    complex-conjugate determinant coefficients, so by brute force
    E_L = conj(c_Phi) H c_phi / conj(c_Phi) c_phi; the oracle's Phi^dagger
    formulas must agree, as must the overlap and every force-bias value."""
    s, run, fs, H = c0
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, 4, 4, run.dtau, alpha=-0.6j)
    rng = np.random.default_rng(21)
    for _ in range(3):
        x = rng.normal(size=ham.U.shape[0])
        Phi = oa.trial_orbitals(ham, x)
        assert np.iscomplexobj(Phi) and np.max(np.abs(Phi.imag)) > 1e-3
        phu, phd = _rand_walker(rng, 8, 4), _rand_walker(rng, 8, 4)
        cP = fs.determinant(Phi, Phi).conj()
        cp = fs.determinant(phu, phd)
        ov = cP @ cp
        e_fs = (cP @ (H @ cp)) / ov
        e, v = oa.local_energy_force_bias(ham, Phi, phu, phd)
        assert abs(e - e_fs) < 1e-10 * max(1.0, abs(e_fs))
        assert abs(np.exp(oa.log_overlap(ham, Phi, phu, phd)) - ov) < 1e-10 * abs(ov)
        for g in (0, 7, 30):
            vg = (cP @ (fs.one_body(s.L[g], 4, 4) @ cp)) / ov
            assert abs(v[g] - vg) < 1e-11 * max(1.0, abs(vg))


def test_complex_trial_orbitals_are_a_unitary_rotation():
    """exp(-i c S) with S real symmetric is unitary: Phi(x)^dagger Phi(x) =
    Phi0^T Phi0 for every x, and alpha = 1 gives the real form unchanged."""
    s = _small_system(9, 3, 3, K=4, seed=12)
    hr = _ham(s, 3, 3, dtau=0.01, U=s.U[:4])
    hc = oa.prepare(s.h, s.L, s.Phi0, s.U[:4], 3, 3, 0.01, alpha=-0.8j)
    x = np.random.default_rng(2).normal(size=(5, 4))
    Phi = oa.trial_orbitals(hc, x)
    gram = np.swapaxes(Phi.conj(), -1, -2) @ Phi
    assert np.allclose(gram, s.Phi0.T @ s.Phi0, atol=1e-12)
    assert not np.iscomplexobj(oa.trial_orbitals(hr, x))


def test_complex_trial_exact_eigenstate_walk():
    """L = 0 and [U_k, h] = 0 with a complex alpha: every sample is the ground
    determinant times a phase, so E_L = E0 for every pair while the path
    signs vary, and the walk keeps the mixed energy at E0."""
    s = _small_system(8, 3, 3, K=4, seed=21)
    rng = np.random.default_rng(6)
    U, _ = _commuting_U(s.h, 4, 3, rng, scale=0.8)
    ham = oa.prepare(s.h, np.zeros((2, 8, 8)), s.Phi0, U, 3, 3, 0.02, alpha=-1.0j)
    e0 = 2.0 * np.sum(np.linalg.eigvalsh(s.h)[:3])
    cfg = oa.OracleConfig(dtau=0.02, n_walkers=4, n_paths=6, seed=29, n_burn=2)
    st = oa.init(ham, cfg)
    phases = []
    for _ in range(3):
        st, d = oa.step(ham, cfg, st)
        assert np.allclose(d["measure"]["e_pair"], e0, atol=1e-10)
        num, den = d["mixed"]
        assert abs(num / den - e0) < 1e-10
        phases.append(np.angle(d["measure"]["S"]))
    assert np.ptp(np.concatenate([p.ravel() for p in phases])) > 0.1   # the samples' phases differ


def test_complex_trial_sampled_estimator_matches_quadrature():
    """K = 1 with a complex alpha: the path-sign-weighted average over paths
    sampled from |<Phi(x)|phi>| p(x) tends to <Psi_T|H|phi>/<Psi_T|phi> by
    Gauss-Hermite quadrature."""
    N, n = 4, 2
    s = _small_system(N, n, n, G=3, K=1, seed=43)
    rng = np.random.default_rng(8)
    ham = oa.prepare(s.h, s.L, s.Phi0, 10.0 * s.U[:1], n, n, 0.01, alpha=-1.0j)
    phu, phd = _rand_walker(rng, N, n), _rand_walker(rng, N, n)
    xq, wq = np.polynomial.hermite_e.hermegauss(80)
    num = den = 0.0
    for xj, wj in zip(xq, wq):
        Phi = oa.trial_orbitals(ham, np.array([xj]))
        ov = np.exp(oa.log_overlap(ham, Phi, phu, phd))
        e, _ = oa.local_energy_force_bias(ham, Phi, phu, phd)
        num, den = num + wj * ov * e, den + wj * ov
    e_exact = num / den
    W, P = 8, 32
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=W, n_paths=P, seed=79, n_burn=0)
    st = oa.init(ham, cfg)
    st.phi_up[:] = phu
    st.phi_dn[:] = phd
    logov = np.array([[oa.log_overlap(ham, st.Phi[w, p], phu, phd) for p in range(P)] for w in range(W)])
    alive = np.ones(W, dtype=bool)
    se = ss = 0.0
    for sweep in range(50):
        oa.mcmc_sweep(ham, cfg, st, logov, alive, 0, sweep, px.TAG_BURN_PROPOSE, px.TAG_BURN_ACCEPT)
        if sweep >= 10:
            m = oa.measure(ham, st)
            se += np.sum(m["S"] * m["e_pair"])
            ss += np.sum(m["S"])
    assert 0.05 < abs(ss) / (40 * W * P) < 0.95
    assert abs(se / ss - e_exact) < 0.02 * abs(e_exact)


@pytest.mark.parametrize("alpha", [1.0, -1j * math.sqrt(0.3)])
def test_multi_slice_trial_averages_to_the_projected_bra(alpha):
    """Two slices (Eq. (19), Eq. (32)) with one Cholesky vector as the hidden
    operator: <Phi(x)| = <phi_T| e^{-tT} e^{a* x_1 L} e^{-tT} e^{a* x_2 L}
    (a = alpha), so by the Gaussian identity E[e^{a* x L}] = e^{(a*)^2 L^2 / 2}
    for the many-body one-body operator L, the bra averaged over the hidden
    variables (2-D Gauss-Hermite) is <phi_T| e^{-tT} e^{(a*)^2 L^2/2} e^{-tT}
    e^{(a*)^2 L^2/2}, built here from dense Fock-space exponentials."""
    N, n = 4, 2
    s = _small_system(N, n, n, G=1, K=1, seed=61)
    fs = FockSpace(N, n, n)
    t = 0.2
    P = sla.expm(-t * s.h)
    L1 = 0.8 * s.L[:1] / np.max(np.abs(s.L[0]))
    ham = oa.prepare(s.h, L1, P @ s.Phi0, L1, n, n, 0.01, alpha=alpha, slices=2, slice_prop=P)
    assert oa.n_hidden(ham) == 2
    xq, wq = np.polynomial.hermite_e.hermegauss(40)
    bra = 0.0
    for x1, w1 in zip(xq, wq):
        for x2, w2 in zip(xq, wq):
            Phi = oa.trial_orbitals(ham, np.array([x1, x2]))
            bra = bra + (w1 * w2 / (2 * np.pi)) * np.conj(fs.determinant(Phi, Phi))
    Th = fs.one_body(s.h, n, n).toarray()
    Lh = fs.one_body(L1[0], n, n).toarray()
    a2 = np.conj(alpha) ** 2
    E = sla.expm(-t * Th)
    G = sla.expm(0.5 * a2 * (Lh @ Lh))
    exact = fs.determinant(s.Phi0, s.Phi0) @ E @ G @ E @ G
    assert np.max(np.abs(bra - exact)) < 1e-10 * np.max(np.abs(exact))
    # one slice is the single-slice form unchanged
    one = oa.prepare(s.h, L1, P @ s.Phi0, L1, n, n, 0.01, alpha=alpha)
    x = np.array([0.37])
    assert np.allclose(oa.trial_orbitals(one, x), oa.trial_orbitals(
        oa.prepare(s.h, L1, P @ s.Phi0, L1, n, n, 0.01, alpha=alpha, slices=1), x), atol=0)


def test_learned_proposal_is_refused_for_multi_slice_trials():
    """The proposal network's features and output live on the K variables of
    one slice, so a multi-slice trial with the learned proposal is rejected
    with a clear error (not a broadcasting failure deep in the sweep)."""
    N, n = 4, 2
    s = _small_system(N, n, n, G=2, K=1, seed=62)
    P = sla.expm(-0.2 * s.h)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, n, n, 0.01, slices=2, slice_prop=P)
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=2, n_paths=2, seed=5, n_burn=1, proposal="mlp")
    st = oa.init(ham, cfg)
    with pytest.raises(ValueError, match="one-slice"):
        oa.step(ham, cfg, st)
