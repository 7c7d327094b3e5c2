"""The whole method against full configuration interaction (FCI).

* Exact trial, no bias and no variance.  When h, every L_g and every trial
  generator U_k are diagonal in one orthonormal basis Q, every eigenstate of H is
  an occupation state of Q's orbitals, a Slater determinant, and every trial
  sample exp(sum_k x_k U_k) Phi0 spans the same orbitals as Phi0.  With Phi0 the
  occupied orbitals of the ground configuration the trial is exact, so the local
  energy <Psi_T|H|phi> / <Psi_T|phi> of every walker equals the FCI energy whatever
  the walker (Sec. II: the mixed estimator is exact for an eigenstate trial), and
  so does the mixed estimate of every step: no phaseless bias and no statistical
  error.  The ground configuration comes from the closed form of the diagonal
  Hamiltonian, E(n) = sum_i eps_i n_i + 1/2 sum_g [(sum_i l_gi n_i)^2 -
  sum_i l_gi^2 n_i], and is checked against the lowest eigenvalue of H built
  literally in determinant space.
"""

import itertools

import numpy as np
import pytest
import scipy.sparse.linalg as ssla

import afqmc_inputs as ai
from fock_space import FockSpace
from oracle import afqmc as oa


def commuting_system(N=8, n=4, G=12, K=5, seed=7):
    """h, L, U diagonal in a random orthonormal basis Q; returns them with the
    exact trial (orbitals of the ground configuration) and the FCI energy."""
    rng = np.random.default_rng(seed)
    Q = np.linalg.qr(rng.standard_normal((N, N)))[0]
    eps = np.sort(rng.uniform(-2.0, 0.0, N))
    lg = rng.normal(0.0, 0.15, (G, N))
    ug = rng.normal(0.0, 0.3, (K, N))
    rot = lambda d: (Q * d) @ Q.T                         # Q diag(d) Q^T
    h = rot(eps)
    L = np.stack([rot(l) for l in lg])
    U = np.stack([rot(u) for u in ug])

    def e_conf(occ_up, occ_dn):
        nocc = np.zeros(N)
        nocc[list(occ_up)] += 1
        nocc[list(occ_dn)] += 1
        return eps @ nocc + 0.5 * sum((l @ nocc) ** 2 - (l * l) @ nocc for l in lg)

    confs = list(itertools.combinations(range(N), n))
    e_best, occ_up, occ_dn = min((e_conf(a, b), a, b) for a in confs for b in confs)
    assert occ_up == occ_dn                               # a closed-shell ground configuration
    H = FockSpace(N, n, n).hamiltonian(h, L)
    e_fci = float(ssla.eigsh(H, k=1, which="SA")[0][0])
    assert abs(e_fci - e_best) < 1e-10                    # the closed form is the FCI ground state
    return h, L, U, Q[:, list(occ_up)].copy(), e_fci


def random_walkers(rng, W, N, n_up, n_dn):
    """W random orthonormal complex orbital matrices per spin."""
    def one(n):
        z = rng.normal(size=(W, N, n)) + 1j * rng.normal(size=(W, N, n))
        return np.stack([np.linalg.qr(a)[0] for a in z])
    return one(n_up), one(n_dn)


def test_exact_trial_has_no_bias_and_no_variance():
    h, L, U, Phi0, e_fci = commuting_system()
    ham = oa.prepare(h, L, Phi0, U, 4, 4, 0.01)
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=8, n_paths=4, seed=5, n_burn=3, e_shift=e_fci, pop_period=2)
    st = oa.init(ham, cfg)
    # the trial samples, and so the initial walkers, are the ground determinant itself (the propagator
    # keeps its orbitals' span): start from random orthonormal walkers instead
    st.phi_up, st.phi_dn = random_walkers(np.random.default_rng(3), 8, 8, 4, 4)
    n_acc = 0
    for _ in range(6):
        st, d = oa.step(ham, cfg, st)
        num, den = d["mixed"]
        assert abs(num / den - e_fci) < 1e-10
        assert np.max(np.abs(d["e_bar"] - e_fci)) < 1e-10     # every walker, every path sample
        n_acc += d["n_accept"]
    assert np.all(st.weight > 0)
    assert n_acc > 0                                          # the paths did move
    # the walkers are not eigenstates themselves: the energy of a walker's own determinant is not E_FCI
    fs = FockSpace(8, 4, 4)
    H = fs.hamiltonian(h, L)
    c = fs.determinant(st.phi_up[0], st.phi_dn[0])
    assert abs((np.conj(c) @ (H @ c)).real / np.vdot(c, c).real - e_fci) > 1e-3


@pytest.mark.gpu
def test_exact_trial_long_run_on_the_gpu():
    """The FP64 CUDA path on the exact-trial system for 2000 steps (512 walkers x 16
    paths, comb every 5 steps): every step's mixed energy is the FCI energy."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2505_18519_gb300 import afqmc as lib, build
    build.build()
    lib.load_library()
    h, L, U, Phi0, e_fci = commuting_system()
    steps = 2000
    cfg = lib.make_config(8, 4, 4, L.shape[0], U.shape[0], 512, 16, 0.01, 99, n_burn=20, e_shift=e_fci, pop_period=5)
    ctx = lib.Context(cfg, h, L, Phi0, U)
    st = ctx.state_arrays()
    st["phi_up"], st["phi_dn"] = random_walkers(np.random.default_rng(4), 512, 8, 4, 4)
    ctx.load_state_arrays(st)
    ctx.step(steps)
    hist = ctx.history(steps)
    st = ctx.stats()
    ctx.close()
    e = hist[:, 0] / hist[:, 1]
    assert np.max(np.abs(e - e_fci)) < 1e-9
    assert st["status"] == 0 and st["live_walkers"] == 512
