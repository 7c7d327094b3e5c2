"""The general walker-side tensor-core contraction (contract_tcw_kernel:
Z_{p,g} = B_p^T (X_g phi_w) in split 16-bit arithmetic, any size of the FP64
path) against the FP64 oracle.

Tolerances are the mixed path's stated targets: at most 1e-4 Ha per walker
local energy and on the mixed energy; overlaps stay FP64 (1e-9); the force bias
is held to the contraction's accuracy (1e-4).  The error-controlled refinement
(pairs with the largest ||A_p^-1||_F recomputed in double-float) is on, as in
production; with a vanishing tolerance it recomputes every pair, which must then
match the oracle to 1e-9.
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
    "c0": (ai.SystemSpec(8, 4, 4, 32, 8, False, 1000), 16, 8, 0.01, 11),
    "ragged": (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 6, 5, 0.01, 12),
    "one_spin": (ai.SystemSpec(12, 3, 0, 20, 6, True, 78), 5, 4, 0.01, 13),
    "one_electron_each": (ai.SystemSpec(9, 1, 1, 11, 3, False, 79), 4, 3, 0.02, 14),
    "single_path": (ai.SystemSpec(10, 4, 3, 16, 5, False, 80), 7, 1, 0.01, 15),
    "n70_two_k_chunks": (ai.SystemSpec(70, 14, 13, 90, 10, True, 81), 3, 7, 0.005, 16),
    "medium": (ai.SystemSpec(50, 10, 10, 250, 50, True, 1001), 3, 32, 0.005, 17),
    "wide": (ai.SystemSpec(60, 20, 16, 120, 30, True, 85), 3, 4, 0.005, 18),
    # 150 orbitals, one spin of 45 electrons: the A image streamed with the Y images
    "one_spin_n150": (ai.SystemSpec(150, 45, 0, 300, 20, True, 83), 2, 3, 0.005, 19),
    # the largest workload's system: 200 orbitals, 40 + 40 electrons, 1000 Cholesky vectors
    "largest_shape": (ai.CONFIGS["largest_n200"][0], 2, 2, 0.005, 8),
}


def _measure_case(name, precision):
    spec, W, P, dtau, seed_off = SYSTEMS[name]
    seed = 300 + seed_off
    s = ai.make_system(spec)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, n_burn=2,
                          precision=precision, tc_form="walker", wait_polls=1 << 22)
    assert lib.contract_kernel(cfg) == "contract_tcw_kernel"
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, n_burn=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    assert np.any(ost.weight > 0)
    ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                               Phi=ost.Phi))
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    assert ctx.stats()["status"] == 0
    m = oa.measure(ham, ost)
    ctx.close()
    return e, obs, m, ost


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_general_walker_side_form_against_oracle(name):
    e, obs, m, ost = _measure_case(name, "fp16x3")
    live = ost.weight > 0
    d_walker = np.abs(e["e_walker"] - m["e_bar"])[live]
    print("%s: worst walker %.2e, force bias %.2e" % (name, d_walker.max(),
                                                      np.max(np.abs(obs["force_bias"] - m["v_bar"])[live])))
    assert np.max(np.abs(obs["logov"].real - m["logov"].real)) < 1e-9
    assert np.max(d_walker) < E_WALKER_TOL
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])[live]) < 1e-4
    num, den = oa.mixed_energy(ost.weight, m["e_bar"])
    assert abs(e["e_mix"] - num / den) < E_MIX_TOL
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])) > 1e-12      # the tensor cores really ran


@pytest.mark.parametrize("name", ["c0", "ragged", "medium"])
def test_general_walker_side_form_bf16(name):
    e, obs, m, ost = _measure_case(name, "bf16x3")
    live = ost.weight > 0
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])[live]) < E_WALKER_TOL
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])[live]) < 1e-4


@pytest.mark.parametrize("name", ["c0", "ragged", "one_spin", "one_electron_each", "n70_two_k_chunks", "wide"])
def test_tensor_core_overlaps_match_double_float(name):
    """The overlap matrices A_p = Phi_p^T phi_w on the tensor cores (exact 8-bit digit
    products, about 40 bits; overlap_form "auto") against the compensated
    double-float sums (overlap_form "df") from the same state: the log-overlaps of a
    measurement agree to 1e-10 (an entry's error of about 2^-38 of
    N max|Phi| max|phi|, times ||A^-1|| in log det A; 4.4e-11 measured at N = 8) and
    both match the oracle to 1e-9; two steps (ratio and Metropolis overlaps from the
    tensor cores as well) take the same Metropolis decisions and give the same
    weights to 1e-9 and paths and walkers to 1e-10."""
    spec, W, P, dtau, seed_off = SYSTEMS[name]
    seed = 500 + seed_off
    s = ai.make_system(spec)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, n_burn=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    m = oa.measure(ham, ost)
    res = {}
    for form in ("auto", "df"):
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, n_burn=2,
                              precision="fp16x6", tc_form="walker", wait_polls=1 << 22, overlap_form=form)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
        ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                                   Phi=ost.Phi))
        ctx.energy()
        lo = ctx.observables()["logov"]
        ctx.step(2)
        res[form] = (lo, ctx.state_arrays(), ctx.stats()["status"])
        ctx.close()
    (lt, gt, st_t), (ld, gd, st_d) = res["auto"], res["df"]
    assert st_t == 0 and st_d == 0
    print("%s: |dlogov| tc-df %.2e, tc-oracle %.2e" % (name, np.max(np.abs(lt - ld)),
                                                      np.max(np.abs(lt.real - m["logov"].real))))
    assert np.max(np.abs(lt - ld)) < 1e-10
    assert np.max(np.abs(lt.real - m["logov"].real)) < 1e-9
    assert np.array_equal(gt["x"], gd["x"])
    assert np.array_equal(gt["weight"] == 0, gd["weight"] == 0)
    assert np.allclose(gt["weight"], gd["weight"], rtol=1e-9, atol=0)
    assert np.max(np.abs(gt["Phi"] - gd["Phi"])) < 1e-10
    assert np.max(np.abs(gt["phi_up"] - gd["phi_up"])) < 1e-10


# the systems whose three-part operands fit the walker-side form's shared memory (45
# electrons in one spin do not: GEMM-Z's ring and transpose exceed it)
FP16X6_SYSTEMS = [n for n in SYSTEMS if n != "one_spin_n150"]


@pytest.mark.parametrize("name", FP16X6_SYSTEMS)
def test_three_part_operands_against_oracle(name):
    """fp16x6 (integer FP16 part and two FP16 remainders per operand, six products)
    with its refinement on: the same targets as fp16x3."""
    e, obs, m, ost = _measure_case(name, "fp16x6")
    live = ost.weight > 0
    d_walker = np.abs(e["e_walker"] - m["e_bar"])[live]
    print("%s: worst walker %.2e" % (name, d_walker.max()))
    assert np.max(np.abs(obs["logov"].real - m["logov"].real)) < 1e-9
    assert np.max(d_walker) < E_WALKER_TOL
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])[live]) < 1e-4
    num, den = oa.mixed_energy(ost.weight, m["e_bar"])
    assert abs(e["e_mix"] - num / den) < E_MIX_TOL


def test_three_part_operands_are_more_precise():
    """Without refinement, the per-pair local energies of fp16x6 against the FP64
    path sit well below fp16x3's (its operands carry about 31 bits against 20, the
    traces see FP32 entries): on the 120-orbital system the median error falls at
    least eightfold."""
    spec, run = ai.CONFIGS["large_n120"]
    s = ai.make_system(spec)
    W, P = 8, run.n_paths
    res, state = {}, None
    for prec in ("fp64", "fp16x3", "fp16x6"):
        kw = dict(tc_form="walker", wait_polls=1 << 24) if prec != "fp64" else {}
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau,
                              ai.philox_run_seed(4), n_burn=20, precision=prec, refine_tol=0.0, **kw)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
        if state is None:
            state = ctx.save_state()
        else:
            ctx.load_state(state)
        ctx.energy()
        res[prec] = ctx.observables()["e_local"]
        ctx.close()
    d3 = np.abs(res["fp16x3"] - res["fp64"]).ravel()
    d6 = np.abs(res["fp16x6"] - res["fp64"]).ravel()
    print("median per-pair error fp16x3 %.2e, fp16x6 %.2e; max %.2e, %.2e"
          % (np.median(d3), np.median(d6), d3.max(), d6.max()))
    assert np.median(d6) * 8 < np.median(d3)
    assert d6.max() * 4 < d3.max()


def test_refining_every_pair_matches_the_oracle():
    """With a vanishing tolerance every pair is recomputed in double-float by the
    refinement (Theta formed for the listed pairs in place of B_p), so per-pair
    energies and force biases match the oracle to the FP64 path's 1e-9."""
    spec, W, P, dtau, off = SYSTEMS["ragged"]
    s = ai.make_system(spec)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, 640, n_burn=2,
                          precision="fp16x3", tc_form="walker", refine_tol=1e-300, wait_polls=1 << 22)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=640, n_burn=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                               Phi=ost.Phi))
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    m = oa.measure(ham, ost)
    assert ctx.stats()["refined_pairs"] == W * P
    assert np.max(np.abs(obs["logov"] - m["logov"])) < 1e-9
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])) < 1e-9
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])) < 1e-9
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])) < 1e-9
    ctx.close()


@pytest.mark.parametrize("config,W", [("large_n120", 32), ("largest_n200", 12)])
def test_large_systems_against_fp64_gpu_path(config, W):
    """The mixed-precision and learned-proposal workloads' systems (120 orbitals,
    24 + 24 electrons, 600 vectors, 64 paths; 200 orbitals, 40 + 40, 1000 vectors,
    16 paths) after 20 burn-in sweeps: the general walker-side form, with and
    without its refinement, against the FP64 GPU path (pinned to the oracle by
    the other tests) from the same state.  Refined, every walker meets 1e-4 Ha
    and the mixed energy 0.1 mHa (the tensor-core values alone printed for the
    record)."""
    spec, run = ai.CONFIGS[config]
    s = ai.make_system(spec)
    P = run.n_paths
    res, refined, state = {}, {}, None
    for prec, tol in (("fp64", 1e-4), ("fp16x3", 1e-4), ("fp16x3", 0.0), ("fp16x6", 1e-4)):
        kw = dict(tc_form="walker", wait_polls=1 << 24) if prec != "fp64" else {}
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau,
                              ai.philox_run_seed(4), n_burn=20, precision=prec, refine_tol=tol, **kw)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
        if state is None:
            state = ctx.save_state()
        else:
            ctx.load_state(state)
        res[(prec, tol)] = ctx.energy(walkers=True)
        if prec != "fp64" and tol > 0:
            refined[(prec, tol)] = ctx.stats()["refined_pairs"]
        ctx.close()
    ref = res[("fp64", 1e-4)]
    d_walker = np.abs(res[("fp16x3", 1e-4)]["e_walker"] - ref["e_walker"])
    d_raw = np.abs(res[("fp16x3", 0.0)]["e_walker"] - ref["e_walker"])
    d_mix = abs(res[("fp16x3", 1e-4)]["e_mix"] - ref["e_mix"])
    print("%s: refined %d of %d pairs; worst walker %.2e (tensor cores alone %.2e), median %.2e, dE_mix %.2e"
          % (config, refined[("fp16x3", 1e-4)], W * P, d_walker.max(), d_raw.max(), np.median(d_walker), d_mix))
    assert np.max(d_walker) < E_WALKER_TOL
    assert d_mix < E_MIX_TOL
    assert 0 < refined[("fp16x3", 1e-4)] <= W * P
    if ("fp16x6", 1e-4) in res:
        d6 = np.abs(res[("fp16x6", 1e-4)]["e_walker"] - ref["e_walker"])
        print("%s fp16x6: refined %d, worst walker %.2e, dE_mix %.2e"
              % (config, refined[("fp16x6", 1e-4)], d6.max(), abs(res[("fp16x6", 1e-4)]["e_mix"] - ref["e_mix"])))
        assert np.max(d6) < E_WALKER_TOL
        assert abs(res[("fp16x6", 1e-4)]["e_mix"] - ref["e_mix"]) < E_MIX_TOL
        assert refined[("fp16x6", 1e-4)] < refined[("fp16x3", 1e-4)]
