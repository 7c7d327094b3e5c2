"""Complex and multi-slice trial samples on the GPU (FP64 path) against the
oracle: the single-slice VAFQMC form Phi(x) = exp(alpha sum_k x_k U_k) Phi0 with
alpha = -i sqrt(s) (Eq. (30)), and the multi-slice form
exp(alpha S_m) P ... P exp(alpha S_1) Phi0 (Eq. (19), (32)) with P = exp(-t h),
for real and complex alpha.  Overlaps and Green's functions take Phi^dagger.

Tolerances as for the real trial: per-walker and per-pair local energies,
log-overlaps, force bias, orbitals 1e-9; weights 1e-9 relative; Metropolis
decisions exact.
"""

import math

import numpy as np
import pytest
import scipy.linalg as sla

import afqmc_inputs as ai
from oracle import afqmc as oa

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2505_18519_gb300 import afqmc as lib  # noqa: E402

TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2505_18519_gb300 import build
    build.build()
    lib.load_library()


C0 = ai.SystemSpec(8, 4, 4, 32, 8, False, 1000)
CASES = {
    "complex_c0": (C0, 8, 4, 0.01, -1j * math.sqrt(0.3), 1),
    "complex_ragged": (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 4, 3, 0.01, -1j * math.sqrt(0.2), 1),
    "complex_two_slices": (C0, 6, 4, 0.01, -1j * math.sqrt(0.3), 2),
    "real_two_slices": (C0, 6, 4, 0.01, 1.0, 2),
    "complex_three_slices_one_spin": (ai.SystemSpec(12, 3, 0, 20, 6, True, 78), 5, 3, 0.01, 0.2 - 0.5j, 3),
}


def _setup(name, seed, **kw):
    spec, W, P, dtau, alpha, slices = CASES[name]
    s = ai.make_system(spec)
    Pm = sla.expm(-0.2 * s.h) if slices > 1 else None
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau, alpha=alpha, slices=slices, slice_prop=Pm)
    okw = {k: v for k, v in kw.items() if k in ("n_sweeps", "n_burn", "proposal", "pcn_beta")}
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, **okw)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, trial_alpha=alpha,
                          trial_slices=slices, **kw)
    assert lib.contract_kernel(cfg) == "contract_fp64c_kernel"
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, slice_prop=Pm)
    return ham, ocfg, ctx


def _as_dict(st):
    # the library keeps the orbitals of any trial other than the real one-slice form as complex
    return dict(step=st.step, phi_up=st.phi_up, phi_dn=st.phi_dn, weight=st.weight, x=st.x,
                Phi=st.Phi.astype(np.complex128))


def _compare_state(g, ost):
    assert g["step"] == ost.step
    assert np.allclose(g["weight"], ost.weight, rtol=TOL, atol=0)
    assert np.max(np.abs(g["x"] - ost.x)) < TOL                 # the same Metropolis decisions
    assert np.max(np.abs(g["Phi"] - ost.Phi)) < TOL
    assert np.max(np.abs(g["phi_up"] - ost.phi_up)) < TOL
    if ost.phi_dn.size:
        assert np.max(np.abs(g["phi_dn"] - ost.phi_dn)) < TOL


@pytest.mark.parametrize("name", list(CASES))
def test_init_matches_oracle(name):
    """Initial walkers Phi(x_w), paths and burn-in: the complex trial orbitals
    from the Chebyshev series of exp(alpha S) (and the slice chain) equal the
    oracle's eigendecomposition to 1e-9, so every Metropolis decision agrees."""
    ham, ocfg, ctx = _setup(name, 71, n_burn=3)
    ost = oa.init(ham, ocfg)
    g = ctx.state_arrays()
    if name != "real_two_slices":
        assert np.iscomplexobj(g["Phi"]) and np.max(np.abs(g["Phi"].imag)) > 1e-3
    _compare_state(g, ost)
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_measure_and_one_step_match_oracle(name):
    ham, ocfg, ctx = _setup(name, 73, n_burn=2, n_sweeps=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    assert np.any(ost.weight > 0)
    ctx.load_state_arrays(_as_dict(ost))
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    m = oa.measure(ham, ost)
    assert np.max(np.abs(obs["logov"].real - m["logov"].real)) < TOL
    assert np.max(np.abs(np.angle(np.exp(1j * (obs["logov"].imag - m["logov"].imag))))) < TOL
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])) < TOL
    live = ost.weight > 0
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])[live]) < TOL
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])[live]) < TOL
    ctx.step(1)
    ost2, d = oa.step(ham, ocfg, ost)
    _compare_state(ctx.state_arrays(), ost2)
    rec = ctx.history(1)[0]
    num, den = d["mixed"]
    assert abs(rec[0] / rec[1] - num / den) < TOL
    assert rec[3] == d["n_accept"]
    ctx.close()


def test_complex_trial_checkpoint_resume_is_bitwise():
    ham, ocfg, a = _setup("complex_two_slices", 75, n_burn=2)
    _, _, b = _setup("complex_two_slices", 75, n_burn=2)
    a.step(2)
    blob = a.save_state()
    a.step(2)
    b.load_state(blob)
    b.step(2)
    assert a.save_state() == b.save_state()
    a.close()
    b.close()


# Mixed precision: the walker-side tensor-core contraction with the complex
# trial-side factor B_p = conj(Phi_p) A_p^-T; its stated targets are 1e-4 Ha per
# walker and on the mixed energy.  Overlaps, trial orbitals and every step after
# the contraction stay FP64 or double-float.
MIXED_TOL = 1e-4


def _setup_mixed(name, seed, precision, **kw):
    spec, W, P, dtau, alpha, slices = CASES[name]
    s = ai.make_system(spec)
    Pm = sla.expm(-0.2 * s.h) if slices > 1 else None
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, trial_alpha=alpha,
                          trial_slices=slices, precision=precision, **kw)
    assert lib.contract_kernel(cfg) == "contract_tcw_kernel"
    return lib.Context(cfg, s.h, s.L, s.Phi0, s.U, slice_prop=Pm)


@pytest.mark.parametrize("precision", ["fp16x6", "fp16x3"])
@pytest.mark.parametrize("name", ["complex_c0", "complex_ragged", "complex_two_slices",
                                  "complex_three_slices_one_spin"])
def test_mixed_precision_measure_and_step_match_oracle(name, precision):
    """The measurement of the oracle's state after one step: log-overlaps to
    1e-9 (FP64), per-pair and per-walker local energies, force bias and the
    mixed energy to 1e-4; then one step: the same Metropolis decisions and
    weights within 1e-4 relative (the mixed force bias enters the propagation);
    with a vanishing refinement tolerance every pair is recomputed in FP64 and
    the measurement matches the oracle to 1e-9."""
    ham, ocfg, _ = _setup(name, 77, n_burn=2, n_sweeps=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    m = oa.measure(ham, ost)
    live = ost.weight > 0
    assert np.any(live)
    ctx = _setup_mixed(name, 77, precision, n_burn=2, n_sweeps=2)
    ctx.load_state_arrays(_as_dict(ost))
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    assert np.max(np.abs(obs["logov"].real - m["logov"].real)) < TOL
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])[live]) < MIXED_TOL
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])[live]) < MIXED_TOL
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])[live]) < MIXED_TOL
    num, den = oa.mixed_energy(ost.weight, m["e_bar"])
    assert abs(e["e_mix"] - num / den) < MIXED_TOL
    ctx.step(1)
    ost2, _ = oa.step(ham, ocfg, ost)
    g = ctx.state_arrays()
    assert np.max(np.abs(g["x"] - ost2.x)) < TOL                 # the same Metropolis decisions
    assert np.allclose(g["weight"], ost2.weight, rtol=MIXED_TOL, atol=0)
    ctx.close()
    exact = _setup_mixed(name, 77, precision, n_burn=2, n_sweeps=2, refine_tol=1e-300)
    exact.load_state_arrays(_as_dict(ost))
    e = exact.energy(walkers=True)
    obs = exact.observables()
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])[live]) < TOL
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])[live]) < TOL
    exact.close()
