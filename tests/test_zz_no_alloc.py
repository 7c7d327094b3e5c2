"""The entry point that allocates nothing, against the context-based one and
against the oracle.

afqmc_local_energy_noalloc serves callers that cannot allocate device memory
(code inside another framework's operator hook whose memory must come from that
framework's pool, or loops where an allocation is not allowed): they pass
inputs and outputs only, and the intermediate matrices live in one fixed device
array inside the library.  Two calls in a row, on different walker states, must
agree with afqmc_energy/afqmc_observables of a context within the tolerances of
the other parity tests.  A smaller call after a larger one (other sizes, other
spin split) must match the oracle, so the larger call's leftovers in the shared
array do not leak into it; so must a one-spin batch (n_dn = 0), and a singular
pair must give log|ov| = -inf without disturbing the other pairs.
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

E_TOL = 1e-9


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2505_18519_gb300 import build
    build.build()
    lib.load_library()


def _noalloc_on(state, s, spec, P):
    W = state["weight"].shape[0]
    pairs = W * P
    dev = torch.device("cuda")
    h = torch.from_numpy(s.h).to(dev)
    L = torch.from_numpy(s.L).to(dev)
    Phi = torch.from_numpy(np.ascontiguousarray(state["Phi"])).to(dev)
    phi = np.concatenate([state["phi_up"], state["phi_dn"]], axis=2)
    phi_d = torch.from_numpy(np.ascontiguousarray(phi).view(np.float64)).to(dev)
    logov = torch.empty(2 * pairs, dtype=torch.float64, device=dev)
    e_local = torch.empty(2 * pairs, dtype=torch.float64, device=dev)
    fb = torch.empty(2 * pairs * spec.n_chol, dtype=torch.float64, device=dev)
    lib.local_energy_noalloc(spec.N, spec.n_up, spec.n_dn, spec.n_chol, pairs, P, h, L, Phi, phi_d, logov, e_local, fb)
    torch.cuda.synchronize()
    c = lambda t, *shape: t.cpu().numpy().view(np.complex128).reshape(*shape)
    return c(logov, W, P), c(e_local, W, P), c(fb, W, P, spec.n_chol)


def _oracle_state(spec, W, P, dtau, seed):
    """A state with complex walkers from the oracle (init, then one step)."""
    s = ai.make_system(spec)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, n_burn=2)
    st = oa.init(ham, ocfg)
    st, _ = oa.step(ham, ocfg, st)
    return s, ham, st


def _as_dict(st):
    return dict(phi_up=st.phi_up, phi_dn=st.phi_dn, weight=st.weight, x=st.x, Phi=st.Phi)


def _compare_pairs_with_oracle(ham, st, logov, e_local, v_pair, skip=()):
    W, P = st.x.shape[:2]
    for w in range(W):
        for p in range(P):
            if (w, p) in skip:
                continue
            lo = oa.log_overlap(ham, st.Phi[w, p], st.phi_up[w], st.phi_dn[w])
            e, v = oa.local_energy_force_bias(ham, st.Phi[w, p], st.phi_up[w], st.phi_dn[w])
            assert abs(logov[w, p].real - lo.real) < 1e-9, (w, p)
            assert abs(np.angle(np.exp(1j * (logov[w, p].imag - lo.imag)))) < 1e-9, (w, p)
            assert abs(e_local[w, p] - e) < E_TOL, (w, p)
            assert np.max(np.abs(v_pair[w, p] - v)) < 1e-9, (w, p)


def test_noalloc_matches_context_entry_point_two_calls():
    spec = ai.SystemSpec(37, 7, 5, 40, 9, True, 77)
    s = ai.make_system(spec)
    W, P = 6, 5
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, 0.01, 4242, n_burn=2)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    for call in range(2):
        ctx.step(1)
        ctx.energy()
        ref = ctx.observables()
        state = ctx.state_arrays()
        logov, e_local, v_pair = _noalloc_on(state, s, spec, P)
        assert np.max(np.abs(e_local - ref["e_local"])) < E_TOL, call
        assert np.max(np.abs(logov.real - ref["logov"].real)) < 1e-9, call
        assert np.max(np.abs(np.angle(np.exp(1j * (logov.imag - ref["logov"].imag))))) < 1e-9, call
        S = np.exp(1j * logov.imag)
        vbar = (S[:, :, None] * v_pair).sum(axis=1) / S.sum(axis=1)[:, None]
        assert np.max(np.abs(vbar - ref["force_bias"])) < 1e-9, call
    ctx.close()


def test_noalloc_smaller_call_after_a_larger_one_matches_oracle():
    """The first call (50 orbitals, 10 + 10 electrons, 96 pairs) leaves its Theta
    matrices in the shared array; the second (37 orbitals, 7 + 5 electrons, other
    walkers per pair block) reads only what it writes itself."""
    big = ai.SystemSpec(50, 10, 10, 250, 50, True, 1001)
    s_big, _, st_big = _oracle_state(big, 3, 32, 0.005, 611)
    _noalloc_on(_as_dict(st_big), s_big, big, 32)
    small = ai.SystemSpec(37, 7, 5, 40, 9, True, 77)
    s, ham, st = _oracle_state(small, 4, 3, 0.01, 612)
    logov, e_local, v_pair = _noalloc_on(_as_dict(st), s, small, 3)
    _compare_pairs_with_oracle(ham, st, logov, e_local, v_pair)


def test_noalloc_one_spin_matches_oracle():
    """n_dn = 0: the spin-down overlap is the empty determinant (log 1 = 0)."""
    spec = ai.SystemSpec(12, 3, 0, 20, 6, True, 78)
    s, ham, st = _oracle_state(spec, 5, 4, 0.01, 613)
    logov, e_local, v_pair = _noalloc_on(_as_dict(st), s, spec, 4)
    _compare_pairs_with_oracle(ham, st, logov, e_local, v_pair)


def test_noalloc_singular_pair():
    """A trial sample with a zero orbital has a zero overlap: that pair gets
    log|ov| = -inf and finite values; every other pair still matches the oracle."""
    spec = ai.SystemSpec(37, 7, 5, 40, 9, True, 77)
    s, ham, st = _oracle_state(spec, 3, 4, 0.01, 614)
    st.Phi[1, 2, :, 3] = 0.0
    logov, e_local, v_pair = _noalloc_on(_as_dict(st), s, spec, 4)
    assert logov[1, 2].real == -np.inf
    assert np.isfinite(e_local[1, 2]) and np.all(np.isfinite(v_pair[1, 2]))
    _compare_pairs_with_oracle(ham, st, logov, e_local, v_pair, skip={(1, 2)})


def test_noalloc_rejects_batches_beyond_its_scratch():
    cap = lib.load_library().afqmc_noalloc_scratch_bytes()
    assert cap == 32 << 20
    dev = torch.device("cuda")
    one = torch.zeros(2, dtype=torch.float64, device=dev)
    too_many = cap // (50 * 20 * 16) + 1
    with pytest.raises(lib.AfqmcError) as ei:
        lib.local_energy_noalloc(50, 10, 10, 250, too_many, 32, one, one, one, one, one, one, one)
    assert ei.value.status == 1 and "maximum" in str(ei.value)
    # a pair count whose byte size would wrap a 64-bit product is refused the same way
    with pytest.raises(lib.AfqmcError) as ei:
        lib.local_energy_noalloc(1, 1, 1, 1, 1 << 59, 1, one, one, one, one, one, one, one)
    assert ei.value.status == 1 and "maximum" in str(ei.value)
