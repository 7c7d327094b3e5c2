"""The entry point that allocates nothing, against the context-based one.

afqmc_local_energy_noalloc serves callers that cannot allocate device memory
(code inside another framework's operator hook whose memory must come from that
framework's pool, or loops where an allocation is not allowed): they pass
inputs and outputs only, and the intermediate matrices live in one fixed device
array inside the library.  Two calls in a row, on different walker states, must
agree with afqmc_energy/afqmc_observables of a context within the tolerances of
the other parity tests; the second call also shows that the previous call's
leftovers in the shared array do not leak into the result.
"""

import numpy as np
import pytest

import afqmc_inputs as ai

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
        assert np.max(np.abs(e_local - ref["e_local"])) < 1e-9, call
        assert np.max(np.abs(logov.real - ref["logov"].real)) < 1e-9, call
        assert np.max(np.abs(np.angle(np.exp(1j * (logov.imag - ref["logov"].imag))))) < 1e-9, call
        S = np.exp(1j * logov.imag)
        vbar = (S[:, :, None] * v_pair).sum(axis=1) / S.sum(axis=1)[:, None]
        assert np.max(np.abs(vbar - ref["force_bias"])) < 1e-9, call
    ctx.close()


def test_noalloc_rejects_batches_beyond_its_scratch():
    cap = lib.load_library().afqmc_noalloc_scratch_bytes()
    assert cap == 32 << 20
    dev = torch.device("cuda")
    one = torch.zeros(2, dtype=torch.float64, device=dev)
    too_many = cap // (50 * 20 * 16) + 1
    with pytest.raises(lib.AfqmcError) as ei:
        lib.local_energy_noalloc(50, 10, 10, 250, too_many, 32, one, one, one, one, one, one, one)
    assert ei.value.status == 1 and "maximum" in str(ei.value)
