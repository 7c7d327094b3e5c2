"""Failure detection without a GPU fault.

* A bounded wait that runs out: the tensor-core kernels poll their mbarriers at
  most ``wait_polls`` times.  With a limit of one poll the first wait on a copy
  or an MMA still in flight gives up; the block sets bit 4 of the device status
  word, lets its own copies and MMAs complete and returns.  The measurement then
  reports AFQMC_ERR_TIMEOUT, nothing faults, and a fresh context on the same GPU
  measures correctly.
* A non-finite value injected on the host: a state whose walker has a NaN
  orbital entry is loaded; that walker is removed in the step (weight 0, bit 2 of
  the status word) and every other walker still follows the oracle.
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

AFQMC_ERR_NUMERIC = 4
AFQMC_ERR_TIMEOUT = 6
STATUS_NONFINITE = 2
STATUS_TIMEOUT = 4


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2505_18519_gb300 import build
    build.build()
    lib.load_library()


def _raw_stats(ctx):
    """Statistics without raising on the status word."""
    out = np.empty(12)
    lib.load_library().afqmc_stats(ctx._ctx, out.ctypes.data, 12)
    return out


@pytest.mark.parametrize("spec,kernel", [
    (ai.SystemSpec(50, 10, 10, 250, 50, True, 1001), "contract_tcy_kernel"),   # walker-side form
    (ai.SystemSpec(70, 14, 13, 90, 10, True, 81), "contract_tc_kernel"),       # per-pair form
])
def test_tensor_core_wait_timeout_is_reported(spec, kernel):
    s = ai.make_system(spec)
    W, P, dtau, seed = 3, 8, 0.005, 97
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, n_burn=1,
                          precision="fp16x3", refine_tol=0.0, wait_polls=1)
    assert lib.contract_kernel(cfg) == kernel
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    with pytest.raises(lib.AfqmcError) as ei:
        ctx.energy()
    assert ei.value.status == AFQMC_ERR_TIMEOUT
    assert int(_raw_stats(ctx)[4]) & STATUS_TIMEOUT
    ctx.close()
    torch.cuda.synchronize()                      # the device is still usable
    # a fresh context with the default limit measures as the oracle does
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, n_burn=1,
                          precision="fp16x3", refine_tol=0.0)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, n_burn=1)
    ost = oa.init(ham, ocfg)
    e = ctx.energy(walkers=True)
    assert ctx.stats()["status"] == 0
    m = oa.measure(ham, ost)
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])) < 1e-4
    ctx.close()


def test_nonfinite_orbital_removes_only_its_walker():
    spec = ai.SystemSpec(8, 4, 4, 32, 8, False, 1000)
    s = ai.make_system(spec)
    W, P, dtau, seed = 8, 4, 0.01, 55
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, n_burn=2)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, n_burn=2)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ost = oa.init(ham, ocfg)
    ost.phi_up[3, 5, 1] = np.nan                  # one walker's orbital entry
    ctx.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                               Phi=ost.Phi))
    ctx.step(1)
    ost2, d = oa.step(ham, ocfg, ost)
    g = ctx.state_arrays()
    assert g["weight"][3] == 0.0 and ost2.weight[3] == 0.0
    keep = np.arange(W) != 3
    assert np.allclose(g["weight"][keep], ost2.weight[keep], rtol=1e-9, atol=0)
    assert np.all(ost2.weight[keep] > 0)
    assert np.max(np.abs(g["phi_up"][keep] - ost2.phi_up[keep])) < 1e-9
    assert np.max(np.abs(g["phi_dn"][keep] - ost2.phi_dn[keep])) < 1e-9
    assert np.max(np.abs(g["x"] - ost2.x)) < 1e-9
    rec = ctx.history(1)[0]                       # the step's mixed energy leaves the walker out
    num, den = d["mixed"]
    assert np.isfinite(rec[0]) and abs(rec[0] / rec[1] - num / den) < 1e-9
    assert int(_raw_stats(ctx)[4]) & STATUS_NONFINITE
    with pytest.raises(lib.AfqmcError) as ei:
        ctx.energy()
    assert ei.value.status == AFQMC_ERR_NUMERIC
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp16x3"])
def test_walker_blocks_reproduce_one_context(precision):
    """Two contexts holding walker blocks [0, W/2) and [W/2, W) (walker_offset)
    reproduce one context of W walkers bit for bit, and their mixed-estimator sums
    add up to its sums: the sharded multi-GPU run on one GPU."""
    spec = ai.SystemSpec(37, 7, 5, 40, 9, True, 77)
    s = ai.make_system(spec)
    W, P, dtau, seed = 6, 8, 0.01, 1234
    full = lib.Context(lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, n_burn=3,
                                       precision=precision), s.h, s.L, s.Phi0, s.U)
    halves = [lib.Context(lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W // 2, P, dtau, seed,
                                          n_burn=3, precision=precision, walker_offset=off), s.h, s.L, s.Phi0, s.U)
              for off in (0, W // 2)]
    for c in [full] + halves:
        c.step(3)
    a = full.state_arrays()
    b = [h.state_arrays() for h in halves]
    for key in ("phi_up", "phi_dn", "weight", "x", "Phi"):
        assert np.array_equal(a[key], np.concatenate([b[0][key], b[1][key]])), key
    hf = full.history(3)
    hh = halves[0].history(3) + halves[1].history(3)
    assert np.allclose(hh[:, :3], hf[:, :3], rtol=1e-12, atol=1e-12)
    assert np.array_equal(hh[:, 3], hf[:, 3])
    for c in [full] + halves:
        c.close()
