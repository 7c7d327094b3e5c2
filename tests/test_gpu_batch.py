"""Batched stepping of several systems through one CUDA graph per step, and
the launch-shape autotuner: both must leave every result bit for bit equal to
stepping each context on its own with the built-in launch shapes."""

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


SYSTEMS = [
    (ai.SystemSpec(8, 4, 4, 32, 8, False, 1000), 16, 8, "fp64"),
    (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 6, 5, "fp16x3"),
    (ai.SystemSpec(50, 10, 10, 250, 50, True, 1001), 4, 8, "fp64"),
    (ai.SystemSpec(70, 14, 13, 90, 10, True, 81), 3, 7, "bf16x3"),
]


def _ctx(spec, W, P, prec, seed):
    s = ai.make_system(spec)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, 0.01, seed, n_burn=2, precision=prec)
    return lib.Context(cfg, s.h, s.L, s.Phi0, s.U, stream=torch.cuda.Stream())


def test_batch_graph_equals_individual_steps():
    batched = [_ctx(spec, W, P, prec, 50 + i) for i, (spec, W, P, prec) in enumerate(SYSTEMS)]
    single = [_ctx(spec, W, P, prec, 50 + i) for i, (spec, W, P, prec) in enumerate(SYSTEMS)]
    b = lib.Batch(batched)
    before = lib.launch_count()
    b.step(3)
    b.sync()
    graph_kernels = lib.launch_count() - before
    before = lib.launch_count()
    for c in single:
        c.step(3)
    torch.cuda.synchronize()
    assert graph_kernels == lib.launch_count() - before   # the graph runs the same kernels
    for cb, cs in zip(batched, single):
        assert cb.save_state() == cs.save_state()
        assert np.array_equal(cb.history(3), cs.history(3))
    # the contexts stay usable on their own between batch steps
    e = batched[1].energy()
    assert np.isfinite(e["e_mix"])
    b.step(1)
    b.sync()
    single[1].step(1)
    assert batched[1].save_state() == single[1].save_state()
    b.close()
    for c in batched + single:
        c.close()


def test_batch_graph_combs_like_individual_steps():
    """Whether a step combs is decided on the device, so the one captured graph
    serves the steps that comb and those that do not (the FP64 system with the
    cached half-rotated matrices, whose refresh is sized on the device too)."""
    def mk(i, spec, W, P, prec):
        s = ai.make_system(spec)
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, 0.01, 70 + i, n_burn=2,
                              precision=prec, pop_period=2, importance="local_energy", rcache=prec == "fp64")
        return lib.Context(cfg, s.h, s.L, s.Phi0, s.U, stream=torch.cuda.Stream())
    batched = [mk(i, *sy) for i, sy in enumerate(SYSTEMS[:2])]
    single = [mk(i, *sy) for i, sy in enumerate(SYSTEMS[:2])]
    b = lib.Batch(batched)
    b.step(4)
    b.sync()
    for c in single:
        c.step(4)
    torch.cuda.synchronize()
    for cb, cs in zip(batched, single):
        assert cb.save_state() == cs.save_state()
        assert cb.stats()["combs"] == cs.stats()["combs"] == 2
    b.close()
    for c in batched + single:
        c.close()


@pytest.mark.parametrize("prec", ["fp64", "fp16x3"])
def test_autotune_changes_no_result(prec):
    spec = ai.SystemSpec(50, 10, 10, 250, 50, True, 1001)
    a = _ctx(spec, 16, 32, prec, 7)
    ref = _ctx(spec, 16, 32, prec, 7)
    chosen = a.autotune()
    assert set(chosen) == {"overlap_warps_per_block", "tc_pairs_per_block", "trial_threads"}
    ea, er = a.energy(walkers=True), ref.energy(walkers=True)
    assert np.array_equal(ea["e_walker"], er["e_walker"])
    a.step(2)
    ref.step(2)
    assert a.save_state() == ref.save_state()
    a.close()
    ref.close()


def test_uneven_batch_of_sixteen_systems():
    """Sixteen synthetic molecules of uneven size (N ~ U[40, 125], n = N/5,
    Gamma = 5N, K = N), mixed precision, 32 walkers x 16 paths each, autotuned,
    one graph launch per step; one system checked against its own run."""
    specs = ai.batched_system_specs(16, n_range=(40, 125))
    ctxs = []
    for i, spec in enumerate(specs):
        c = _ctx(spec, 32, 16, "fp16x3", 900 + i)
        c.autotune()
        ctxs.append(c)
    b = lib.Batch(ctxs)
    b.step(2)
    b.sync()
    for c in ctxs:
        h = c.history(2)
        assert np.all(np.isfinite(h)) and c.stats()["status"] == 0
    k = 5
    alone = _ctx(specs[k], 32, 16, "fp16x3", 900 + k)
    alone.step(2)
    assert alone.save_state() == ctxs[k].save_state()
    b.close()
    for c in ctxs + [alone]:
        c.close()


def test_fresh_process_near_48k_shared_memory():
    """A first launch whose dynamic shared memory alone is below 48 KB but
    whose static + dynamic total is above it (trial orbitals at N = 60, n = 12:
    46,080 B dynamic) must work in a process where no larger launch came before."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import torch, afqmc_inputs as ai\n"
        "from paper_2505_18519_gb300 import afqmc as lib\n"
        "sp = ai.SystemSpec(60, 12, 12, 300, 60, True, 3001)\n"
        "s = ai.make_system(sp)\n"
        "cfg = lib.make_config(60, 12, 12, 300, 60, 8, 4, 0.005, 5, n_burn=1, precision='fp16x3')\n"
        "ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)\n"
        "ctx.step(1)\n"
        "print('E', ctx.energy()['e_mix'])\n" % root)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "E " in r.stdout


def test_batched_systems_step_like_the_oracle():
    """Every system of a batch, stepped through the one graph, against the
    oracle's step from the same state: FP64 systems to 1e-9 (weights relative;
    orbitals, paths and trial orbitals absolute, the same Metropolis decisions),
    and a mixed-precision system with its refinement recomputing every pair
    (refine_tol 1e-300), which makes its contraction double-float and its step
    equal to the oracle's within 1e-9 as well."""
    from oracle import afqmc as oa
    cases = [(ai.SystemSpec(8, 4, 4, 32, 8, False, 1000), 6, 4, "fp64", {}),
             (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 4, 3, "fp64", {}),
             (ai.SystemSpec(70, 14, 13, 90, 10, True, 81), 3, 4, "fp16x6", {"refine_tol": 1e-300})]
    ctxs, olds = [], []
    for i, (spec, W, P, prec, kw) in enumerate(cases):
        s = ai.make_system(spec)
        seed = 90 + i
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, 0.01, seed, n_burn=2,
                              precision=prec, **kw)
        c = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, stream=torch.cuda.Stream())
        ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, 0.01)
        ocfg = oa.OracleConfig(dtau=0.01, n_walkers=W, n_paths=P, seed=seed, n_burn=2)
        ost = oa.init(ham, ocfg)
        c.load_state_arrays(dict(step=ost.step, phi_up=ost.phi_up, phi_dn=ost.phi_dn, weight=ost.weight, x=ost.x,
                                 Phi=ost.Phi))
        ctxs.append(c)
        olds.append((ham, ocfg, ost))
    b = lib.Batch(ctxs)
    b.step(1)
    b.sync()
    for c, (ham, ocfg, ost) in zip(ctxs, olds):
        ost2, _ = oa.step(ham, ocfg, ost)
        g = c.state_arrays()
        assert g["step"] == ost2.step
        assert np.allclose(g["weight"], ost2.weight, rtol=1e-9, atol=0)
        assert np.max(np.abs(g["x"] - ost2.x)) < 1e-9
        assert np.max(np.abs(g["Phi"] - ost2.Phi)) < 1e-9
        assert np.max(np.abs(g["phi_up"] - ost2.phi_up)) < 1e-9
        if ost2.phi_dn.size:
            assert np.max(np.abs(g["phi_dn"] - ost2.phi_dn)) < 1e-9
    b.close()
    for c in ctxs:
        c.close()


def test_shared_contraction_launch_equals_individual_steps():
    """Systems on the walker-side tensor-core form share one persistent GEMM-Z
    launch per batch step (their blocks taken from one list); a system on another
    form keeps its own kernels.  Every result stays bit for bit equal to stepping
    each context alone, including a system whose walkers need two pair tiles and
    one with a single spin."""
    systems = [(ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 6, 5, "fp16x6"),
               (ai.SystemSpec(70, 14, 13, 90, 10, True, 81), 3, 7, "fp16x6"),
               (ai.SystemSpec(12, 3, 0, 20, 6, True, 78), 5, 4, "fp16x6"),
               (ai.SystemSpec(50, 10, 10, 250, 50, True, 1001), 4, 8, "fp16x3")]
    batched = [_ctx(spec, W, P, prec, 60 + i) for i, (spec, W, P, prec) in enumerate(systems)]
    single = [_ctx(spec, W, P, prec, 60 + i) for i, (spec, W, P, prec) in enumerate(systems)]
    b = lib.Batch(batched)
    assert b.shared_contractions == 3          # the fp16x3 system (N = 50) takes the N <= 64 form
    before = lib.launch_count()
    b.step(3)
    b.sync()
    graph_kernels = lib.launch_count() - before
    before = lib.launch_count()
    for c in single:
        c.step(3)
    torch.cuda.synchronize()
    # a context alone runs GEMM-Z of both its spins in one launch: three launches
    # per step become one
    assert graph_kernels == lib.launch_count() - before - 3 * (3 - 1)
    for cb, cs in zip(batched, single):
        assert cb.save_state() == cs.save_state()
        assert np.array_equal(cb.history(3), cs.history(3))
        assert cb.stats()["status"] == 0
    b.close()
    for c in batched + single:
        c.close()
