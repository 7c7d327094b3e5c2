"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Element by element on the same seeded inputs and the same counter-based
random streams: per-pair log-overlaps, local energies and force-bias values,
per-walker path averages, one full leapfrog step from a shared state, short
trajectories from init, sampled walkers of the full-size medium workload, the
Philox generator bit for bit, checkpoint/resume, frozen dead walkers and the
constraint and proposal variants.

Tolerances (FP64 everywhere, both sides): per-walker local energy 1e-9 Ha
(absolute); log-overlaps, force bias, orbitals 1e-9; weights 1e-9 relative.
Metropolis decisions must agree exactly (a draw within 1e-9 of its threshold
would be reported as such).
"""

import ctypes
import dataclasses
import os
import subprocess
import tempfile

import numpy as np
import pytest

import afqmc_inputs as ai
from oracle import afqmc as oa
from oracle import philox as px

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


def _setup(spec, W, P, dtau, seed, **kw):
    s = ai.make_system(spec)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, dtau)
    okw = {k: v for k, v in kw.items() if k in ("n_sweeps", "n_burn", "constraint", "proposal", "pcn_beta", "e_shift",
                                                 "importance", "pop_period")}
    ocfg = oa.OracleConfig(dtau=dtau, n_walkers=W, n_paths=P, seed=seed, **okw)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, dtau, seed, **kw)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    return s, ham, ocfg, ctx


def _as_dict(st: oa.State):
    return dict(step=st.step, phi_up=st.phi_up, phi_dn=st.phi_dn, weight=st.weight, x=st.x, Phi=st.Phi)


def _phase_diff(a, b):
    return np.abs(np.angle(np.exp(1j * (a - b))))


def _compare_measure(ctx, ham, ost, tol=E_TOL):
    e = ctx.energy(walkers=True)
    obs = ctx.observables()
    m = oa.measure(ham, ost)
    assert np.max(np.abs(obs["logov"].real - m["logov"].real)) < 1e-9
    assert np.max(_phase_diff(obs["logov"].imag, m["logov"].imag)) < 1e-9
    assert np.max(np.abs(obs["e_local"] - m["e_pair"])) < tol
    assert np.max(np.abs(e["e_walker"] - m["e_bar"])) < tol
    assert np.max(np.abs(obs["force_bias"] - m["v_bar"])) < 1e-9
    num, den = oa.mixed_energy(ost.weight, m["e_bar"])
    assert den > 0, "every walker of this state is dead: the mixed energy is undefined"
    assert abs(e["e_mix"] - num / den) < tol
    return e, m


def _compare_state(g, ost, rel=1e-9):
    assert g["step"] == ost.step
    assert np.allclose(g["weight"], ost.weight, rtol=rel, atol=0), np.max(np.abs(g["weight"] - ost.weight))
    assert np.array_equal(g["weight"] == 0, ost.weight == 0)
    assert np.max(np.abs(g["phi_up"] - ost.phi_up)) < 1e-9
    if ost.phi_dn.size:
        assert np.max(np.abs(g["phi_dn"] - ost.phi_dn)) < 1e-9
    assert np.max(np.abs(g["x"] - ost.x)) < 1e-9          # same Metropolis decisions
    assert np.max(np.abs(g["Phi"] - ost.Phi)) < 1e-9


SYSTEMS = {
    "c0": (ai.SystemSpec(8, 4, 4, 32, 8, False, 1000), 16, 8, 0.01),
    "ragged": (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 6, 5, 0.01),
    "one_spin": (ai.SystemSpec(12, 3, 0, 20, 6, True, 78), 5, 4, 0.01),
    "one_electron_each": (ai.SystemSpec(9, 1, 1, 11, 3, False, 79), 4, 3, 0.02),
    "single_path": (ai.SystemSpec(10, 4, 3, 16, 5, False, 80), 7, 1, 0.01),
    "medium": (ai.SystemSpec(50, 10, 10, 250, 50, True, 1001), 4, 32, 0.005),
    # the walker-side FP64 contraction (blocks of 8 or 16 pairs of a walker): a ragged
    # last block, one spin only, and 16 pairs per block
    "ragged_walker_side": (ai.SystemSpec(37, 7, 5, 40, 9, True, 77), 3, 11, 0.01),
    "one_spin_walker_side": (ai.SystemSpec(12, 3, 0, 20, 6, True, 78), 3, 9, 0.01),
    "two_blocks_walker_side": (ai.SystemSpec(20, 5, 4, 60, 7, True, 82), 2, 35, 0.01),
    # N = 200 with 40 + 40 electrons and 1000 Cholesky vectors (the largest workload's
    # system, few walkers): Theta streamed in row slabs through the contraction, the
    # propagation's work arrays in global memory, a ragged last column block (200 = 6 x 32 + 8).
    # Two walkers, as the phaseless constraint kills one of them in the first step here
    "largest_shape": (ai.CONFIGS["largest_n200"][0], 2, 2, 0.005),
    # one spin, Theta slabs with the propagation still in shared memory
    "one_spin_slab": (ai.SystemSpec(150, 45, 0, 300, 20, True, 83), 2, 3, 0.005),
}

# Per-case offsets of the Philox run seeds, fixed here so that renaming a case does
# not move its seed.  With two walkers and two burn-in sweeps the first step can
# kill every walker of the N = 200 case: offset 8 keeps walker 0 alive (checked on
# the oracle); the tests assert a live walker before comparing mixed energies.
CASE_SEED = {"c0": 2, "ragged": 6, "one_spin": 8, "one_electron_each": 17, "single_path": 11, "medium": 6,
             "ragged_walker_side": 18, "one_spin_walker_side": 20, "two_blocks_walker_side": 22,
             "largest_shape": 8, "one_spin_slab": 13}


def _seed(base, name):
    return base + CASE_SEED[name]


# ---------------------------------------------------------------- generator

def test_philox_bitwise_equal_to_oracle():
    n = 1 << 18
    out = torch.empty(4 * n, dtype=torch.int32, device="cuda")
    key = 0x0123456789ABCDEF
    lib.philox_fill(out, n, 11, 22, 33, 44, key)
    gpu = out.cpu().numpy().view(np.uint32).reshape(n, 4)
    ctr = np.stack([np.arange(n, dtype=np.uint64) + 11, np.full(n, 22), np.full(n, 33), np.full(n, 44)], axis=1)
    ref = px.philox4x32_10(ctr.astype(np.uint32), (key & 0xFFFFFFFF, key >> 32))
    assert np.array_equal(gpu, ref)


_CURAND_SRC = r"""
#include <curand_kernel.h>
__global__ void k(unsigned* out, long long n, unsigned c1, unsigned c2, unsigned c3, unsigned k0, unsigned k1) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint4 c = make_uint4((unsigned)i, c1, c2, c3);
  uint2 key = make_uint2(k0, k1);
  uint4 r = curand_Philox4x32_10(c, key);
  out[4*i] = r.x; out[4*i+1] = r.y; out[4*i+2] = r.z; out[4*i+3] = r.w;
}
extern "C" int run(unsigned* out, long long n, unsigned c1, unsigned c2, unsigned c3, unsigned k0, unsigned k1) {
  k<<<(unsigned)((n + 255) / 256), 256>>>(out, n, c1, c2, c3, k0, k1);
  return (int)cudaDeviceSynchronize();
}
"""


def test_philox_matches_an_independent_implementation():
    """The library's Philox4x32-10 against the one in CUDA's curand headers."""
    d = tempfile.mkdtemp()
    src, so = os.path.join(d, "ref.cu"), os.path.join(d, "ref.so")
    open(src, "w").write(_CURAND_SRC)
    r = subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared", "-Xcompiler", "-fPIC",
                        "-o", so, src], capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("could not build the curand reference: " + r.stderr[-300:])
    ref_lib = ctypes.CDLL(so)
    n = 1 << 16
    a = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    b = torch.zeros(4 * n, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert ref_lib.run(ctypes.c_void_p(a.data_ptr()), ctypes.c_longlong(n), 5, 6, 7, 0xDEADBEEF, 0x12345678) == 0
    lib.philox_fill(b, n, 0, 5, 6, 7, 0x12345678DEADBEEF)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


# ---------------------------------------------------------------- measurement and one step

@pytest.mark.parametrize("name", list(SYSTEMS))
def test_measure_matches_oracle(name):
    spec, W, P, dtau = SYSTEMS[name]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=_seed(900, name), n_burn=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)                  # complex walkers
    assert np.any(ost.weight > 0), "the oracle's first step killed every walker: choose another seed"
    ctx.load_state_arrays(_as_dict(ost))
    _compare_measure(ctx, ham, ost)
    ctx.close()


@pytest.mark.parametrize("name", list(SYSTEMS))
def test_one_step_matches_oracle(name):
    spec, W, P, dtau = SYSTEMS[name]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=_seed(500, name), n_burn=2, n_sweeps=2)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    assert np.any(ost.weight > 0), "the oracle's first step killed every walker: choose another seed"
    ctx.load_state_arrays(_as_dict(ost))
    ctx.step(1)
    ost2, d = oa.step(ham, ocfg, ost)
    g = ctx.state_arrays()
    _compare_state(g, ost2)
    rec = ctx.history(1)[0]
    num, den = d["mixed"]
    assert den > 0
    assert abs(rec[0] / rec[1] - num / den) < E_TOL
    assert rec[3] == d["n_accept"]
    ctx.close()


@pytest.mark.parametrize("constraint", ["combined", "separate", "half_plane"])
@pytest.mark.parametrize("proposal", ["prior", "pcn"])
def test_variants_match_oracle(constraint, proposal):
    spec, W, P, dtau = SYSTEMS["c0"]
    kw = dict(n_burn=3, constraint=constraint, proposal=proposal, pcn_beta=0.4, e_shift=11.0)
    s, ham, ocfg, ctx = _setup(spec, W, P, 0.05, seed=31, **kw)
    ost = oa.init(ham, ocfg)
    ctx.load_state_arrays(_as_dict(ost))
    for _ in range(3):
        ctx.step(1)
        ost, _ = oa.step(ham, ocfg, ost)
        _compare_state(ctx.state_arrays(), ost)
    ctx.close()


def test_local_energy_importance_matches_oracle():
    """Weights with |I| = exp(-tau Re E_w) (the local-energy form of Sec. III A)."""
    spec, W, P, dtau = SYSTEMS["c0"]
    kw = dict(n_burn=3, importance="local_energy", e_shift=11.0)
    s, ham, ocfg, ctx = _setup(spec, W, P, 0.05, seed=37, **kw)
    ost = oa.init(ham, ocfg)
    hyb = ost.copy()
    ctx.load_state_arrays(_as_dict(ost))
    for _ in range(3):
        ctx.step(1)
        ost, _ = oa.step(ham, ocfg, ost)
        hyb, _ = oa.step(ham, dataclasses.replace(ocfg, importance="hybrid"), hyb)
        _compare_state(ctx.state_arrays(), ost)
    live = (ost.weight > 0) & (hyb.weight > 0)
    assert live.sum() >= W // 2
    assert np.max(np.abs(ost.weight[live] / hyb.weight[live] - 1.0)) > 1e-4   # the two forms differ
    ctx.close()


@pytest.mark.parametrize("importance,period", [("hybrid", 1), ("local_energy", 2)])
def test_comb_matches_oracle(importance, period):
    """Population control: the comb after every period-th step picks the same
    walkers (bit-equal selection, then the gathered state within 1e-9) and
    gives every walker the mean weight."""
    spec, W, P, dtau = SYSTEMS["c0"]
    kw = dict(n_burn=3, importance=importance, pop_period=period)
    s, ham, ocfg, ctx = _setup(spec, W, P, 0.05, seed=41 + period, **kw)
    ost = oa.init(ham, ocfg)
    ost.weight = np.random.default_rng(period).exponential(size=W)
    ost.weight[[2, 7, 8]] = 0.0
    ctx.load_state_arrays(_as_dict(ost))
    n_steps, combs, replaced = 4, 0, 0
    for k in range(n_steps):
        ctx.step(1)
        ost, d = oa.step(ham, ocfg, ost)
        if d["comb_src"] is not None:
            combs += 1
            replaced += int(np.sum(d["comb_src"] != np.arange(W)))
            if combs == 1:
                assert len(set(d["comb_src"].tolist())) < W      # the first comb duplicates walkers
            assert np.all(ost.weight == ost.weight[0]) and ost.weight[0] > 0
        _compare_state(ctx.state_arrays(), ost)
    assert combs == n_steps // period
    st = ctx.stats()
    assert st["combs"] == combs and st["comb_replaced"] == replaced >= 3
    ctx.close()


@pytest.mark.parametrize("name", ["c0", "ragged", "one_spin", "one_electron_each", "single_path", "medium",
                                  "two_blocks_walker_side"])
def test_half_rotation_cache_matches_oracle(name):
    """FP64 with the cached half-rotated matrices X_g Phi_p: the measurement after a
    state load (every pair formed) and three steps whose accepted moves leave pairs
    to refresh match the oracle; the refresh count is every pair once plus the
    pairs whose path moved."""
    spec, W, P, dtau = SYSTEMS[name]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=_seed(700, name), n_burn=2, n_sweeps=2, rcache=True)
    assert lib.contract_kernel(ctx.cfg) == "contract_fp64r_kernel"
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    ctx.load_state_arrays(_as_dict(ost))
    _compare_measure(ctx, ham, ost)
    accepted = 0
    for _ in range(3):
        ctx.step(1)
        ost, d = oa.step(ham, ocfg, ost)
        accepted += d["n_accept"]
        _compare_state(ctx.state_arrays(), ost)
    _compare_measure(ctx, ham, ost)
    formed = ctx.stats()["rcache_formed"]
    assert W * P < formed <= W * P + accepted
    ctx.close()


def test_half_rotation_cache_follows_the_comb():
    """The comb copies the cached matrices and their refresh flags with the walkers."""
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, ctx = _setup(spec, W, P, 0.05, seed=43, n_burn=3, pop_period=1, rcache=True)
    ost = oa.init(ham, ocfg)
    ost.weight = np.random.default_rng(5).exponential(size=W)
    ost.weight[[1, 6]] = 0.0
    ctx.load_state_arrays(_as_dict(ost))
    for _ in range(3):
        ctx.step(1)
        ost, d = oa.step(ham, ocfg, ost)
        _compare_state(ctx.state_arrays(), ost)
        _compare_measure(ctx, ham, ost)
    assert ctx.stats()["comb_replaced"] > 0
    ctx.close()


def test_half_rotation_cache_checkpoint_resume_is_bitwise():
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, a = _setup(spec, W, P, dtau, seed=91, n_burn=2, rcache=True)
    _, _, _, b = _setup(spec, W, P, dtau, seed=91, n_burn=2, rcache=True)
    a.step(2)
    blob = a.save_state()
    a.step(2)
    b.load_state(blob)
    b.step(2)
    assert a.save_state() == b.save_state()
    assert np.array_equal(a.history(2), b.history(2))
    a.close()
    b.close()


@pytest.mark.parametrize("name,proposal", [("c0", "prior"), ("ragged", "pcn")])
def test_measurement_paths_match_oracle(name, proposal):
    """Extra measurement-only paths: the estimate, every walker's E'_w and R_w
    against the oracle; the propagation's state is left as it was (the next
    step still matches); one round without sweeps is the plain estimate."""
    spec, W, P, dtau = SYSTEMS[name]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=801, n_burn=2, proposal=proposal, pcn_beta=0.5)
    ost = oa.init(ham, ocfg)
    ost, _ = oa.step(ham, ocfg, ost)
    ost.weight[1] = 0.0
    ctx.load_state_arrays(_as_dict(ost))
    g = ctx.energy_paths(3, 2)
    o = oa.measure_paths(ham, ocfg, ost, 3, 2)
    live = o["alive"]
    assert live.sum() >= W // 2 and not live[1]
    assert abs(g["e_mix"] - o["e_mix"]) < E_TOL
    assert np.max(np.abs(g["e_walker"][live] - o["e_walker"][live])) < E_TOL
    assert np.max(np.abs(g["ratio"][live] - o["R"][live])) < 1e-9
    assert np.all(g["ratio"][~live] == 0)
    assert np.max(np.abs(o["R"][live] - 1.0)) > 1e-6        # the measurement paths moved
    _compare_state(ctx.state_arrays(), ost)
    ctx.step(1)
    ost2, _ = oa.step(ham, ocfg, ost)
    _compare_state(ctx.state_arrays(), ost2)
    g1 = ctx.energy_paths(1, 0)
    assert abs(g1["e_mix"] - ctx.energy()["e_mix"]) < 1e-11
    ctx.close()


def test_measurement_paths_are_refused_with_the_cache():
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=5, n_burn=1, rcache=True)
    with pytest.raises(lib.AfqmcError):
        ctx.energy_paths(1, 0)
    ctx.close()


def test_dead_walkers_stay_frozen():
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=3, n_burn=1)
    ost = oa.init(ham, ocfg)
    ost.weight[[1, 5]] = 0.0
    ctx.load_state_arrays(_as_dict(ost))
    ctx.step(2)
    for _ in range(2):
        ost, _ = oa.step(ham, ocfg, ost)
    g = ctx.state_arrays()
    _compare_state(g, ost)
    assert g["weight"][1] == 0 and g["weight"][5] == 0
    ctx.close()


# ---------------------------------------------------------------- init and trajectories

def test_init_matches_oracle():
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=ai.philox_run_seed(0), n_burn=10)
    ost = oa.init(ham, ocfg)
    _compare_state(ctx.state_arrays(), ost)
    ctx.close()


def test_trajectory_c0_matches_oracle():
    """The small FP64 workload (8 orbitals, 4+4 electrons, 32 Cholesky vectors,
    8 hidden variables, tau = 0.01), 64 walkers x 16 paths, 12 steps from init."""
    spec, run = ai.CONFIGS["small_n8"]
    s, ham, ocfg, ctx = _setup(spec, run.n_walkers, run.n_paths, run.dtau, seed=ai.philox_run_seed(0), n_burn=20,
                               e_shift=11.5)
    ost = oa.init(ham, ocfg)
    n = 12
    ctx.step(n)
    mixed = []
    for _ in range(n):
        ost, d = oa.step(ham, ocfg, ost)
        mixed.append(d["mixed"][0] / d["mixed"][1])
    hist = ctx.history(n)
    assert np.max(np.abs(hist[:, 0] / hist[:, 1] - np.array(mixed))) < E_TOL
    _compare_state(ctx.state_arrays(), ost, rel=1e-8)
    ctx.close()


def test_full_size_medium_workload_sampled_walkers():
    """The medium FP64 workload at full size (50 orbitals, 10+10 electrons,
    250 Cholesky vectors, 50 hidden variables, 512 walkers x 32 paths, as
    timed by the benchmark): sampled walkers recomputed one by one by the
    oracle, for the measurement and for one whole step."""
    spec, run = ai.CONFIGS["medium_n50"]
    s = ai.make_system(spec)
    W, P = run.n_walkers, run.n_paths
    seed = ai.philox_run_seed(1)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=2)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ctx.step(1)
    before = ctx.state_arrays()
    e = ctx.energy(walkers=True)
    fb = ctx.observables()["force_bias"]
    ctx.step(1)
    after = ctx.state_arrays()
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, run.dtau)
    ocfg = oa.OracleConfig(dtau=run.dtau, n_walkers=3, n_paths=P, seed=seed)
    sample = np.array([0, 257, W - 1])
    ost = oa.State(before["step"], before["phi_up"][sample], before["phi_dn"][sample], before["weight"][sample],
                   before["x"][sample], before["Phi"][sample], walker_index=sample)
    m = oa.measure(ham, ost)
    assert np.max(np.abs(e["e_walker"][sample] - m["e_bar"])) < E_TOL
    assert np.max(np.abs(fb[sample] - m["v_bar"])) < 1e-9
    ost2, _ = oa.step(ham, ocfg, ost)
    assert np.allclose(after["weight"][sample], ost2.weight, rtol=1e-9, atol=0)
    assert np.max(np.abs(after["phi_up"][sample] - ost2.phi_up)) < 1e-9
    assert np.max(np.abs(after["x"][sample] - ost2.x)) < 1e-9
    ctx.close()


# ---------------------------------------------------------------- checkpoint and bookkeeping

def test_checkpoint_resume_is_bitwise():
    spec, W, P, dtau = SYSTEMS["ragged"]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=8, n_burn=2)
    ctx.step(2)
    saved = ctx.save_state()
    ctx.step(3)
    a = ctx.save_state()
    ctx.load_state(saved)
    ctx.step(3)
    b = ctx.save_state()
    assert a == b
    ctx.close()


def test_stats_count_proposals():
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=9, n_burn=1, n_sweeps=3)
    ctx.step(4)
    st = ctx.stats()
    assert st["steps"] == 4 and st["status"] == 0
    assert st["proposed"] == 4 * 3 * W * P
    assert 0 < st["accepted"] <= st["proposed"]
    assert np.sum(ctx.history(4)[:, 3]) == st["accepted"]
    ctx.close()


def test_bad_state_buffer_is_rejected():
    spec, W, P, dtau = SYSTEMS["c0"]
    s, ham, ocfg, ctx = _setup(spec, W, P, dtau, seed=9, n_burn=0)
    blob = ctx.save_state()
    with pytest.raises(lib.AfqmcError) as ei:
        ctx.load_state(blob[:-8])
    assert ei.value.status == 5
    ctx.close()


def test_fp64_contraction_forms_agree():
    """The per-pair FP64 contraction (R_g = Phi^T L_g first; used by the entry
    point that allocates nothing) and the walker-side one (Y_g = L_g phi_w once
    per block of a walker's pairs, then Phi^T Y A^-1; used by contexts with at
    least 8 paths) on the same walker and path states."""
    spec = ai.SystemSpec(50, 10, 10, 250, 50, True, 1001)
    s = ai.make_system(spec)
    W, P = 3, 16
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, 0.005, 77, n_burn=3)
    assert lib.contract_kernel(cfg) == "contract_fp64z_kernel"
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U)
    ctx.step(2)
    ctx.energy()
    ref = ctx.observables()
    st = ctx.state_arrays()
    dev = torch.device("cuda")
    pairs = W * P
    h = torch.from_numpy(s.h).to(dev)
    L = torch.from_numpy(s.L).to(dev)
    Phi = torch.from_numpy(np.ascontiguousarray(st["Phi"])).to(dev)
    phi = np.ascontiguousarray(np.concatenate([st["phi_up"], st["phi_dn"]], axis=2))
    phi_d = torch.from_numpy(phi.view(np.float64)).to(dev)
    logov = torch.empty(2 * pairs, dtype=torch.float64, device=dev)
    e_local = torch.empty(2 * pairs, dtype=torch.float64, device=dev)
    fb = torch.empty(2 * pairs * spec.n_chol, dtype=torch.float64, device=dev)
    lib.local_energy_noalloc(spec.N, spec.n_up, spec.n_dn, spec.n_chol, pairs, P, h, L, Phi, phi_d, logov, e_local, fb)
    torch.cuda.synchronize()
    el = e_local.cpu().numpy().view(np.complex128).reshape(W, P)
    assert np.max(np.abs(el - ref["e_local"])) < 1e-9
    ctx.close()
