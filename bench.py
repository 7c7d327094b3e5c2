#!/usr/bin/env python
"""Benchmark of the sampled-trial phaseless AFQMC step on GB300.

Metric: walker-sample steps per second including the local energy, i.e.
(walkers x paths x steps) / device time, with every step running the whole
leapfrog (overlaps, contraction for force bias and local energy, path
averages and mixed estimator, fields, propagation, ratios, Metropolis path
updates, hand-off constraint, re-orthonormalisation).

Headline workload: the mixed-precision synthetic molecule -- N = 120 orbitals,
24 + 24 electrons, 600 Cholesky vectors, 120 hidden variables, 1024 walkers x
64 paths, tau = 0.005, one Metropolis sweep per step (afqmc_inputs seed 1002) --
on the mixed-precision path: the contraction on the tensor cores (walker-side
form, split FP16, FP32 accumulation), the error-controlled double-float
refinement of the pairs whose error would put their walker above 1e-4 Ha, the
trial orbitals and propagation in double-float, overlaps, LU, weights and
energy sums in FP64.  Beside it: the plain FP64 path on the same workload (a
sample of walkers, from the same state: its time and the per-walker and mixed
energy differences), and the other workloads as variants.  With --gpus N
(torchrun) every rank runs its own block of walkers of one population (weak
scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "large_n120"          # the headline: the mixed-precision workload
MEDIUM = "medium_n50"            # the medium FP64 workload of the variants
HEADLINE_PATH = dict(precision="fp16x6", tc_form="walker", refine_tol=1e-4)


def mixed_path(lib, spec, W, P):
    """The headline's mixed path for a system: three-part operands where the
    walker-side form's shared memory holds them, else two-part ones."""
    c = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, 0.005, 1, **HEADLINE_PATH)
    return dict(HEADLINE_PATH, precision="fp16x6" if lib.workspace_bytes(c) > 0 else "fp16x3")
METRIC = "walker-sample steps/s incl. local energy"
UNIT = "walker-sample steps/s"
# FP64 peak of GB300 from unit counts and clock: 152 SMs x 4 FP64 flop/clk
# (2 DFMA) x 2070 MHz.
FP64_PEAK_GFLOPS = 152 * 4 * 2.070
# Double-float multiply-add peak from unit counts and clock: 152 SMs x 128 FP32
# lanes x 2070 MHz instructions, 12 FP32 instructions per double-float
# multiply-add (Dot2 step: a product with its error in 4, the compensated sum in 8),
# 2 flops each.
DF_PEAK_TFLOPS = 152 * 128 * 2.070e9 / 12 * 2 / 1e12
L2_BYTES = 129e6


def workload_desc(spec, run, name=WORKLOAD):
    return (f"{name}: synthetic molecule, N={spec.N} orbitals, {spec.n_up}+{spec.n_dn} electrons, "
            f"{spec.n_chol} Cholesky vectors, K={spec.K} hidden variables, {run.n_walkers} walkers x "
            f"{run.n_paths} paths per GPU, tau={run.dtau}, 1 Metropolis sweep/step")


def contract_flops_per_pair(spec):
    """Algorithmic FLOPs of the fused contraction for one (walker, path) pair in
    the per-pair association order: R = Phi^T X (X = h and every L_g): 2 n_up N^2
    each; M_s = R Theta_s (real x complex): 4 N n_s^2 each; exchange traces
    Tr(M M): 8 n_s^2 per g."""
    N, nu, nd, G = spec.N, spec.n_up, spec.n_dn, spec.n_chol
    return (G + 1) * 2 * nu * N * N + (G + 1) * 4 * N * (nu * nu + nd * nd) + G * 8 * (nu * nu + nd * nd)


def contract_flops_walker_side(spec, P):
    """Algorithmic FLOPs per pair of the walker-side FP64 form: Y_g = X_g phi_w
    (real x complex, 4 N^2 (n_up + n_dn) per matrix, once per walker, shared by
    its P pairs), Z = Phi_s^T Y_s (4 N n_s^2), M = Z A_s^-1 (complex, 8 n_s^3),
    exchange traces (8 n_s^2 per g)."""
    N, nu, nd, G = spec.N, spec.n_up, spec.n_dn, spec.n_chol
    s2, s3 = nu * nu + nd * nd, nu ** 3 + nd ** 3
    return (G + 1) * (4 * N * s2 + 8 * s3) + G * 8 * s2 + (G + 1) * 4 * N * N * (nu + nd) / P


def contract_flops_cached(spec):
    """Algorithmic FLOPs per pair of the FP64 form with the half-rotated matrices
    R_g = Phi^T X_g cached per pair: M_s = R Theta_s (4 N n_s^2 per matrix) and the
    exchange traces (8 n_s^2 per g); the refresh of a pair whose path moved costs
    contract_flops_refresh more."""
    N, nu, nd, G = spec.N, spec.n_up, spec.n_dn, spec.n_chol
    s2 = nu * nu + nd * nd
    return (G + 1) * 4 * N * s2 + G * 8 * s2


def contract_flops_refresh(spec):
    """FLOPs of forming one pair's cached matrices X_g Phi_p (2 n_up N^2 each)."""
    return (spec.n_chol + 1) * 2 * spec.n_up * spec.N * spec.N


def step_working_set_bytes(spec, run, rcache=False):
    """Bytes a step touches per GPU: per-pair state and buffers, plus the cached
    half-rotated matrices (read in full by every contraction) when they are on."""
    N, nt, nu, G, K = spec.N, spec.n_up + spec.n_dn, spec.n_up, spec.n_chol, spec.K
    pairs = run.n_walkers * run.n_paths
    cached = pairs * (G + 1) * N * nu * 8 if rcache else 0
    return pairs * (N * nt * 16 + N * nu * 8 * 3 + N * N * 8 + G * 16 + K * 16) + cached


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ oracle (CPU) legs
ORACLE_PATHS = 4   # paths per walker of the CPU sample (the oracle's pair cost does not depend on P)


def _oracle_walker_job(args):
    """Run in a spawned process: the oracle, as it stands, on one walker of the
    headline workload with ORACLE_PATHS paths: initialised by the oracle (two
    burn-in sweeps), then ``n_warm`` + ``n_timed`` steps, the last ``n_timed``
    timed.  Returns the list of timed step seconds."""
    widx, n_warm, n_timed = args
    import numpy as np
    import afqmc_inputs as ai
    from oracle import afqmc as oa
    spec, run = ai.CONFIGS[WORKLOAD]
    s = ai.make_system(spec)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, spec.n_up, spec.n_dn, run.dtau)
    cfg = oa.OracleConfig(dtau=run.dtau, n_walkers=1, n_paths=ORACLE_PATHS, seed=ai.philox_run_seed(2), n_burn=2)
    st = oa.init(ham, cfg, walker_index=np.array([widx]))
    times = []
    for k in range(n_warm + n_timed):
        t0 = time.perf_counter()
        st, _ = oa.step(ham, cfg, st)
        if k >= n_warm:
            times.append(time.perf_counter() - t0)
    return times


def oracle_pool_steps(n_walkers, n_warm, n_timed):
    """Run the oracle on ``n_walkers`` walkers of the workload, one walker per
    spawned process, all at once; returns (per-step wall seconds, processes)."""
    import multiprocessing as mp
    procs = min(n_walkers, os.cpu_count() or 1)
    # one BLAS thread per process (set before the spawned children import numpy)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    jobs = [(i, n_warm, n_timed) for i in range(n_walkers)]
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_walker_job, jobs)
    # walkers run concurrently: a step's wall time is the slowest walker's, per round of `procs` walkers
    rounds = math.ceil(n_walkers / procs)
    per_step = [max(r[k] for r in res) * rounds for k in range(n_timed)]
    return per_step, procs


def _sample_desc(n, procs, run):
    return (f"{n} walkers x {ORACLE_PATHS} paths (of the {run.n_walkers} x {run.n_paths} of {WORKLOAD}), "
            f"oracle-initialised (2 burn-in sweeps), one walker per process, {procs} processes on "
            f"{os.cpu_count()} host cores; the oracle's cost per walker-path pair does not depend on the "
            f"paths per walker")


def cpu_baseline_leg(run):
    """The oracle, as it stands, on a bounded sample of the workload: one step
    of every host core's walker."""
    n = os.cpu_count() or 1
    per_step, procs = oracle_pool_steps(n, 0, 1)
    value = n * ORACLE_PATHS / per_step[0]
    return {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": _sample_desc(n, procs, run)}


def reference_arm(args):
    import afqmc_inputs as ai
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    spec, run = ai.CONFIGS[WORKLOAD]
    n = os.cpu_count() or 1
    per_step, procs = oracle_pool_steps(n, args.warmup, args.steps)
    total = sum(per_step)
    value = n * ORACLE_PATHS * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_desc(spec, run)},
            "cpu_baseline": {"kind": "oracle", "cores": procs, "value": value, "unit": UNIT,
                             "sample": "each step: " + _sample_desc(n, procs, run)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ traffic of the dominant kernel
def kernel_digest(kernel_source: str, end_marker: str = "size_t contract_fp64_smem", start_marker: str = None) -> str:
    """sha256 (16 hex digits) of a kernel's device code: the text of its
    source file from the line starting with ``start_marker`` (the file's start
    if None) up to the line starting with ``end_marker`` (the first host
    function), so that edits of launchers or of other kernels keep it."""
    text = open(kernel_source, "rb").read()
    begin = 0
    if start_marker is not None:
        b = text.find(b"\n" + start_marker.encode())
        begin = b + 1 if b >= 0 else 0
    cut = text.find(b"\n" + end_marker.encode(), begin)
    return hashlib.sha256(text[begin:cut + 1] if cut >= 0 else text[begin:]).hexdigest()[:16]


def recorded_traffic(kernel_source: str, summary: str = "contract_fp64_medium_n50.md",
                     end_marker: str = "size_t contract_fp64_smem", start_marker: str = None):
    """DRAM bytes per launch of a contraction kernel from its committed ncu
    summary, or None if the kernel's device code changed since the counters
    were taken."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    digest = kernel_digest(kernel_source, end_marker, start_marker)
    fields = {}
    for line in open(path):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("source_sha256_16") != digest:
        return None
    for key in ("dram_bytes_per_full_launch", "dram_bytes_per_pair"):
        try:
            return float(fields[key])
        except (KeyError, ValueError):
            continue
    return None



TCW_TRAFFIC = ("contract_tcw_large_n120.md", "// ---------------------------------------------------------------- per pair: v_g and E_L",
               "// ---------------------------------------------------------------- GEMM-Z and the traces")


def tcw_traffic(W, P):
    """DRAM bytes of the GEMM-Z kernel per contraction of the headline workload,
    from its committed ncu summary (taken on a smaller population of the same
    system and scaled by pairs, as the summary states), or None if the kernel's
    device code changed since."""
    per_pair = recorded_traffic(os.path.join(ROOT, "paper_2505_18519_gb300", "csrc", "contract_tcw.cu"),
                                TCW_TRAFFIC[0], TCW_TRAFFIC[1], TCW_TRAFFIC[2])
    return None if per_pair is None else per_pair * W * P


_FP64_PEAK = {}


def fp64_peak():
    """Measured FP64 FMA rate of this GPU (TFLOP/s) and where it came from."""
    if "v" not in _FP64_PEAK:
        from paper_2505_18519_gb300 import afqmc as lib
        try:
            _FP64_PEAK["v"] = (lib.fp64_fma_rate(), "measured: FP64 FMA loop (afqmc_fp64_fma_rate)")
        except Exception:
            _FP64_PEAK["v"] = (FP64_PEAK_GFLOPS / 1e3, "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz")
    return _FP64_PEAK["v"]


# ------------------------------------------------------------------ the widened paths
def _timed(step, sync, stream, steps, world, local):
    """Device time in ms of ``step(steps)`` on ``stream`` (max over ranks),
    bracketed by barriers and synchronisation, with clocks sampled."""
    import torch
    import torch.distributed as dist
    from paper_2505_18519_gb300 import afqmc as lib
    from paper_2505_18519_gb300.sharding import max_over_ranks
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        sync()
        l0 = lib.launch_count()
        e0.record(stream)
        step(steps)
        e1.record(stream)
        sync()
        l1 = lib.launch_count()
        if world > 1:
            dist.barrier()
    return max_over_ranks(e0.elapsed_time(e1)), clk.summary(), int(l1 - l0)


FP64_WALKER_SIDE = "// ---------------------------------------------------------------- walker-side form"
FP64_TRAFFIC = {   # kernel -> (committed summary, end of its device code, start of it), for the medium workload
    "contract_fp64_kernel": ("contract_fp64_medium_n50.md", FP64_WALKER_SIDE, None),
    "contract_fp64z_kernel": ("contract_fp64z_medium_n50.md", "size_t contract_fp64_smem", FP64_WALKER_SIDE),
    "contract_fp64r_kernel": ("contract_fp64r_medium_n50.md", "// Running count of refreshed pairs",
                              "// One warp per pair: Theta stays"),
}
FP64_SOURCE = {"contract_fp64r_kernel": "rcache.cu"}   # else contract_fp64.cu
TC_TRAFFIC = {   # kernel -> (committed summary, end of its device code, start of it), for the medium workload
    "contract_tcy_kernel": ("contract_tcy_medium_n50.md", "struct TcyShape",
                            "// ---------------------------------------------------------------- walker-side form"),
}


def hbm_peak():
    """Measured copy bandwidth of this GPU type (GB/s) and where it came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peak = json.load(open(path)).get("hbm_gbs") if os.path.exists(path) else None
    return (peak, "measured copy") if peak else (6800.0, "fallback copy")


def tensor_roofline(spec, W, P, prof, kernel):
    """Algorithmic FLOP rate of the tensor-core contraction against the
    measured sustained BF16 peak (FP16 has the same nominal rate)."""
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops_sustained")
    source = "measured bf16 sustained (fp16 nominal ratio 1)"
    if peak is None:
        peak, source = 1700.0, "fallback sustained bf16 (fp16 nominal ratio 1)"
    # the contraction of one step: for the walker-side form, the Y-image kernel and
    # the pair kernel (plus, for the per-pair form, the refinement's launches)
    steps = max(1, prof["steps"])
    ms = prof["ms"]["contract"] / steps
    flops = contract_flops_per_pair(spec) * W * P
    achieved = flops / (ms / 1e3) / 1e12
    traffic = None
    if kernel in TC_TRAFFIC and (W, P) == (512, 32):
        summary, marker, start = TC_TRAFFIC[kernel]
        traffic = recorded_traffic(os.path.join(ROOT, "paper_2505_18519_gb300", "csrc", "contract_tc.cu"), summary,
                                   marker, start)
    return {"bound": "tensor", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "peak_source": source, "traffic": traffic, "flops_per_launch": flops,
            "ms_per_launch": ms, "launches_per_contraction": prof["launches"]["contract"] / steps,
            "note": "one contraction per step (for the walker-side form its two kernels, tcy_y_kernel and "
                    "contract_tcy_kernel; flops, time and DRAM traffic are theirs together); algorithmic FLOPs of "
                    "the real contraction; the split-FP16 scheme issues 4 MMA products per real product and pads N "
                    "and n to MMA tile sizes"}


def tau_int(series):
    """Integrated autocorrelation time of a series, Sokal's self-consistent window (c = 5)."""
    import numpy as np
    x = np.asarray(series, dtype=np.float64)
    x = x - x.mean()
    n = x.size
    var = float(np.dot(x, x)) / n
    if var == 0.0:
        return 1.0
    tau = 1.0
    for t in range(1, n // 2):
        tau += 2.0 * float(np.dot(x[:-t], x[t:])) / (n * var)
        if t >= 5 * tau:
            break
    return max(tau, 1.0)


def _emix(hist):
    import numpy as np
    return np.where(hist[:, 1] > 0, hist[:, 0] / np.where(hist[:, 1] > 0, hist[:, 1], 1.0), np.nan)


def run_variants(args, lib, s, spec, run, seed, rank, world, dev, ew64, hist64, local, only=None, state0=None):
    """The mixed-precision contraction, the learned proposal and the batch of
    uneven systems, each timed like the headline on this GPU's walker block."""
    import numpy as np
    import torch
    import afqmc_inputs as ai
    W, P = run.n_walkers, run.n_paths
    out = {}
    steps, warmup = args.steps, args.warmup

    if only in (None, "fp64", "mixed"):
        # the medium workload on the plain FP64 path with the cached half-rotated matrices
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=20,
                              walker_offset=rank * W, e_shift=28.5, rcache=True)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
        state0 = ctx.save_state()
        ew64 = ctx.energy(walkers=True)["e_walker"]
        for _ in range(warmup):
            ctx.step(1)
        ctx.profile(True)
        ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, steps, world, local)
        prof = ctx.profile_read()
        hist64 = ctx.history(warmup + steps)
        ctx.close()
        cms = prof["ms"]["contract"] / max(1, prof["steps"])
        flops_pp = contract_flops_per_pair(spec) * W * P
        peak, psrc = fp64_peak()
        out["fp64_medium"] = {
            "precision": "fp64", "what": workload_desc(spec, run, MEDIUM) + "; FP64 with the cached half-rotated "
            "matrices (rcache = 1), 20 burn-in sweeps",
            "value": W * P * world * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "gpu_launches": launches, "clocks": clocks,
            "roofline": {"bound": "alu", "kernel": lib.contract_kernel(cfg), "ms_per_launch": cms,
                         "achieved_per_pair_count": flops_pp / (cms / 1e3) / 1e12, "peak": peak, "peak_source": psrc,
                         "unit": "TFLOP/s", "frac_per_pair_count": flops_pp / (cms / 1e3) / 1e12 / peak,
                         "note": "per-pair algorithmic count; the cached form executes fewer FP64 operations "
                                 "(M = R Theta plus the refreshed pairs)"},
            "phases_ms_per_step": {k: round(v / max(1, prof["steps"]), 3) for k, v in prof["ms"].items()}}

    if only in (None, "mixed"):
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=20,
                              walker_offset=rank * W, e_shift=28.5, precision="fp16x3")
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
        if state0 is not None:
            ctx.load_state(state0)   # the FP64 run's initial state: the differences below are the contraction's
        ew = ctx.energy(walkers=True)["e_walker"]
        for _ in range(warmup):
            ctx.step(1)
        ctx.profile(True)
        ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, steps, world, local)
        prof = ctx.profile_read()
        hist = ctx.history(warmup + steps)
        ctx.close()
        d = {"precision": "fp16x3", "what": "same workload, Philox streams and initial state as the headline; the "
             "contraction (force bias + local energy) on the tensor cores in split FP16 with FP32 accumulation, the "
             "trial orbitals, proposal and field matrices and the propagation in double-float (FP32 pairs), "
             "everything else FP64", "value": W * P * world * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
             "gpu_launches": launches, "clocks": clocks,
             "roofline": tensor_roofline(spec, W, P, prof, lib.contract_kernel(cfg)),
             "phases_ms_per_step": {k: round(v / max(1, prof["steps"]), 3) for k, v in prof["ms"].items()}}
        if ew64 is not None:
            dw = np.abs(ew.real - ew64.real)
            d["dE_walker_initial_ha"] = {"median": float(np.median(dw)), "max": float(dw.max()),
                                         "frac_above_1e-4": float(np.mean(dw > 1e-4))}
        if hist64 is not None and len(hist64) == len(hist):
            de = np.abs(_emix(hist) - _emix(hist64))
            d["dE_mix_ha"] = {"max_over_steps": float(np.nanmax(de)), "last": float(de[-1]),
                              "steps_compared": int(len(de))}
        out["mixed_fp16x3"] = d

    if only in (None, "learned"):
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=20,
                              walker_offset=rank * W, e_shift=28.5, precision="fp16x3", proposal="mlp",
                              mlp_train=True)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
        n_train = max(warmup, 20)
        for _ in range(n_train):
            ctx.step(1)
        ctx.profile(True)
        ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, steps, world, local)
        prof = ctx.profile_read()
        hist = ctx.history(steps)
        theta = ctx.mlp_params()
        ctx.close()
        acc = float(hist[:, 3].sum() / (steps * W * P))
        # mixing: the trained network frozen against the prior proposal, from one common
        # state, on a block of walkers: acceptance and integrated autocorrelation time of
        # every path's first hidden variable (Sokal window), averaged over paths
        Wt, T = min(64, W), 40
        mixing, start = {}, None
        for prop in ("prior", "mlp", "pcn"):
            try:
                c = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, Wt, P, run.dtau, seed,
                                    n_burn=20, walker_offset=rank * Wt, e_shift=28.5, precision="fp16x3",
                                    proposal=prop, mlp_train=False, pcn_beta=0.5)
                cx = lib.Context(c, s.h, s.L, s.Phi0, s.U, device=dev)
                if prop == "mlp":
                    cx.mlp_params(theta)
                if start is None:
                    start = cx.save_state()
                else:
                    cx.load_state(start)
                xs, es, acc_t = [], [], []
                for _ in range(T):
                    cx.step(1)
                    xs.append(cx.state_arrays()["x"][:, :, 0].ravel().copy())
                    acc_t.append(cx.history(1)[0][3] / (Wt * P))
                    es.append(cx.energy(walkers=True)["e_walker"].real.copy())
                cx.close()
                X, E = np.array(xs), np.array(es)
                cols = [j for j in range(E.shape[1]) if np.all(np.isfinite(E[:, j]))]
                mixing[prop] = {"acceptance": float(np.mean(acc_t)),
                                "tau_int_x": float(np.mean([tau_int(X[:, j]) for j in range(X.shape[1])])),
                                "tau_int_e_walker": float(np.mean([tau_int(E[:, j]) for j in cols])) if cols else None}
            except Exception as exc:   # a failed comparison must not cost the variant
                mixing[prop] = {"error": f"{type(exc).__name__}: {exc}"}
        d = {"precision": "fp16x3", "proposal": "mlp (K->256->256->2K, BF16 GEMMs, trained online every step)",
             "what": f"same workload; {n_train} untimed training steps, then the timed steps (training continues)",
             "value": W * P * world * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
             "gpu_launches": launches, "clocks": clocks, "acceptance": acc,
             "roofline": tensor_roofline(spec, W, P, prof, lib.contract_kernel(cfg)),
             "phases_ms_per_step": {k: round(v / max(1, prof["steps"]), 3) for k, v in prof["ms"].items()}}
        if hist64 is not None and len(hist64):
            d["acceptance_prior_proposal"] = float(hist64[-steps:, 3].sum() / (min(steps, len(hist64)) * W * P))
        d["mixing"] = dict(mixing, what=f"{Wt} walkers x {P} paths from one common state, {T} steps each, the "
                                        "trained network frozen (mlp_mix 0.1), the prior proposal and pCN (beta 0.5); "
                                        "tau_int of each path's x_1 and of each walker's Re E_w, in steps, averaged "
                                        "over paths and walkers")
        out["learned_proposal"] = d

    if only in (None, "batched"):
        specs = ai.batched_system_specs(16)
        Wb, Pb = 256, 16
        ctxs = []
        for i, sp in enumerate(specs):
            sy = ai.make_system(sp)
            c = lib.make_config(sp.N, sp.n_up, sp.n_dn, sp.n_chol, sp.K, Wb, Pb, 0.005, ai.philox_run_seed(10 + i),
                                n_burn=20, walker_offset=rank * Wb, **mixed_path(lib, sp, Wb, Pb))
            ctx = lib.Context(c, sy.h, sy.L, sy.Phi0, sy.U, device=dev, stream=torch.cuda.Stream(dev))
            ctx.autotune()
            ctxs.append(ctx)
        b = lib.Batch(ctxs, stream=torch.cuda.Stream(dev))
        shared = b.shared_contractions
        b.step(warmup)
        b.sync()
        ms, clocks, launches = _timed(b.step, b.sync, b.stream, steps, world, local)
        stats = [c.stats() for c in ctxs]
        refined = sum(st["refined_pairs"] for st in stats) / (warmup + steps)
        b.close()
        for c in ctxs:
            c.close()
        units = len(specs) * Wb * Pb * world
        out["batched_uneven"] = {
            "precision": ",".join(sorted({mixed_path(lib, sp, Wb, Pb)["precision"] for sp in specs})), "what": f"{len(specs)} synthetic molecules, N ~ U[40,200] (N = "
            f"{','.join(str(sp.N) for sp in specs)}), n = N/5 per spin, n_chol = 5N, K = N, {Wb} walkers x {Pb} "
            "paths each, autotuned launch shapes, one CUDA-graph launch per step for the whole batch",
            "value": units * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "gpu_launches": launches, "clocks": clocks,
            "live_walkers_frac": sum(st["live_walkers"] for st in stats) / (len(specs) * Wb),
            "refined_pairs_per_step": refined, "refined_frac": refined / (len(specs) * Wb * Pb),
            "refine_tol_ha": 1e-4,
            "tensor_core_forms": sorted({lib.contract_kernel(c.cfg) for c in ctxs}),
            "shared_contractions": shared,
            "shared_note": "systems whose GEMM-Z runs in the batch's one persistent launch (both spins' Y images "
                           "must fit one chunk of walkers: the smaller systems)",
            "device_status_words": [int(st["status"]) for st in stats],
            "status_bits": "1 singular overlap, 2 non-finite value (the walker is removed), 4 tensor-core wait timed out"}

    if only in (None, "popctl"):
        # the local-energy importance function and a comb after every step, on the
        # mixed-precision step of the same workload
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=20,
                              walker_offset=rank * W, e_shift=28.5, precision="fp16x3", importance="local_energy",
                              pop_period=1)
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
        for _ in range(warmup):
            ctx.step(1)
        ctx.profile(True)
        ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, steps, world, local)
        prof = ctx.profile_read()
        stats = ctx.stats()
        hist = ctx.history(steps)
        ctx.close()
        comb_ms = prof["ms"]["comb"] / max(1, prof["steps"])
        # bytes a comb must move: the state (phi, x, Phi(x)) of every replaced walker read
        # from its source and written to its slot, plus the weights
        row = spec.N * (spec.n_up + spec.n_dn) * 16 + P * spec.K * 8 + P * spec.N * spec.n_up * 8
        replaced = stats["comb_replaced"] / max(1, stats["combs"])
        moved = 2 * replaced * row + 2 * W * 8
        gbs = moved / (comb_ms / 1e3) / 1e9
        hbm, hbm_source = hbm_peak()
        out["population_control"] = {
            "precision": "fp16x3", "importance": "local_energy: |I| = exp(-tau (Re E_w - E_T))",
            "what": "same workload and mixed-precision step; a comb resamples the walkers (phi, paths x and Phi(x)) "
                    "after every step",
            "value": W * P * world * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "gpu_launches": launches, "clocks": clocks, "combs": int(stats["combs"]),
            "walkers_replaced_per_comb": replaced,
            "live_walkers_frac": stats["live_walkers"] / W,
            "e_mix_last_step": float(hist[-1, 0] / hist[-1, 1]),
            "comb_ms_per_step": comb_ms,
            "roofline": {"bound": "hbm", "kernel": "comb_select_kernel + comb_gather_kernel",
                         "achieved": gbs, "peak": hbm, "peak_source": hbm_source, "unit": "GB/s",
                         "frac": gbs / hbm, "traffic": None, "algorithmic_bytes": moved,
                         "note": "walkers with a copy keep their slot, so only the replaced walkers' rows move; "
                                 "the selection (running sum of the weights, block scans) is latency-bound"},
            "phases_ms_per_step": {k: round(v / max(1, prof["steps"]), 3) for k, v in prof["ms"].items()}}

    if only in (None, "measpaths"):
        # extra measurement-only paths on the mixed-precision step of the same workload:
        # P' = 4 P paths from one sweep per round, against the plain estimate
        cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=20,
                              walker_offset=rank * W, e_shift=28.5, precision="fp16x3")
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
        for _ in range(warmup):
            ctx.step(1)
        plain = ctx.energy()["e_mix"]
        rounds, sweeps = 4, 1
        ctx.energy_paths(rounds, sweeps)   # untimed first call
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(ctx.stream)
        r = ctx.energy_paths(rounds, sweeps)
        e1.record(ctx.stream)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1)
        ratio = r["ratio"][np.abs(r["ratio"]) > 0]
        ctx.close()
        out["measurement_paths"] = {
            "precision": "fp16x3", "what": f"afqmc_energy_paths after {warmup} steps: {rounds} rounds x {sweeps} "
            f"measurement-only sweep(s), P' = {rounds * P} paths per walker, against afqmc_energy's {P}",
            "ms_per_call": ms, "ms_per_round": ms / rounds, "e_mix_plain": plain, "e_mix_paths": r["e_mix"],
            "ratio_abs_median": float(np.median(np.abs(ratio))) if len(ratio) else None,
            "ratio_abs_range": [float(np.min(np.abs(ratio))), float(np.max(np.abs(ratio)))] if len(ratio) else None}

    if only in (None, "pscaling"):
        # the cost of a step per walker-path pair against the paths per walker, at the
        # medium workload's 16384 pairs (W = 16384 / P), FP64 with the cached half-rotation:
        # the paper's cost model is linear in P at fixed walkers, i.e. flat per pair
        try:
            rows = []
            for Pn in (4, 8, 16, 32, 64):
                Wn = (W * P) // Pn
                c = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, Wn, Pn, run.dtau, seed,
                                    n_burn=20, walker_offset=rank * Wn, e_shift=28.5, rcache=True)
                cx = lib.Context(c, s.h, s.L, s.Phi0, s.U, device=dev)
                cx.step(1)
                ms, clocks, launches = _timed(cx.step, lambda: torch.cuda.synchronize(dev), cx.stream, 2, world,
                                              local)
                cx.close()
                del cx
                torch.cuda.empty_cache()
                rows.append({"paths": Pn, "walkers": Wn, "ms_per_step": ms / 2,
                             "value": Wn * Pn * world * 2 / (ms / 1e3), "sm_mhz": clocks.get("sm_mhz")})
            out["paths_scaling"] = {
                "precision": "fp64", "unit": UNIT, "rows": rows,
                "what": "medium workload system, W x P = 16384 pairs per GPU, rcache on, 1 warm-up and 2 timed "
                        "steps per P; a flat value means a cost per step linear in P at fixed walkers"}
        except Exception as exc:   # the measurement is optional; the line must still print
            out["paths_scaling"] = {"error": f"{type(exc).__name__}: {exc}"}

    if only in (None, "largest"):
        # the largest system (N = 200, 40 + 40 electrons, 1000 Cholesky vectors) in FP64 on a
        # bounded sample: 19 walkers x 16 paths = 304 pairs, two full waves of the per-pair
        # kernel (one block per SM), 1 warm-up and 2 timed steps
        spec4, run4 = ai.CONFIGS["largest_n200"]
        sy = ai.make_system(spec4)
        W4, P4, st4 = 19, run4.n_paths, 2
        c = lib.make_config(spec4.N, spec4.n_up, spec4.n_dn, spec4.n_chol, spec4.K, W4, P4, run4.dtau,
                            ai.philox_run_seed(4), n_burn=2, walker_offset=rank * W4)
        ctx = lib.Context(c, sy.h, sy.L, sy.Phi0, sy.U, device=dev)
        ctx.step(1)
        ctx.profile(True)
        ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, st4, world, local)
        prof = ctx.profile_read()
        kernel = lib.contract_kernel(c)
        ctx.close()
        cms = prof["ms"]["contract"] / max(1, prof["launches"]["contract"])
        flops = contract_flops_per_pair(spec4) * W4 * P4
        achieved = flops / (cms / 1e3) / 1e12
        out["largest_fp64_sample"] = {
            "precision": "fp64", "what": f"system of the largest workload (N = {spec4.N}, {spec4.n_up} + {spec4.n_dn} "
            f"electrons, n_chol = {spec4.n_chol}, K = {spec4.K}), {W4} walkers x {P4} paths (304 pairs = 2 x 152 "
            f"blocks of the per-pair kernel, Theta streamed in row slabs), 1 warm-up and {st4} timed steps",
            "value": W4 * P4 * world * st4 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / st4,
            "full_workload_step_s_extrapolated": ms / st4 / 1e3 * (run4.n_walkers * run4.n_paths) / (W4 * P4),
            "gpu_launches": launches, "clocks": clocks,
            "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": fp64_peak()[0],
                         "peak_source": fp64_peak()[1], "unit": "TFLOP/s", "frac": achieved / fp64_peak()[0],
                         "traffic": None, "flops_per_launch": flops, "ms_per_launch": cms},
            "phases_ms_per_step": {k: round(v / max(1, prof["steps"]), 3) for k, v in prof["ms"].items()}}

    if only in (None, "largest_mixed"):
        # the learned-proposal workload's system (N = 200, 40 + 40 electrons, 1000 Cholesky vectors,
        # K = 200, 16 paths) on a quarter of its 2048 walkers: the mixed-precision step with the general
        # walker-side tensor-core form and its refinement, and the learned proposal trained online
        try:
            spec4, run4 = ai.CONFIGS["largest_n200"]
            sy = ai.make_system(spec4)
            W4, P4 = 512, run4.n_paths
            c = lib.make_config(spec4.N, spec4.n_up, spec4.n_dn, spec4.n_chol, spec4.K, W4, P4, run4.dtau,
                                ai.philox_run_seed(4), n_burn=40, walker_offset=rank * W4, proposal="mlp",
                                mlp_train=True, **mixed_path(lib, spec4, W4, P4))
            ctx = lib.Context(c, sy.h, sy.L, sy.Phi0, sy.U, device=dev)
            ctx.step(2)
            ctx.profile(True)
            r0 = ctx.stats()["refined_pairs"]
            ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, 2, world, local)
            prof = ctx.profile_read()
            st4 = ctx.stats()
            hist = ctx.history(2)
            state4 = ctx.save_state()
            ctx.close()
            del ctx
            torch.cuda.empty_cache()
            ph = {k: round(v / max(1, prof["steps"]), 3) for k, v in prof["ms"].items()}
            try:   # the mixed and the FP64 paths from the saved state, on 16 of the walkers (256 pairs)
                Ws = 16
                st = lib.unpack_state(state4)
                sub = dict(step=st["step"], phi_up=st["phi_up"][:Ws], phi_dn=st["phi_dn"][:Ws], weight=st["weight"][:Ws],
                           x=st["x"][:Ws], Phi=st["Phi"][:Ws])
                cm = lib.make_config(spec4.N, spec4.n_up, spec4.n_dn, spec4.n_chol, spec4.K, Ws, P4, run4.dtau,
                                     ai.philox_run_seed(4), n_burn=0, walker_offset=rank * W4,
                                     **mixed_path(lib, spec4, Ws, P4))
                cmx = lib.Context(cm, sy.h, sy.L, sy.Phi0, sy.U, device=dev)
                cmx.load_state_arrays(sub)
                ew4 = cmx.energy(walkers=True)["e_walker"]
                cmx.close()
                fp4 = fp64_sample_leg(lib, sy, spec4, run4, ai.philox_run_seed(4), rank, W4, dev, state4, ew4, local,
                                      world, n_walk=Ws)
                fp4["speedup"] = fp4["full_workload_ms_per_step_extrapolated"] / (ms / 2)
                fp4["state"] = ("the mixed run's state after its timed steps; both paths measured from it in fresh "
                                "contexts; walkers with zero weight (removed for non-finite values) excluded")
            except Exception as exc:
                fp4 = {"error": f"{type(exc).__name__}: {exc}"}
            flops = contract_flops_per_pair(spec4) * W4 * P4
            out["largest_mixed_learned"] = {
                "precision": mixed_path(lib, spec4, W4, P4)["precision"], "proposal": "mlp (trained online)",
                "kernel": lib.contract_kernel(c),
                "what": workload_desc(spec4, run4, "largest_n200") + f"; {W4} of its {run4.n_walkers} walkers, 40 "
                        "burn-in sweeps, 2 untimed and 2 timed steps",
                "value": W4 * P4 * world * 2 / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / 2,
                "gpu_launches": launches, "clocks": clocks,
                "acceptance": float(hist[:, 3].sum() / (2 * W4 * P4)),
                "refined_frac": (st4["refined_pairs"] - r0) / (2 * W4 * P4),
                "live_walkers": int(st4["live_walkers"]), "device_status": int(st4["status"]),
                "tensor_contraction_tflops": flops / (ph["contract"] / 1e3) / 1e12 if ph["contract"] > 0 else None,
                "vs_fp64_same_state": fp4,
                "phases_ms_per_step": ph}
        except Exception as exc:   # the measurement is optional; the line must still print
            out["largest_mixed_learned"] = {"error": f"{type(exc).__name__}: {exc}"}

    if only == "large_mixed":
        # the mixed-precision workload's system (N = 120, 24 + 24 electrons, 600 Cholesky
        # vectors, 64 paths) on 128 walkers: per-walker error against the FP64 path from
        # one state, with and without the error-controlled FP64 refinement, and step times
        spec2, run2 = ai.CONFIGS["large_n120"]
        sy = ai.make_system(spec2)
        W2, P2, st2 = 128, run2.n_paths, 2
        res, state = {}, None
        for key, prec, tol in (("fp64", "fp64", 1e-4), ("refined", "fp16x3", 1e-4), ("tensor_only", "fp16x3", 0.0),
                               ("refined_fp16x6", "fp16x6", 1e-4), ("tensor_only_fp16x6", "fp16x6", 0.0)):
            c = lib.make_config(spec2.N, spec2.n_up, spec2.n_dn, spec2.n_chol, spec2.K, W2, P2, run2.dtau,
                                ai.philox_run_seed(2), n_burn=20, walker_offset=rank * W2, precision=prec,
                                refine_tol=tol)
            ctx = lib.Context(c, sy.h, sy.L, sy.Phi0, sy.U, device=dev)
            if state is None:
                state = ctx.save_state()
            else:
                ctx.load_state(state)
            ew = ctx.energy(walkers=True)["e_walker"]
            st0 = ctx.stats()
            refined0, terms0 = st0["refined_pairs"], st0["cheb_terms"]
            k = 1 if prec == "fp64" else st2
            ctx.step(1)
            ms, clocks, launches = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, k, world, local)
            refined = ctx.stats()["refined_pairs"]
            res[key] = dict(ew=ew, ms=ms / k, clocks=clocks, refined0=refined0,
                            refined_per_step=(refined - refined0) / (k + 1), kernel=lib.contract_kernel(c))
            ctx.close()
        d = {"what": f"system of the mixed-precision workload (N = {spec2.N}, {spec2.n_up} + {spec2.n_dn} electrons, "
                     f"n_chol = {spec2.n_chol}, K = {spec2.K}), {W2} walkers x {P2} paths after 20 burn-in sweeps; "
                     "per-walker energy differences against the FP64 path at one common state; "
                     f"{st2} timed steps per mixed context (1 for FP64) after 1 untimed step",
             "unit": UNIT, "clocks": res["refined"]["clocks"], "kernel": res["refined"]["kernel"]}
        for key in ("refined", "tensor_only", "refined_fp16x6", "tensor_only_fp16x6", "fp64"):
            r = res[key]
            e = {"value": W2 * P2 * world / (r["ms"] / 1e3), "ms_per_step": r["ms"]}
            if key != "fp64":
                dw = np.abs(r["ew"] - res["fp64"]["ew"])
                e["dE_walker_ha"] = {"max": float(dw.max()), "median": float(np.median(dw)),
                                     "frac_above_1e-4": float(np.mean(dw > 1e-4))}
            e["kernel"] = r["kernel"]
            if key.startswith("refined"):
                e["refined_pairs_at_common_state"] = int(r["refined0"])
                e["refined_pairs_per_step"] = float(r["refined_per_step"])
                e["refine_tol_ha"] = 1e-4
            d[key] = e
        out["large_mixed_sample"] = d
    return out


# ------------------------------------------------------------------ our arm
def tcw_flops_per_pair(spec, P):
    """MMA-free count of the walker-side association per pair: Z = B^T Y
    (complex x complex, 8 N (n_up^2 + n_dn^2) per matrix) plus the pair's share of
    Y_g = X_g phi_w (4 N^2 (n_up + n_dn) per matrix, once per walker) and the
    traces (8 (n_up^2 + n_dn^2) per matrix)."""
    N, nu, nd, G = spec.N, spec.n_up, spec.n_dn, spec.n_chol
    s2 = nu * nu + nd * nd
    return (G + 1) * (8 * N * s2 + 4 * N * N * (nu + nd) / P) + G * 8 * s2


def fp64_sample_leg(lib, s, spec, run, seed, rank, W, dev, state0, ew_mixed, local, world, n_walk=64):
    """The plain FP64 path on the headline workload from the mixed run's
    initial state, on its first ``n_walk`` walkers: the per-walker energy
    difference at that state, the mixed energy difference over the sample, and
    two timed steps (the full-workload step time extrapolated by walkers)."""
    import numpy as np
    import torch
    from paper_2505_18519_gb300 import afqmc as L
    Ws, P = min(n_walk, W), run.n_paths
    st = L.unpack_state(state0)
    sub = dict(step=st["step"], phi_up=st["phi_up"][:Ws], phi_dn=st["phi_dn"][:Ws], weight=st["weight"][:Ws],
               x=st["x"][:Ws], Phi=st["Phi"][:Ws])
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, Ws, P, run.dtau, seed, n_burn=0,
                          walker_offset=rank * W)
    ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
    ctx.load_state_arrays(sub)
    e64 = ctx.energy(walkers=True)
    dw = np.abs(e64["e_walker"] - ew_mixed[:Ws])
    live = sub["weight"] > 0
    wr = sub["weight"][live]
    emix_mixed = float(np.sum(wr * ew_mixed[:Ws][live].real) / np.sum(wr))
    ctx.step(1)
    ms, clocks, _ = _timed(ctx.step, lambda: torch.cuda.synchronize(dev), ctx.stream, 2, world, local)
    ctx.close()
    return {"precision": "fp64", "kernel": lib.contract_kernel(cfg),
            "what": f"the plain FP64 path on the first {Ws} walkers (x{P} paths) of the same workload, from the "
                    "mixed run's initial state; 1 untimed and 2 timed steps",
            "ms_per_step_sample": ms / 2, "value_sample": Ws * P * world * 2 / (ms / 1e3),
            "full_workload_ms_per_step_extrapolated": ms / 2 * W / Ws,
            "dE_walker_ha": {"max": float(dw[live].max()), "median": float(np.median(dw[live])),
                             "frac_above_1e-4": float(np.mean(dw[live] > 1e-4)), "walkers": int(live.sum())},
            "dE_mix_ha": abs(float(e64["e_mix"]) - emix_mixed), "clocks": clocks}


def our_arm(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import afqmc_inputs as ai
    from paper_2505_18519_gb300 import afqmc as lib
    from paper_2505_18519_gb300 import build
    from paper_2505_18519_gb300.sharding import combine_mixed, max_over_ranks

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    lib.load_library()

    # medium workload: the variants that predate the headline's workload
    spec1, run1 = ai.CONFIGS[MEDIUM]
    s1 = ai.make_system(spec1)
    if args.only:
        # one widened path alone (a profiling run): no headline, no baselines
        with torch.cuda.device(dev):
            v = run_variants(args, lib, s1, spec1, run1, ai.philox_run_seed(1), rank, world, dev, None, None, local,
                             only=args.only)
        if rank == 0:
            print(json.dumps({"only": args.only, "variants": v}), flush=True)
        if world > 1:
            dist.destroy_process_group()
        return

    spec, run = ai.CONFIGS[WORKLOAD]
    if args.walkers:
        import dataclasses
        run = dataclasses.replace(run, n_walkers=args.walkers)
    s = ai.make_system(spec)
    W, P = run.n_walkers, run.n_paths
    seed = ai.philox_run_seed(2)
    cfg = lib.make_config(spec.N, spec.n_up, spec.n_dn, spec.n_chol, spec.K, W, P, run.dtau, seed, n_burn=20,
                          walker_offset=rank * W, **HEADLINE_PATH)
    with torch.cuda.device(dev):
        ctx = lib.Context(cfg, s.h, s.L, s.Phi0, s.U, device=dev)
        stream = ctx.stream
        state0 = ctx.save_state()
        ew0 = ctx.energy(walkers=True)["e_walker"]
        for _ in range(args.warmup):
            ctx.step(1)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ctx.profile(True)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            st0 = ctx.stats()
            refined0, terms0 = st0["refined_pairs"], st0["cheb_terms"]
            torch.cuda.synchronize(dev)
            l0 = lib.launch_count()
            e0.record(stream)
            ctx.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            l1 = lib.launch_count()
            stats = ctx.stats()
            if world > 1:
                dist.barrier()
        prof = ctx.profile_read()
        ctx.profile(False)
        ms = e0.elapsed_time(e1)
        ms_max = max_over_ranks(ms)
        clocks = clk.summary()
        hist = ctx.history(args.steps)
        ctx.close()
        del ctx
        torch.cuda.empty_cache()
        # the global mixed estimate of the last timed step: every rank's sums, all-reduced
        emix_global = combine_mixed((hist[-1, 0], hist[-1, 1], hist[-1, 2])) if len(hist) else None

        # end to end through the public API: host (pinned) inputs uploaded by afqmc_init
        # (its 20 burn-in sweeps included) inside the timed region, then the K steps, each
        # followed by a device-to-host read of its energy record
        host = [torch.from_numpy(a).pin_memory() for a in (s.h, s.L, s.Phi0, s.U)]
        h2d = sum(t.numel() * 8 for t in host)
        e2e_s = None
        if not args.no_e2e:
            torch.cuda.synchronize(dev)
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            ctx2 = lib.Context(cfg, *host, device=dev)
            for _ in range(args.steps):
                ctx2.step(1)
                ctx2.history(1)
            t1 = time.perf_counter()
            e2e_s = max_over_ranks(t1 - t0)
            ctx2.close()
            del ctx2
            torch.cuda.empty_cache()
        fp64 = fp64_sample_leg(lib, s, spec, run, seed, rank, W, dev, state0, ew0, local, world)
        variants = None
        if not args.no_variants:
            variants = run_variants(args, lib, s1, spec1, run1, ai.philox_run_seed(1), rank, world, dev, None, None,
                                    local)

    pairs_total = W * P * world
    value = pairs_total * args.steps / (ms_max / 1e3)
    e2e_value = pairs_total * args.steps / e2e_s if e2e_s else None
    steps_p = max(1, prof["steps"])
    phases = {k: round(v / steps_p, 3) for k, v in prof["ms"].items()}
    # the tensor-core contraction (Y images, pair images, GEMM-Z, per-pair finish) against the
    # measured sustained BF16 peak, on the paper's per-pair algorithmic count and on the
    # walker-side association's own count; the refinement (double-float per-pair kernel on the
    # CUDA cores) is reported beside it
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    peak_src = "measured bf16 sustained" if peaks.get("bf16_tflops_sustained") else "fallback sustained bf16"
    c_ms, r_ms = phases["contract"], phases["refine"]
    flops = contract_flops_per_pair(spec) * W * P
    flops_ws = tcw_flops_per_pair(spec, P) * W * P
    achieved = flops / (c_ms / 1e3) / 1e12
    refined_per_step = (stats["refined_pairs"] - refined0) / args.steps
    roof_tc = {"bound": "tensor", "kernel": "contract_tcw_kernel (+ tcw_y_kernel, tcw_a_kernel, tcw_finish_kernel)",
               "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "peak_source": peak_src + " (fp16 nominal ratio 1)",
               "traffic": tcw_traffic(W, P), "flops_per_launch": flops, "ms_per_launch": c_ms,
               "flops_per_launch_walker_side": flops_ws, "frac_walker_side": flops_ws / (c_ms / 1e3) / 1e12 / peak,
               "mma_products_per_real_product": 6 if HEADLINE_PATH["precision"] == "fp16x6" else 4,
               "note": "one contraction per step; flops_per_launch is the per-pair algorithmic count (R = Phi^T X, "
                       "M = R Theta: 2 n N^2 + 4 N (n_up^2 + n_dn^2) + traces per matrix); the walker-side "
                       "association executes flops_per_launch_walker_side in mma_products_per_real_product "
                       "split-FP16 MMA products each; "
                       "traffic is the GEMM-Z kernel's DRAM bytes per contraction"}
    rf_flops = contract_flops_per_pair(spec) * refined_per_step
    roof_rf = {"bound": "alu", "kernel": "contract_fp64_kernel<double-float> (refinement of the listed pairs)",
               "ms_per_launch": r_ms, "pairs_per_launch": refined_per_step,
               "refined_frac": refined_per_step / (W * P),
               "achieved": rf_flops / (r_ms / 1e3) / 1e12 if r_ms > 0 else None, "unit": "TFLOP/s (double-float)",
               "peak": DF_PEAK_TFLOPS,
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2070 MHz, 12 FP32 instructions per double-float "
                              "multiply-add",
               "frac": rf_flops / (r_ms / 1e3) / 1e12 / DF_PEAK_TFLOPS if r_ms > 0 else None, "traffic": None,
               "note": "recomputes in double-float (about 44 bits) the pairs whose estimated tensor-core error would "
                       "put their walker above refine_tol; CUDA-core FP32 pipe"}
    dominant = roof_tc if c_ms >= r_ms else dict(roof_rf, tensor_contraction=roof_tc)
    # the trial orbitals exp(S) Phi0 of the Metropolis proposals (chebyshev_expm_tc_kernel): every
    # Chebyshev term is one product t V (N x N by N x n_up, real); the tensor cores execute it as
    # 20 blocks of 128 x NB x K digit products (19 products and one block of zeros)
    t_ms = phases["trial_orbitals"]
    terms = (stats["cheb_terms"] - terms0) / args.steps
    nb = 16 if spec.n_up <= 16 else 32
    kk = 64 if spec.N <= 64 else 128
    t_alg = terms * 2.0 * spec.N * spec.N * spec.n_up
    t_exe = terms * 20 * 2.0 * 128 * nb * kk
    roof_tt = {"bound": "tensor", "kernel": "chebyshev_expm_tc_kernel (8-bit digit products, exact FP32 accumulation)",
               "ms_per_launch": t_ms, "terms_per_step": terms, "redone_per_step": (stats["cheb_redone"] - st0["cheb_redone"]) / args.steps,
               "achieved_algorithmic": t_alg / (t_ms / 1e3) / 1e12 if t_ms > 0 else None,
               "achieved_executed": t_exe / (t_ms / 1e3) / 1e12 if t_ms > 0 else None,
               "peak": peak, "unit": "TFLOP/s",
               "frac_executed": t_exe / (t_ms / 1e3) / 1e12 / peak if t_ms > 0 else None,
               "note": "algorithmic = 2 N^2 n_up per term; executed = the MMA work of the digit products; the "
                       "recurrence and digit splitting of every term run between the products (one problem per SM)"}

    if world > 1:
        dist.barrier()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = cpu_baseline_leg(run) if (world == 1 and not args.no_cpu_baseline) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": HEADLINE_PATH["precision"] + " contraction (operands split into " +
                 ("three" if HEADLINE_PATH["precision"] == "fp16x6" else "two") + " FP16 parts on the tensor cores, "
                 "FP32 accumulation) + double-float refinement; trial orbitals as exact 8-bit digit products on the "
                 "tensor cores (about 40 bits); overlap matrices and proposal matrices as exact 8-bit digit "
                 "products (about 40 bits), LU and inverses in double-float; f64 weights, energy sums",
        "data": "synthetic",
        "config": {"workload": workload_desc(spec, run), "walkers_total": W * world, "paths": P,
                   "system_seed": spec.seed, "philox_seed": seed, "path": dict(HEADLINE_PATH),
                   "l2": f"working set {step_working_set_bytes(spec, run) / 1e9:.1f} GB per step > 129 MB L2; no flush"},
        "roofline": dominant,
        "roofline_tensor_contraction": roof_tc,
        "roofline_refinement": roof_rf,
        "roofline_trial_orbitals": roof_tt,
        "vs_fp64_same_config": dict(fp64, speedup=(fp64["full_workload_ms_per_step_extrapolated"] /
                                                   (ms_max / args.steps))),
        "cpu_baseline": cpu,
        "e2e": None if e2e_value is None else {
            "value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": 32,
            "includes": "afqmc_init from pinned host arrays (incl. 20 burn-in sweeps) + K steps, each followed by "
                        "a device-to-host read of its energy record"},
        "clocks": clocks, "gpu_launches": int(l1 - l0), "phases_ms_per_step": phases,
        "device_status": int(stats["status"]), "live_walkers": int(stats["live_walkers"]),
        "mixed_energy_last_step": float(hist[-1, 0] / hist[-1, 1]) if len(hist) else None,
        "mixed_energy_last_step_all_ranks": emix_global[0] if emix_global else None,
        "variants": variants,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--walkers", type=int, default=0, help="walkers per GPU (profiling runs on a small case)")
    ap.add_argument("--no-rcache", action="store_true",
                    help="FP64 headline without the cached half-rotated matrices (the walker-side form)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the mixed-precision, learned-proposal and batched measurements")
    ap.add_argument("--only", choices=("fp64", "mixed", "learned", "batched", "popctl", "measpaths", "pscaling",
                                       "largest", "largest_mixed", "large_mixed"),
                    default=None,
                    help="time one variant alone (profiling); skips the FP64 headline's extras")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
