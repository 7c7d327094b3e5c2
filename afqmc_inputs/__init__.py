"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws random numbers and packs arrays. It holds none of the
AFQMC arithmetic (no overlaps, Green's functions, propagators or weights), so
that the CPU oracle and the CUDA path can both consume it without sharing any
of the method.

A synthetic system mimics a molecule in the "Monte Carlo form" of the paper
(Sec. II A, Eq. (1) and (3)): a real symmetric one-body matrix ``h`` (N x N), Gamma
real symmetric Cholesky-like vectors ``L[g]`` (so that V = sum_g L_g (x) L_g is
positive semidefinite by construction), a trial determinant ``Phi0`` (the lowest
``n_up`` eigenvectors of ``h``) and K real symmetric hidden-variable operators
``U[k]`` that define the sampled trial Phi(x) = exp(sum_k x_k U_k) Phi0
(Eq. (20)-(21) with one slice).

Generator recipe:
  * symmetric matrices draw the upper triangle including the diagonal i.i.d.
    and mirror it;
  * h: diagonal ~ U(-2, 0), off-diagonal ~ N(0, 0.1^2);
  * L_g: diagonal ~ N(0, 0.05^2), off-diagonal ~ N(0, 0.05^2);
  * U_k: diagonal ~ N(0, 0.1^2), off-diagonal ~ N(0, 0.1^2);
  * for the medium and large systems every off-diagonal standard deviation is
    multiplied by 1/sqrt(N) (diagonals unchanged);
  * Phi0: lowest n_up eigenvectors of h, each column's sign fixed so that its
    largest-magnitude entry is positive (platform independent).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = ["SystemSpec", "RunSpec", "System", "CONFIGS", "make_system", "make_config",
           "batched_system_specs", "philox_run_seed"]


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    N: int              # orbitals
    n_up: int           # spin-up electrons
    n_dn: int           # spin-down electrons
    n_chol: int         # Cholesky vectors Gamma
    K: int              # hidden variables of the trial
    scale_offdiag: bool  # multiply off-diagonal std by 1/sqrt(N)
    seed: int


@dataclasses.dataclass(frozen=True)
class RunSpec:
    n_walkers: int
    n_paths: int
    dtau: float
    n_steps: int


@dataclasses.dataclass
class System:
    spec: SystemSpec
    h: np.ndarray      # (N, N) float64
    L: np.ndarray      # (n_chol, N, N) float64
    Phi0: np.ndarray   # (N, n_up) float64
    U: np.ndarray      # (K, N, N) float64


def _sym(rng: np.random.Generator, N: int, diag: np.ndarray, off_std: float) -> np.ndarray:
    a = np.zeros((N, N))
    iu = np.triu_indices(N, 1)
    a[iu] = rng.normal(0.0, off_std, size=iu[0].size)
    a = a + a.T
    a[np.diag_indices(N)] = diag
    return a


def make_system(spec: SystemSpec) -> System:
    """Draw h, L, Phi0, U for one synthetic system from ``spec.seed``."""
    N = spec.N
    rng = np.random.default_rng(spec.seed)
    s = 1.0 / math.sqrt(N) if spec.scale_offdiag else 1.0
    h = _sym(rng, N, rng.uniform(-2.0, 0.0, size=N), 0.1 * s)
    L = np.empty((spec.n_chol, N, N))
    for g in range(spec.n_chol):
        L[g] = _sym(rng, N, rng.normal(0.0, 0.05, size=N), 0.05 * s)
    U = np.empty((spec.K, N, N))
    for k in range(spec.K):
        U[k] = _sym(rng, N, rng.normal(0.0, 0.1, size=N), 0.1 * s)
    evals, evecs = np.linalg.eigh(h)
    Phi0 = np.array(evecs[:, : spec.n_up])
    for a in range(spec.n_up):
        j = int(np.argmax(np.abs(Phi0[:, a])))
        if Phi0[j, a] < 0:
            Phi0[:, a] = -Phi0[:, a]
    return System(spec, h, L, np.ascontiguousarray(Phi0), U)


def philox_run_seed(workload_index: int) -> int:
    """64-bit key of the counter-based random streams for a named workload."""
    return 0x5EED0000 + workload_index


# The five workloads (small FP64, medium FP64, mixed precision, batched uneven,
# learned proposal).  Walker counts, path counts, time step and step counts.
CONFIGS = {
    "small_n8": (SystemSpec(8, 4, 4, 32, 8, False, 1000), RunSpec(64, 16, 0.01, 200)),
    "medium_n50": (SystemSpec(50, 10, 10, 250, 50, True, 1001), RunSpec(512, 32, 0.005, 500)),
    "large_n120": (SystemSpec(120, 24, 24, 600, 120, True, 1002), RunSpec(1024, 64, 0.005, 500)),
    "largest_n200": (SystemSpec(200, 40, 40, 1000, 200, True, 1004), RunSpec(2048, 16, 0.005, 500)),
}


def make_config(name: str):
    spec, run = CONFIGS[name]
    return make_system(spec), run


def batched_system_specs(n_systems: int = 16, seed: int = 1003, n_range=(40, 200)):
    """Sizes of the uneven batch: N ~ U[n_range] rounded to a multiple of 5,
    n = N/5 electrons per spin, Gamma = 5N, K = N; system s uses seed 3000+s."""
    rng = np.random.default_rng(seed)
    specs = []
    for s in range(n_systems):
        N = int(5 * round(rng.uniform(*n_range) / 5))
        specs.append(SystemSpec(N, N // 5, N // 5, 5 * N, N, True, 3000 + s))
    return specs
