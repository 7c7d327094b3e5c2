"""Plain FP64 CPU oracle of phaseless AFQMC with a stochastically sampled trial.

ORACLE / TEST INFRASTRUCTURE ONLY.  Nothing in the library imports this
module; only tests, the smoke check and the CPU-baseline leg of the benchmark
may.  It shares no code with the CUDA path: the two meet only through the
seeded inputs of ``afqmc_inputs`` and the published Philox definition, which
each side implements on its own.

It is written for a reader checking it against the paper by eye: every step
follows the paper's order and notation, uses numpy library routines (matmul,
slogdet, inv, eigh, qr, einsum) as single steps, and does no blocking, fusion or
reordering.  Notation: N orbitals, n_up/n_dn electrons, Gamma Cholesky vectors
L_g, K hidden variables, W walkers, P paths (trial samples) per walker, tau the
time step.  A "pair" is one (walker, path).

Readings of points where the paper is silent or ambiguous (those of R1-R17 that
concern the oracle):
  R1  H = sum_ij h_ij c+_i c_j + 1/2 sum_ijkl V_ijkl c+_i c+_k c_l c_j with
      V_ijkl = sum_g L_g,ij L_g,kl; so H = T + 1/2 sum_g L_g^2 (Eq. (3)) with
      T = h - 1/2 sum_g L_g L_g.
  R3  force bias xbar_g = -i sqrt(tau) <L_g> (the sqrt(-tau) of Eq. (4) carried
      into Eq. (15)); no mean-field subtraction.
  R4  the mixed estimate reports Re of the walker-averaged local energy.
  R5  weight update variants: combined angle (default), separate cosines,
      half-plane hand-off.
  R6  exp(A) of the auxiliary-field propagator = Taylor series to 6th order
      applied to the orbitals; exp(-tau T/2) and exp(sum_k x_k U_k) exact.
  R7  Metropolis accepts iff u < alpha with u in [0, 1) (53-bit).
  R8  proposals: independent draws from the prior p_T (the paper's choice),
      preconditioned Crank-Nicolson x' = sqrt(1-beta^2) x + beta xi, a
      Gaussian random walk x' = x + s xi, or the learned proposal (oracle.mlp)
      mixed with the random walk; Metropolis-Hastings with the proposal ratio.
  R9  walkers are re-orthonormalised every step (QR, diag(R) > 0).
  R10 population control (the branching random walk of Sec. II B and II D
      leaves the scheme open): optional comb every pop_period steps, at the
      end of the step, drawn with one Philox uniform; otherwise weights are
      carried.  Optional constant E_T.
  R11 initial walkers phi_w = Phi(x_w), x_w ~ p; paths x_wp ~ p; W = 1;
      n_burn Metropolis sweeps at fixed phi before the first step.
  R14 the local energy is measured every step at the start of the step.
  R17 importance function of the weight update (Sec. III A): "hybrid", |I| of
      Eq. (14) with the sampled-trial ratio Eq. (25) (default), or
      "local_energy", |I| = exp(-tau Re E_w(phi)) with E_w the path-averaged
      local energy Eq. (27) at the start of the step; the phase dtheta comes
      from the overlap ratio in both.
  R18 extra measurement paths (Sec. III A, last paragraph; Appendix B.3): from
      the current paths, `rounds` times `sweeps` measurement-only Metropolis
      sweeps at the current walker (own Philox tags; the learned proposal is
      replaced by the prior, as in burn-in), the paths after every round
      counting as P more samples; the walker's estimate is the sign-weighted
      average over all P' = rounds P of them, and its weight gets the factor
      R = (sum_p' S'_p' / P') / (sum_p S_p / P) in the numerator and the
      denominator of Eq. (16) (the normalisation by P' and P is a constant
      that cancels there).  Reported: Re of the complex ratio of the sums.
      The propagation's own paths are left as they were.
  R19 complex trial samples (Eq. (30), single slice): Phi(x) = exp(alpha
      sum_k x_k U_k) Phi0 with a complex alpha (-i sqrt(s) and U_k = L_k for
      the VAFQMC form; Phi0 absorbs exp(-t T) exp(-t0 T0) phi_T), so every
      overlap and Green's function takes Phi^dagger; the real form (alpha = 1)
      is unchanged.  Several slices (Eq. (19), Eq. (32)): Phi(x) = exp(alpha S_m)
      P ... P exp(alpha S_1) Phi0 with S_l = sum_k x_lk U_k and a fixed real
      P between slices (exp(-t T) for the ansatz), K hidden variables per slice.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import philox as px

__all__ = ["OracleConfig", "Hamiltonian", "State", "prepare", "trial_orbitals", "log_overlap",
           "green", "local_energy_force_bias", "measure", "init", "step", "reorthonormalise",
           "propagate_walker", "mcmc_sweep", "comb", "measure_paths", "n_hidden", "CONSTRAINTS", "IMPORTANCE"]

CONSTRAINTS = ("combined", "separate", "half_plane")
IMPORTANCE = ("hybrid", "local_energy")


@dataclasses.dataclass
class OracleConfig:
    dtau: float
    n_walkers: int
    n_paths: int
    seed: int
    n_sweeps: int = 1            # Metropolis sweeps M per step
    n_burn: int = 20             # sweeps before the first step (R11)
    constraint: str = "combined"
    proposal: str = "prior"      # "prior" or "pcn"
    pcn_beta: float = 1.0
    e_shift: float = 0.0         # constant E_T, weights *= exp(tau E_T) per step
    taylor_order: int = 6
    kill_threshold: float = 1e-10  # |sum_p S_p| below this kills the walker
    rw_step: float = 0.3         # Gaussian random-walk step (proposal "rw" and the fallback of "mlp")
    mlp_mix: float = 0.1         # probability of a random-walk move under proposal "mlp"
    mlp_params: object = None    # flat parameters of the learned proposal (oracle.mlp layout)
    mlp_hidden: int = 256
    importance: str = "hybrid"   # R17: "hybrid" or "local_energy"
    pop_period: int = 0          # R10: comb after every pop_period-th step (0: never)


@dataclasses.dataclass
class Hamiltonian:
    h: np.ndarray          # (N, N)
    L: np.ndarray          # (G, N, N)
    Phi0: np.ndarray       # (N, n_up)
    U: np.ndarray          # (K, N, N)
    n_up: int
    n_dn: int
    T: np.ndarray          # h - 1/2 sum_g L_g L_g
    expT_half: np.ndarray  # exp(-tau T / 2)
    alpha: complex = 1.0   # R19: Phi(x) = exp(alpha sum_k x_k U_k) Phi0 (1: the real form)
    slices: int = 1        # R19: hidden-variable slices of the trial (1: the one-slice form)
    slice_prop: np.ndarray = None  # (N, N) real propagator between slices (slices > 1)


@dataclasses.dataclass
class State:
    step: int
    phi_up: np.ndarray     # (W, N, n_up) complex128
    phi_dn: np.ndarray     # (W, N, n_dn) complex128
    weight: np.ndarray     # (W,) float64
    x: np.ndarray          # (W, P, K) float64 hidden variables of each path
    Phi: np.ndarray        # (W, P, N, n_up) float64, Phi(x); spin down uses the first n_dn columns
    walker_index: np.ndarray = None  # global index of each walker in the random streams (default 0..W-1)

    def __post_init__(self):
        if self.walker_index is None:
            self.walker_index = np.arange(self.weight.shape[0])

    def copy(self) -> "State":
        return State(self.step, self.phi_up.copy(), self.phi_dn.copy(), self.weight.copy(),
                     self.x.copy(), self.Phi.copy(), self.walker_index.copy())


# ---------------------------------------------------------------------------
# Hamiltonian and trial (Sec. II A, Eq. (1)-(5); Sec. II C, Eq. (20)-(21))
# ---------------------------------------------------------------------------

def _expm_sym(A: np.ndarray) -> np.ndarray:
    """exp of a real symmetric matrix (batched) through its eigendecomposition."""
    lam, V = np.linalg.eigh(A)
    return (V * np.exp(lam)[..., None, :]) @ np.swapaxes(V, -1, -2)


def prepare(h, L, Phi0, U, n_up: int, n_dn: int, dtau: float, alpha: complex = 1.0, slices: int = 1,
            slice_prop=None) -> Hamiltonian:
    """One-body operator of the Monte Carlo form, Eq. (3) with reading R1, and
    the exact half-step kinetic propagator exp(-tau T/2) of Eq. (5).  ``alpha``
    is the factor of the hidden-variable exponent (R19): 1 for the real trial
    samples, -i sqrt(s) for the single-slice VAFQMC form of Eq. (30) with
    U_k = L_k and Phi0 = exp(-t T) exp(-t0 T0) phi_T.  ``slices`` > 1 gives the
    multi-slice trial of Eq. (19) and Eq. (32) with ``slice_prop`` (e.g.
    exp(-t T)) between consecutive slices; each slice has its own K hidden
    variables."""
    if slices < 1 or (slices > 1 and slice_prop is None):
        raise ValueError("slices >= 1, and slice_prop for slices > 1")
    h = np.asarray(h, dtype=np.float64)
    L = np.asarray(L, dtype=np.float64)
    T = h - 0.5 * np.einsum("gij,gjk->ik", L, L)
    return Hamiltonian(h, L, np.asarray(Phi0, dtype=np.float64), np.asarray(U, dtype=np.float64),
                       n_up, n_dn, T, _expm_sym(-0.5 * dtau * T), complex(alpha) if alpha != 1.0 else 1.0,
                       int(slices), None if slice_prop is None else np.asarray(slice_prop, dtype=np.float64))


def n_hidden(ham: Hamiltonian) -> int:
    """Hidden variables of one trial sample: K per slice."""
    return ham.slices * ham.U.shape[0]


def trial_orbitals(ham: Hamiltonian, x: np.ndarray) -> np.ndarray:
    """Phi(x) = exp(alpha sum_k x_k U_k) Phi0, the determinant of one
    hidden-variable sample of the trial, Eq. (20)-(21) with one slice (alpha = 1,
    real), or the complex single-slice form of Eq. (30) (R19); x has shape (..., K)."""
    if ham.slices > 1:   # Phi(x) = e^{alpha S_m} P ... P e^{alpha S_1} Phi0, slice l using x[..., l K:(l+1) K]
        K = ham.U.shape[0]
        one = dataclasses.replace(ham, slices=1)
        Y = None
        for l in range(ham.slices):
            x_l = x[..., l * K:(l + 1) * K]
            if Y is None:
                Y = trial_orbitals(one, x_l)
            else:
                Y = _exp_hidden(ham, x_l) @ (ham.slice_prop @ Y)
        return Y
    return _exp_hidden(ham, x) @ ham.Phi0


def _exp_hidden(ham: Hamiltonian, x: np.ndarray) -> np.ndarray:
    """exp(alpha sum_k x_k U_k) (batched over the leading axes of x)."""
    S = np.einsum("...k,kij->...ij", x, ham.U)
    if ham.alpha == 1.0:
        return _expm_sym(S)
    lam, V = np.linalg.eigh(S)        # exp(alpha S) = V exp(alpha lam) V^T for real symmetric S
    return (V * np.exp(ham.alpha * lam)[..., None, :]) @ np.swapaxes(V, -1, -2)


# ---------------------------------------------------------------------------
# Overlaps, mixed Green's function, local energy and force bias
# ---------------------------------------------------------------------------

def _slog(A: np.ndarray) -> np.ndarray:
    """log det A as a complex number: log|det A| + i Arg det A."""
    if A.shape[-1] == 0:
        return np.zeros(A.shape[:-2], dtype=np.complex128)
    sign, logabs = np.linalg.slogdet(A)
    return logabs + 1j * np.angle(sign)


def _adj(A: np.ndarray) -> np.ndarray:
    """Conjugate transpose over the last two axes (the transpose for real A)."""
    return np.swapaxes(np.conj(A), -1, -2)


def log_overlap(ham: Hamiltonian, Phi: np.ndarray, phi_up: np.ndarray, phi_dn: np.ndarray) -> np.ndarray:
    """log <Phi|phi> = sum over spins of log det(Phi_s^dagger phi_s) (Eq. (25), (26));
    Phi^dagger = Phi^T for the real trial samples.  Shapes broadcast over leading axes."""
    Pu = Phi
    Pd = Phi[..., : ham.n_dn]
    return _slog(_adj(Pu) @ phi_up) + _slog(_adj(Pd) @ phi_dn)


def green(Phi_s: np.ndarray, phi_s: np.ndarray) -> np.ndarray:
    """Mixed one-body Green's function of one spin, G_ij = <Phi|c+_i c_j|phi>/<Phi|phi>
    = [phi (Phi^dagger phi)^-1 Phi^dagger]_ji."""
    A = _adj(Phi_s) @ phi_s
    M = phi_s @ np.linalg.inv(A) @ _adj(Phi_s)
    return np.swapaxes(M, -1, -2)


def local_energy_force_bias(ham: Hamiltonian, Phi: np.ndarray, phi_up: np.ndarray, phi_dn: np.ndarray):
    """Local energy E_L = <Phi|H|phi>/<Phi|phi> and the local values
    v_g = <Phi|L_g|phi>/<Phi|phi> of every Cholesky vector, for one pair.

    By Wick's theorem with G^s_ij = <c+_i c_j>:
      E_L = sum_s sum_ij h_ij G^s_ij
          + 1/2 sum_ijkl V_ijkl [ sum_st G^s_ij G^t_kl - sum_s G^s_il G^s_kj ],
    with V_ijkl = sum_g L_g,ij L_g,kl (reading R1).  v_g = sum_s sum_ij L_g,ij G^s_ij
    is the local value of L_g used by the force bias, Eq. (15).
    """
    Gs = [green(Phi, phi_up)]
    if ham.n_dn > 0:
        Gs.append(green(Phi[:, : ham.n_dn], phi_dn))
    L = ham.L
    e1 = sum(np.einsum("ij,ij->", ham.h, G) for G in Gs)
    v = sum(np.einsum("gij,ij->g", L, G) for G in Gs)
    coul = 0.5 * np.sum(v * v)
    exch = 0.0
    for G in Gs:
        exch = exch + 0.5 * np.einsum("gij,gkl,il,kj->", L, L, G, G, optimize=True)
    return e1 + coul - exch, v


def measure(ham: Hamiltonian, st: State):
    """Per-pair log-overlaps, local energies and force-bias values at the
    current walkers, and their path-sign-weighted averages over each walker's
    paths (Eq. (26)-(27))."""
    W, P = st.x.shape[:2]
    G = ham.L.shape[0]
    logov = np.empty((W, P), dtype=np.complex128)
    e_pair = np.empty((W, P), dtype=np.complex128)
    v_pair = np.empty((W, P, G), dtype=np.complex128)
    for w in range(W):
        for p in range(P):
            logov[w, p] = log_overlap(ham, st.Phi[w, p], st.phi_up[w], st.phi_dn[w])
            e_pair[w, p], v_pair[w, p] = local_energy_force_bias(ham, st.Phi[w, p], st.phi_up[w], st.phi_dn[w])
    S = np.exp(1j * logov.imag)                 # Eq. (26): phase of each path's overlap
    sumS = S.sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        e_bar = (S * e_pair).sum(axis=1) / sumS  # Eq. (27) with O = H
        v_bar = (S[:, :, None] * v_pair).sum(axis=1) / sumS[:, None]  # Eq. (27) with O = L_g
    return dict(logov=logov, e_pair=e_pair, v_pair=v_pair, S=S, sumS=sumS, e_bar=e_bar, v_bar=v_bar)


def mixed_energy(weight: np.ndarray, e_bar: np.ndarray):
    """Mixed estimator, Eq. (16), real part (R4); walkers with W = 0 do not enter,
    nor walkers without a finite estimate (non-finite orbitals, which the kill rule
    R15 removes in the same step)."""
    alive = (weight > 0) & np.isfinite(e_bar)
    num = float(np.sum(weight[alive] * e_bar[alive].real))
    den = float(np.sum(weight[alive]))
    return num, den


# ---------------------------------------------------------------------------
# Propagation (Eq. (5), (12)-(15)), Metropolis on the paths (Eq. (23)), reorthonormalisation
# ---------------------------------------------------------------------------

def propagate_walker(ham: Hamiltonian, phi: np.ndarray, y: np.ndarray, dtau: float, order: int) -> np.ndarray:
    """phi' = exp(-tau T/2) exp(i sqrt(tau) sum_g y_g L_g) exp(-tau T/2) phi,
    i.e. B(x - xbar) of Eq. (5) and (12) with y = x - xbar; the middle exponential is its
    Taylor series to ``order`` (R6)."""
    A = 1j * math.sqrt(dtau) * np.einsum("g,gij->ij", y, ham.L)
    psi = ham.expT_half @ phi
    term = psi
    acc = psi.copy()
    for m in range(1, order + 1):
        term = (A @ term) / m
        acc = acc + term
    return ham.expT_half @ acc


def reorthonormalise(phi: np.ndarray) -> np.ndarray:
    """phi = Q R with diag(R) real positive; return Q (R9).  The determinant
    ratios and Green's functions are unchanged because phi -> phi R^-1 only
    rescales every overlap by the same det R."""
    if phi.shape[-1] == 0:
        return phi.copy()
    Q, R = np.linalg.qr(phi)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    return Q * (d / np.abs(d))[..., None, :]


def mcmc_sweep(ham: Hamiltonian, cfg: OracleConfig, st: State, logov_cur: np.ndarray, alive: np.ndarray,
               step: int, sweep: int, tag_prop: int, tag_acc: int, mlp_mu_logv=None) -> int:
    """One Metropolis update of every path of every live walker against the
    walkers' current orbitals (leapfrog step 2, Sec. III A; Appendix B.2):
    propose x', build Phi(x'), accept iff u < alpha with the Metropolis-Hastings
    ratio alpha of the target p(x)|<Phi(x)|phi>| (Eq. (23)) and the proposal:
    prior or pCN proposals leave alpha = |<Phi(x')|phi>| / |<Phi(x)|phi>| (the
    paper's form); the random walk adds p(x')/p(x); the learned proposal
    q = N(mu_w, diag v_w) adds p(x') q(x) / (p(x) q(x')).  Updates st.x, st.Phi
    and logov_cur in place; returns the number of accepted moves."""
    W, P, K = st.x.shape
    pair_ids = (st.walker_index[:, None] * P + np.arange(P)[None, :]).reshape(-1)
    xi = px.normals(cfg.seed, tag_prop, step, pair_ids, sweep, K).reshape(W, P, K)
    uu = px.uniforms(cfg.seed, tag_acc, step, pair_ids, sweep, 2).reshape(W, P, 2)
    u, u_mix = uu[..., 0], uu[..., 1]
    extra = np.zeros((W, P))
    if cfg.proposal == "prior":
        x_new = xi
    elif cfg.proposal == "pcn":
        b = cfg.pcn_beta
        x_new = math.sqrt(1.0 - b * b) * st.x + b * xi
    elif cfg.proposal == "rw":
        x_new = st.x + cfg.rw_step * xi
        extra = -0.5 * (np.sum(x_new * x_new, axis=-1) - np.sum(st.x * st.x, axis=-1))
    elif cfg.proposal == "mlp":
        mu, logv = mlp_mu_logv
        use_rw = u_mix < cfg.mlp_mix
        x_rw = st.x + cfg.rw_step * xi
        x_q = mu[:, None, :] + np.exp(0.5 * logv)[:, None, :] * xi
        x_new = np.where(use_rw[..., None], x_rw, x_q)
        extra = -0.5 * (np.sum(x_new * x_new, axis=-1) - np.sum(st.x * st.x, axis=-1))
        lq_old = -0.5 * np.sum((st.x - mu[:, None, :]) ** 2 * np.exp(-logv)[:, None, :], axis=-1)
        lq_new = -0.5 * np.sum((x_new - mu[:, None, :]) ** 2 * np.exp(-logv)[:, None, :], axis=-1)
        extra = extra + np.where(use_rw, 0.0, lq_old - lq_new)
    else:
        raise ValueError(cfg.proposal)
    n_acc = 0
    for w in range(W):
        if not alive[w]:
            continue
        for p in range(P):
            Phi_new = trial_orbitals(ham, x_new[w, p])
            lo_new = log_overlap(ham, Phi_new, st.phi_up[w], st.phi_dn[w])
            delta = lo_new.real - logov_cur[w, p].real + extra[w, p]
            if delta >= 0.0 or u[w, p] < math.exp(delta):
                st.x[w, p] = x_new[w, p]
                st.Phi[w, p] = Phi_new
                logov_cur[w, p] = lo_new
                n_acc += 1
    return n_acc


def measure_paths(ham: Hamiltonian, cfg: OracleConfig, st: State, rounds: int, sweeps: int):
    """Mixed energy from extra, measurement-only paths (R18; Sec. III A and
    Appendix B.3).  ``st`` is not modified.

    Returns e_mix (Re of sum_w W_w R_w E'_w / sum_w W_w R_w over the live
    walkers), the per-walker estimates E'_w, the factors R_w and the live mask.
    """
    W, P = st.x.shape[:2]
    m = measure(ham, st)
    alive = (st.weight > 0) & (np.abs(m["sumS"]) > cfg.kill_threshold)
    work = st.copy()
    logov = m["logov"].copy()
    mcfg = dataclasses.replace(cfg, proposal="prior") if cfg.proposal == "mlp" else cfg
    num = np.zeros(W, dtype=np.complex128)       # sum over the P' paths of S' E_L
    den = np.zeros(W, dtype=np.complex128)       # sum over the P' paths of S'
    for r in range(rounds):
        for s in range(sweeps):
            mcmc_sweep(ham, mcfg, work, logov, alive, st.step, r * sweeps + s, px.TAG_MEAS_PROPOSE,
                       px.TAG_MEAS_ACCEPT)
        mr = measure(ham, work)
        num += (mr["S"] * mr["e_pair"]).sum(axis=1)
        den += mr["S"].sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        e_walker = num / den
        R = (den / (rounds * P)) / (m["sumS"] / P)
    wr = np.where(alive, st.weight * R, 0.0)
    e_mix = complex(np.sum(wr[alive] * e_walker[alive]) / np.sum(wr[alive])).real
    return dict(e_mix=e_mix, e_walker=e_walker, R=R, alive=alive, num=num, den=den)


def init(ham: Hamiltonian, cfg: OracleConfig, walker_index=None) -> State:
    """Initial composite walkers (reading R11 of Appendix B.1).  ``walker_index``
    (default 0..W-1) gives the global walker numbers used in the random streams,
    so a subset of a larger population can be rebuilt on its own."""
    W, P = cfg.n_walkers, cfg.n_paths
    K = n_hidden(ham)
    widx = np.arange(W) if walker_index is None else np.asarray(walker_index)
    W = widx.size
    xw = px.normals(cfg.seed, px.TAG_INIT_WALKER, 0, widx, 0, K)
    Phiw = trial_orbitals(ham, xw)                                   # (W, N, n_up)
    phi_up = reorthonormalise(Phiw.astype(np.complex128))
    phi_dn = reorthonormalise(Phiw[:, :, : ham.n_dn].astype(np.complex128))
    pair_ids = (widx[:, None] * P + np.arange(P)[None, :]).reshape(-1)
    x = px.normals(cfg.seed, px.TAG_INIT_PATH, 0, pair_ids, 0, K).reshape(W, P, K)
    Phi = trial_orbitals(ham, x)
    st = State(0, phi_up, phi_dn, np.ones(W), x, Phi, widx.copy())
    logov = np.empty((W, P), dtype=np.complex128)
    for w in range(W):
        for p in range(P):
            logov[w, p] = log_overlap(ham, Phi[w, p], phi_up[w], phi_dn[w])
    alive = np.ones(W, dtype=bool)
    burn_cfg = dataclasses.replace(cfg, proposal="prior") if cfg.proposal == "mlp" else cfg   # no network output yet
    for b in range(cfg.n_burn):
        mcmc_sweep(ham, burn_cfg, st, logov, alive, 0, b, px.TAG_BURN_PROPOSE, px.TAG_BURN_ACCEPT)
    return st


def _wrap(a):
    return np.angle(np.exp(1j * a))


def comb(weight: np.ndarray, u: float):
    """Comb population control (R10).

    The W walkers' weights are laid end to end on [0, sum W); W teeth spaced
    sum W / W apart, the first at u sum W / W with u in [0, 1), each pick the
    walker whose interval holds them, so walker w gets c_w copies, and every
    new walker has weight sum W / W.  Slots: a walker with c_w >= 1 keeps its
    own slot; the c_w - 1 extra copies of each walker, in increasing w, fill the
    slots of the walkers with c_w = 0, in increasing slot order.  Returns
    (source walker of every slot, new weights); with no positive total weight
    the population is left as it is.  Tooth positions are (j + u) * (sum W / W)
    in FP64, which for u within an ulp of 1 can round onto the next interval's
    boundary (a valid comb still, at probability ~2^-53).
    """
    W = weight.shape[0]
    cum = np.empty(W)
    acc = 0.0
    for w in range(W):                 # running sum, left to right
        acc += weight[w]
        cum[w] = acc
    total = cum[-1]
    if not (total > 0.0 and math.isfinite(total)):
        return np.arange(W), weight.copy()
    width = total / W
    teeth = (np.arange(W) + u) * width
    # tooth j picks the first walker whose running sum exceeds it; rounding can put
    # the last tooth at the total, which then goes to the last walker of positive weight
    picked = np.minimum(np.searchsorted(cum, teeth, side="right"), int(np.nonzero(weight > 0.0)[0][-1]))
    copies = np.bincount(picked, minlength=W)
    extras = [w for w in range(W) for _ in range(copies[w] - 1)]
    free = [j for j in range(W) if copies[j] == 0]
    src = np.arange(W)
    src[free] = extras
    return src, np.full(W, width)


def step(ham: Hamiltonian, cfg: OracleConfig, st: State, mlp_mu_logv=None):
    """One leapfrog step (Sec. III A and the propagation outline of Appendix B.2).

    Returns the new state and a dict of diagnostics; ``mixed`` holds the mixed
    energy numerator and denominator measured at the start of the step (R14).
    """
    i = st.step
    W, P, K = st.x.shape
    G = ham.L.shape[0]
    tau = cfg.dtau
    new = st.copy()

    # Local energies, force-bias values and path signs at phi (Eq. (26)-(27)).
    m = measure(ham, st)
    mixed = mixed_energy(st.weight, m["e_bar"])
    alive = (st.weight > 0) & (np.abs(m["sumS"]) > cfg.kill_threshold)
    new.weight[~alive] = 0.0

    # Leapfrog step 1: fields, force bias (Eq. (15)), propagation (Eq. (12)).
    xi = px.normals(cfg.seed, px.TAG_FIELD, i, st.walker_index, 0, G)
    xbar = -1j * math.sqrt(tau) * m["v_bar"]
    y = xi - xbar
    logov_new = m["logov"].copy()
    ratio = np.ones(W, dtype=np.complex128)
    old_sum = np.zeros(W, dtype=np.complex128)
    I_abs = np.zeros(W)
    I_full = np.zeros(W, dtype=np.complex128)
    for w in range(W):
        if not alive[w]:
            continue
        new.phi_up[w] = propagate_walker(ham, st.phi_up[w], y[w], tau, cfg.taylor_order)
        new.phi_dn[w] = propagate_walker(ham, st.phi_dn[w], y[w], tau, cfg.taylor_order)
        for p in range(P):
            logov_new[w, p] = log_overlap(ham, st.Phi[w, p], new.phi_up[w], new.phi_dn[w])
        # Overlap ratio estimated with the sampled trial, Eq. (25).
        terms = m["S"][w] * np.exp(logov_new[w] - m["logov"][w])
        old_sum[w] = terms.sum()
        ratio[w] = old_sum[w] / m["sumS"][w]
        # Importance function Eq. (14): p(x - xbar)/p(x) times the ratio.
        log_shift = np.sum(xi[w] * xbar[w] - 0.5 * xbar[w] * xbar[w])
        I_full[w] = np.exp(log_shift) * ratio[w]
        if cfg.importance == "hybrid":
            I_abs[w] = abs(I_full[w])
        elif cfg.importance == "local_energy":   # R17: exp(-tau E_L(phi)), Sec. III A
            I_abs[w] = math.exp(-tau * m["e_bar"][w].real)
        else:
            raise ValueError(cfg.importance)

    # Leapfrog step 2: Metropolis update of the paths at phi' (Sec. III A).
    if cfg.proposal == "mlp" and ham.slices > 1:
        # the network's features and output are defined over the K variables of one slice
        raise ValueError("the learned proposal is defined for one-slice trials only")
    if cfg.proposal == "mlp" and mlp_mu_logv is None:
        from . import mlp as _mlp
        f = _mlp.features(ham.Phi0, ham.U, new.phi_up, new.phi_dn)
        fw = _mlp.forward(cfg.mlp_params, f, ham.U.shape[0], cfg.mlp_hidden)
        mlp_mu_logv = (fw["mu"], fw["logv"])
    n_acc = 0
    for s in range(cfg.n_sweeps):
        n_acc += mcmc_sweep(ham, cfg, new, logov_new, alive, i, s, px.TAG_PROPOSE, px.TAG_ACCEPT, mlp_mu_logv)

    # Hand-off ratio Eq. (28) and the constraints Eq. (17), (29).
    for w in range(W):
        if not alive[w]:
            continue
        S_new = np.exp(1j * logov_new[w].imag)
        dtheta = np.angle(ratio[w])
        dtheta_T = np.angle(S_new.sum()) - np.angle(old_sum[w])
        if cfg.constraint == "combined":
            f = max(0.0, math.cos(dtheta + dtheta_T))
        elif cfg.constraint == "separate":
            f = max(0.0, math.cos(dtheta)) * max(0.0, math.cos(dtheta_T))
        elif cfg.constraint == "half_plane":
            f = max(0.0, math.cos(dtheta)) * (1.0 if abs(_wrap(dtheta_T)) <= 0.5 * math.pi else 0.0)
        else:
            raise ValueError(cfg.constraint)
        wnew = st.weight[w] * I_abs[w] * f * math.exp(tau * cfg.e_shift)
        new.weight[w] = wnew if math.isfinite(wnew) else 0.0

    # Reorthonormalise the propagated walkers (R9).
    for w in range(W):
        if alive[w]:
            new.phi_up[w] = reorthonormalise(new.phi_up[w])
            new.phi_dn[w] = reorthonormalise(new.phi_dn[w])
    new.step = i + 1

    # Population control (R10): comb at the end of every pop_period-th step.
    comb_src = None
    if cfg.pop_period > 0 and (i + 1) % cfg.pop_period == 0:
        u = px.uniforms(cfg.seed, px.TAG_COMB, i, st.walker_index[:1], 0, 1)[0, 0]
        comb_src, new.weight = comb(new.weight, u)
        new.phi_up = new.phi_up[comb_src]
        new.phi_dn = new.phi_dn[comb_src]
        new.x = new.x[comb_src]
        new.Phi = new.Phi[comb_src]
    diag = dict(mixed=mixed, n_accept=n_acc, n_proposed=int(alive.sum()) * P * cfg.n_sweeps,
                alive=alive, e_bar=m["e_bar"], v_bar=m["v_bar"], ratio=ratio, measure=m,
                old_sum=old_sum, new_sum=np.exp(1j * logov_new.imag).sum(axis=1), logov_new=logov_new,
                xi=xi, I_abs=I_abs, I=I_full, comb_src=comb_src)
    return new, diag
