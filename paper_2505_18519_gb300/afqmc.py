"""Python binding of ``libafqmc.so`` (the C ABI in include/afqmc.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device workspace and the CUDA stream.
There is no CPU fallback: without the built library or a GPU every call
raises.
"""

from __future__ import annotations

import ctypes
import os
import struct
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libafqmc.so")

CONSTRAINTS = {"combined": 0, "separate": 1, "half_plane": 2}
PROPOSALS = {"prior": 0, "pcn": 1, "rw": 2, "mlp": 3}
PRECISIONS = {"fp64": 0, "bf16x3": 1, "fp16x3": 2, "fp16x6": 3}
IMPORTANCE = {"hybrid": 0, "local_energy": 1}
TC_FORMS = {"auto": 0, "per_pair": 1, "walker": 2}
TRIAL_FORMS = {"auto": 0, "df": 1, "tc": 2}
OVERLAP_FORMS = {"auto": 0, "df": 1}
STATE_MAGIC = 0x4146514D43535431


class AfqmcConfig(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int), ("n_up", ctypes.c_int), ("n_dn", ctypes.c_int), ("n_chol", ctypes.c_int),
        ("K", ctypes.c_int), ("n_walkers", ctypes.c_int), ("n_paths", ctypes.c_int), ("n_sweeps", ctypes.c_int),
        ("n_burn", ctypes.c_int), ("constraint", ctypes.c_int), ("proposal", ctypes.c_int),
        ("precision", ctypes.c_int), ("taylor_order", ctypes.c_int), ("history_capacity", ctypes.c_int),
        ("dtau", ctypes.c_double), ("pcn_beta", ctypes.c_double), ("e_shift", ctypes.c_double),
        ("kill_threshold", ctypes.c_double), ("seed", ctypes.c_uint64), ("walker_offset", ctypes.c_int64),
        ("rw_step", ctypes.c_double), ("mlp_mix", ctypes.c_double), ("mlp_lr", ctypes.c_double),
        ("mlp_train", ctypes.c_int), ("refine_tol", ctypes.c_double),
        ("importance", ctypes.c_int), ("pop_period", ctypes.c_int), ("rcache", ctypes.c_int),
        ("wait_polls", ctypes.c_int64), ("tc_form", ctypes.c_int),
        ("trial_alpha_re", ctypes.c_double), ("trial_alpha_im", ctypes.c_double), ("trial_slices", ctypes.c_int),
        ("trial_form", ctypes.c_int),
        ("overlap_form", ctypes.c_int),
    ]


_lib = None

EXPORTS = ("afqmc_config_default", "afqmc_workspace_bytes", "afqmc_init", "afqmc_init_trial", "afqmc_step",
           "afqmc_energy",
           "afqmc_energy_paths", "afqmc_observables", "afqmc_history", "afqmc_stats", "afqmc_state_save", "afqmc_state_load",
           "afqmc_destroy", "afqmc_last_error", "afqmc_philox_fill", "afqmc_profile", "afqmc_profile_read",
           "afqmc_launch_count", "afqmc_contract_kernel", "afqmc_autotune", "afqmc_batch_create", "afqmc_batch_step", "afqmc_batch_sync",
           "afqmc_batch_destroy", "afqmc_mlp_n_params", "afqmc_mlp_params", "afqmc_mlp_eval", "afqmc_mlp_state",
           "afqmc_fp64_fma_rate", "afqmc_local_energy_noalloc", "afqmc_noalloc_scratch_bytes",
           "afqmc_noalloc_last_error", "afqmc_trial_orbitals", "afqmc_batch_shared_contractions")

PHASES = ("overlap", "contract", "average", "fields", "propagate", "ratio", "propose", "trial_orbitals",
          "mcmc_overlap", "accept", "finish", "comb", "refine")


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2505_18519_gb300.build`")
    lib = ctypes.CDLL(path)
    P, D, I, U64, SZ = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_uint64, ctypes.c_size_t
    cfgp = ctypes.POINTER(AfqmcConfig)
    lib.afqmc_config_default.argtypes = [cfgp]
    lib.afqmc_config_default.restype = None
    lib.afqmc_workspace_bytes.argtypes = [cfgp]
    lib.afqmc_workspace_bytes.restype = SZ
    lib.afqmc_init.argtypes = [cfgp, P, P, P, P, P, SZ, P, ctypes.POINTER(P)]
    lib.afqmc_init.restype = I
    lib.afqmc_init_trial.argtypes = [cfgp, P, P, P, P, P, P, SZ, P, ctypes.POINTER(P)]
    lib.afqmc_init_trial.restype = I
    lib.afqmc_step.argtypes = [P, I]
    lib.afqmc_step.restype = I
    lib.afqmc_energy.argtypes = [P, D, D, D, P]
    lib.afqmc_energy.restype = I
    lib.afqmc_energy_paths.argtypes = [P, I, I, D, P, P]
    lib.afqmc_energy_paths.restype = I
    lib.afqmc_observables.argtypes = [P, P, P, P]
    lib.afqmc_observables.restype = I
    lib.afqmc_trial_orbitals.argtypes = [P, P, ctypes.c_int64, P]
    lib.afqmc_trial_orbitals.restype = I
    lib.afqmc_history.argtypes = [P, P, I, ctypes.POINTER(I)]
    lib.afqmc_history.restype = I
    lib.afqmc_stats.argtypes = [P, P, I]
    lib.afqmc_stats.restype = I
    lib.afqmc_state_save.argtypes = [P, P, ctypes.POINTER(SZ)]
    lib.afqmc_state_save.restype = I
    lib.afqmc_state_load.argtypes = [P, P, SZ]
    lib.afqmc_state_load.restype = I
    lib.afqmc_destroy.argtypes = [P]
    lib.afqmc_destroy.restype = None
    lib.afqmc_last_error.argtypes = []
    lib.afqmc_last_error.restype = ctypes.c_char_p
    lib.afqmc_philox_fill.argtypes = [P, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, U64, P]
    lib.afqmc_philox_fill.restype = I
    lib.afqmc_profile.argtypes = [P, I]
    lib.afqmc_profile.restype = I
    lib.afqmc_profile_read.argtypes = [P, P, I]
    lib.afqmc_profile_read.restype = I
    lib.afqmc_launch_count.argtypes = []
    lib.afqmc_launch_count.restype = ctypes.c_int64
    lib.afqmc_contract_kernel.argtypes = [ctypes.c_void_p]
    lib.afqmc_contract_kernel.restype = ctypes.c_int
    lib.afqmc_autotune.argtypes = [P, P]
    lib.afqmc_autotune.restype = I
    lib.afqmc_batch_create.argtypes = [I, P, P, ctypes.POINTER(P)]
    lib.afqmc_batch_create.restype = I
    lib.afqmc_batch_step.argtypes = [P, I]
    lib.afqmc_batch_step.restype = I
    lib.afqmc_batch_sync.argtypes = [P]
    lib.afqmc_batch_sync.restype = I
    lib.afqmc_batch_shared_contractions.argtypes = [P]
    lib.afqmc_batch_shared_contractions.restype = I
    lib.afqmc_batch_destroy.argtypes = [P]
    lib.afqmc_batch_destroy.restype = None
    lib.afqmc_mlp_n_params.argtypes = [I]
    lib.afqmc_mlp_n_params.restype = ctypes.c_int64
    lib.afqmc_mlp_params.argtypes = [P, P, ctypes.c_int64, I]
    lib.afqmc_mlp_params.restype = I
    lib.afqmc_mlp_eval.argtypes = [P, I, P, P, P, P, P]
    lib.afqmc_mlp_eval.restype = I
    lib.afqmc_mlp_state.argtypes = [P, P, P, P]
    lib.afqmc_mlp_state.restype = I
    lib.afqmc_noalloc_scratch_bytes.argtypes = []
    lib.afqmc_noalloc_scratch_bytes.restype = SZ
    lib.afqmc_local_energy_noalloc.argtypes = [I, I, I, I, ctypes.c_int64, I, P, P, P, P, P, P, P, P]
    lib.afqmc_local_energy_noalloc.restype = I
    lib.afqmc_fp64_fma_rate.argtypes = [D, P]
    lib.afqmc_fp64_fma_rate.restype = I
    lib.afqmc_noalloc_last_error.argtypes = []
    lib.afqmc_noalloc_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


class AfqmcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"afqmc status {status}: {msg}")
        self.status = status


def _check(st: int):
    if st != 0:
        raise AfqmcError(st, load_library().afqmc_last_error().decode())


def make_config(N, n_up, n_dn, n_chol, K, n_walkers, n_paths, dtau, seed, *, n_sweeps=1, n_burn=20,
                constraint="combined", proposal="prior", precision="fp64", taylor_order=6, history_capacity=1024,
                pcn_beta=1.0, e_shift=0.0, kill_threshold=1e-10, walker_offset=0, rw_step=0.3, mlp_mix=0.1,
                mlp_lr=1e-3, mlp_train=False, refine_tol=1e-4, importance="hybrid",
                pop_period=0, rcache=False, wait_polls=0, tc_form="auto", trial_alpha=1.0,
                trial_slices=1, trial_form="auto", overlap_form="auto") -> AfqmcConfig:
    lib = load_library()
    c = AfqmcConfig()
    lib.afqmc_config_default(ctypes.byref(c))
    c.N, c.n_up, c.n_dn, c.n_chol, c.K = N, n_up, n_dn, n_chol, K
    c.n_walkers, c.n_paths, c.n_sweeps, c.n_burn = n_walkers, n_paths, n_sweeps, n_burn
    c.constraint, c.proposal, c.precision = CONSTRAINTS[constraint], PROPOSALS[proposal], PRECISIONS[precision]
    c.taylor_order, c.history_capacity = taylor_order, history_capacity
    c.dtau, c.pcn_beta, c.e_shift, c.kill_threshold, c.seed = dtau, pcn_beta, e_shift, kill_threshold, seed
    c.walker_offset = walker_offset
    c.rw_step, c.mlp_mix, c.mlp_lr, c.mlp_train = rw_step, mlp_mix, mlp_lr, int(bool(mlp_train))
    c.refine_tol = refine_tol
    c.importance, c.pop_period = IMPORTANCE[importance], pop_period
    c.rcache = int(bool(rcache))
    c.wait_polls = int(wait_polls)
    c.tc_form = TC_FORMS[tc_form]
    c.trial_alpha_re, c.trial_alpha_im = complex(trial_alpha).real, complex(trial_alpha).imag
    c.trial_slices = int(trial_slices)
    c.trial_form = TRIAL_FORMS[trial_form]
    c.overlap_form = OVERLAP_FORMS[overlap_form]
    return c


def workspace_bytes(cfg: AfqmcConfig) -> int:
    return int(load_library().afqmc_workspace_bytes(ctypes.byref(cfg)))


def _ptr(a):
    """(pointer, keepalive) of a float64 C-contiguous numpy array or torch tensor."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != torch.float64 or not a.is_contiguous():
                a = a.to(torch.float64).contiguous()
            return a.data_ptr(), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.ctypes.data, a


class Context:
    """One AFQMC run: configuration, Hamiltonian, walkers and paths on one GPU."""

    def __init__(self, cfg: AfqmcConfig, h, L, Phi0, U, device=None, stream=None, slice_prop=None):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.cfg = cfg
        self.device = torch.device(device if device is not None else "cuda")
        nbytes = workspace_bytes(cfg)
        if nbytes == 0:
            # let the library report why
            st = lib.afqmc_init(ctypes.byref(cfg), None, None, None, None, None, 0, None, ctypes.byref(ctypes.c_void_p()))
            _check(st)
        self._ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        keep = [_ptr(x) for x in (h, L, Phi0, U)]
        sp = _ptr(slice_prop) if slice_prop is not None else (None, None)
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.afqmc_init_trial(ctypes.byref(cfg), keep[0][0], keep[1][0], keep[2][0], keep[3][0], sp[0],
                                        self._ws_ptr, nbytes, self.stream.cuda_stream, ctypes.byref(self._ctx)))
        self.W, self.P, self.G, self.K = cfg.n_walkers, cfg.n_paths, cfg.n_chol, cfg.K
        self.N, self.nu, self.nd = cfg.N, cfg.n_up, cfg.n_dn

    # -- stepping and measurement -------------------------------------------------
    def step(self, n_steps: int = 1):
        _check(load_library().afqmc_step(self._ctx, int(n_steps)))

    def energy(self, walkers: bool = False):
        e, sw, ms = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        ew = np.empty(2 * self.W) if walkers else None
        st = load_library().afqmc_energy(self._ctx, ctypes.byref(e), ctypes.byref(sw), ctypes.byref(ms),
                                         ew.ctypes.data if walkers else None)
        _check(st)
        out = dict(e_mix=e.value, sum_w=sw.value, mean_sign=ms.value)
        if walkers:
            out["e_walker"] = ew.view(np.complex128)
        return out

    def trial_orbitals(self, x) -> np.ndarray:
        """Phi(x) for the rows of x (n x K): (n, N, n_up), complex for a complex or multi-slice trial."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, self.K)
        cplx = complex(self.cfg.trial_alpha_re, self.cfg.trial_alpha_im) != 1.0 or self.cfg.trial_slices > 1
        out = np.empty((x.shape[0], self.N, self.nu), dtype=np.complex128 if cplx else np.float64)
        _check(load_library().afqmc_trial_orbitals(self._ctx, x.ctypes.data, x.shape[0], out.ctypes.data))
        return out

    def energy_paths(self, rounds: int, sweeps: int):
        """Mixed energy from extra measurement-only paths (see afqmc_energy_paths)."""
        e = ctypes.c_double()
        ew = np.empty(2 * self.W)
        R = np.empty(2 * self.W)
        _check(load_library().afqmc_energy_paths(self._ctx, int(rounds), int(sweeps), ctypes.byref(e),
                                                 ew.ctypes.data, R.ctypes.data))
        return dict(e_mix=e.value, e_walker=ew.view(np.complex128), ratio=R.view(np.complex128))

    def observables(self):
        lo = np.empty(2 * self.W * self.P)
        el = np.empty(2 * self.W * self.P)
        fb = np.empty(2 * self.W * self.G)
        _check(load_library().afqmc_observables(self._ctx, lo.ctypes.data, el.ctypes.data, fb.ctypes.data))
        return dict(logov=lo.view(np.complex128).reshape(self.W, self.P),
                    e_local=el.view(np.complex128).reshape(self.W, self.P),
                    force_bias=fb.view(np.complex128).reshape(self.W, self.G))

    def history(self, n: int):
        out = np.empty(4 * max(n, 1))
        k = ctypes.c_int()
        _check(load_library().afqmc_history(self._ctx, out.ctypes.data, int(n), ctypes.byref(k)))
        return out[: 4 * k.value].reshape(k.value, 4)

    def stats(self):
        out = np.empty(14)
        _check(load_library().afqmc_stats(self._ctx, out.ctypes.data, 14))
        keys = ("steps", "accepted", "proposed", "live_walkers", "status", "min_weight", "max_weight", "sum_weight",
                "refined_pairs", "combs", "comb_replaced", "rcache_formed", "cheb_terms", "cheb_redone")
        return dict(zip(keys, out.tolist()))

    def autotune(self):
        """Pick the fastest launch shapes for this context (cached per shape)."""
        out = (ctypes.c_int * 3)()
        _check(load_library().afqmc_autotune(self._ctx, out))
        return dict(overlap_warps_per_block=out[0], tc_pairs_per_block=out[1], trial_threads=out[2])

    # -- learned proposal ---------------------------------------------------------
    def mlp_params(self, new=None):
        """Get (new None) or set the flat FP32 parameters of the proposal network."""
        lib = load_library()
        n = int(lib.afqmc_mlp_n_params(self.K))
        if new is None:
            out = np.empty(n, dtype=np.float32)
            _check(lib.afqmc_mlp_params(self._ctx, out.ctypes.data, n, 0))
            return out
        a = np.ascontiguousarray(new, dtype=np.float32)
        _check(lib.afqmc_mlp_params(self._ctx, a.ctypes.data, a.size, 1))

    def mlp_eval(self, features, x):
        """Network output, loss and flat gradient for features (B, K), x (B, P, K)."""
        lib = load_library()
        f = np.ascontiguousarray(features, dtype=np.float32)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        B = f.shape[0]
        mu_logv = np.empty((B, 2 * self.K), dtype=np.float32)
        loss = ctypes.c_double()
        grad = np.empty(int(lib.afqmc_mlp_n_params(self.K)), dtype=np.float32)
        _check(lib.afqmc_mlp_eval(self._ctx, B, f.ctypes.data, xx.ctypes.data, mu_logv.ctypes.data, ctypes.byref(loss),
                                  grad.ctypes.data))
        return dict(mu=mu_logv[:, :self.K], logv=mu_logv[:, self.K:], loss=loss.value, grad=grad)

    def mlp_state(self):
        """Features, mu and logv (each (W, K)) used by the last step's proposals."""
        out = [np.empty((self.W, self.K), dtype=np.float32) for _ in range(3)]
        _check(load_library().afqmc_mlp_state(self._ctx, *[o.ctypes.data for o in out]))
        return dict(features=out[0], mu=out[1], logv=out[2])

    # -- profiling ----------------------------------------------------------------
    def profile(self, enable: bool = True):
        _check(load_library().afqmc_profile(self._ctx, int(bool(enable))))

    def profile_read(self) -> dict:
        n = len(PHASES)
        out = np.zeros(2 * n + 1)
        _check(load_library().afqmc_profile_read(self._ctx, out.ctypes.data, out.size))
        return dict(ms=dict(zip(PHASES, out[:n].tolist())), launches=dict(zip(PHASES, out[n:2 * n].astype(int).tolist())),
                    steps=int(out[2 * n]))

    # -- checkpoint ---------------------------------------------------------------
    def save_state(self) -> bytes:
        lib = load_library()
        n = ctypes.c_size_t()
        _check(lib.afqmc_state_save(self._ctx, None, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib.afqmc_state_save(self._ctx, buf, ctypes.byref(n)))
        return buf.raw

    def load_state(self, blob: bytes):
        _check(load_library().afqmc_state_load(self._ctx, blob, len(blob)))

    def state_arrays(self) -> dict:
        return unpack_state(self.save_state())

    def load_state_arrays(self, st: dict):
        self.load_state(pack_state(st))

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            load_library().afqmc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def local_energy_noalloc(N, n_up, n_dn, n_chol, n_pairs, pairs_per_walker, h, L, Phi, phi, logov, e_local,
                         force_bias, stream=None):
    """Local energies of a batch of pairs with no device allocation (all
    arguments are CUDA float64 tensors; ``phi`` holds re, im pairs).  For callers
    that cannot allocate device memory; see include/afqmc.h."""
    import torch
    lib = load_library()
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib.afqmc_local_energy_noalloc(N, n_up, n_dn, n_chol, int(n_pairs), pairs_per_walker, h.data_ptr(),
                                        L.data_ptr(), Phi.data_ptr(), phi.data_ptr(), logov.data_ptr(),
                                        e_local.data_ptr(), force_bias.data_ptr(), s.cuda_stream)
    if st != 0:
        raise AfqmcError(st, lib.afqmc_noalloc_last_error().decode())


class Batch:
    """Several contexts stepped together by one CUDA graph launch per step.
    Each context must have been created with its own stream."""

    def __init__(self, contexts, stream=None):
        import torch
        self.contexts = list(contexts)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = (ctypes.c_void_p * len(self.contexts))(*[c._ctx.value for c in self.contexts])
        self._b = ctypes.c_void_p()
        _check(load_library().afqmc_batch_create(len(self.contexts), arr, self.stream.cuda_stream, ctypes.byref(self._b)))

    def step(self, n_steps: int = 1):
        _check(load_library().afqmc_batch_step(self._b, int(n_steps)))

    def sync(self):
        _check(load_library().afqmc_batch_sync(self._b))

    @property
    def shared_contractions(self) -> int:
        """Systems whose GEMM-Z runs in the batch's one persistent launch."""
        return int(load_library().afqmc_batch_shared_contractions(self._b))

    def close(self):
        if getattr(self, "_b", None) is not None and self._b.value:
            load_library().afqmc_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


CONTRACT_KERNELS = {0: "contract_fp64_kernel", 1: "contract_tc_kernel", 2: "contract_tcy_kernel",
                    3: "contract_fp64z_kernel", 4: "contract_fp64r_kernel", 5: "contract_tcw_kernel",
                    6: "contract_fp64c_kernel"}


def contract_kernel(cfg: AfqmcConfig) -> str:
    """Name of the kernel that runs the fused contraction for ``cfg``."""
    k = int(load_library().afqmc_contract_kernel(ctypes.byref(cfg)))
    if k not in CONTRACT_KERNELS:
        raise AfqmcError(1, "no contraction kernel supports these sizes")
    return CONTRACT_KERNELS[k]


def fp64_fma_rate(stream=None) -> float:
    """Measured FP64 FMA throughput of the current GPU in TFLOP/s."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    v = ctypes.c_double()
    _check(load_library().afqmc_fp64_fma_rate(ctypes.byref(v), s.cuda_stream))
    return v.value


def launch_count() -> int:
    """Kernels launched by the library in this process so far."""
    return int(load_library().afqmc_launch_count())


def unpack_state(blob: bytes) -> dict:
    """Split a state buffer (layout in include/afqmc.h) into numpy arrays."""
    hdr = struct.unpack_from("<8Q", blob, 0)
    if hdr[0] != STATE_MAGIC:
        raise ValueError("not an afqmc state buffer")
    N, nu, nd, K, W, P, step = hdr[1:]
    nt = nu + nd
    o = 64
    def take(count, dtype):
        nonlocal o
        a = np.frombuffer(blob, dtype=dtype, count=count, offset=o).copy()
        o += a.nbytes
        return a
    phi = take(W * N * nt, np.complex128).reshape(W, N, nt)
    weight = take(W, np.float64)
    x = take(W * P * K, np.float64).reshape(W, P, K)
    # real trial orbitals, or complex ones (complex or multi-slice trials): the rest of the buffer says which
    cplx = len(blob) - o == W * P * N * nu * 16
    Phi = take(W * P * N * nu, np.complex128 if cplx else np.float64).reshape(W, P, N, nu)
    return dict(step=int(step), phi_up=phi[:, :, :nu].copy(), phi_dn=phi[:, :, nu:].copy(), weight=weight, x=x, Phi=Phi)


def pack_state(st: dict) -> bytes:
    W, N, nu = st["phi_up"].shape
    nd = st["phi_dn"].shape[2]
    P, K = st["x"].shape[1:]
    phi = np.concatenate([st["phi_up"], st["phi_dn"]], axis=2).astype(np.complex128)
    hdr = struct.pack("<8Q", STATE_MAGIC, N, nu, nd, K, W, P, int(st["step"]))
    return b"".join([hdr, np.ascontiguousarray(phi).tobytes(), np.ascontiguousarray(st["weight"], np.float64).tobytes(),
                     np.ascontiguousarray(st["x"], np.float64).tobytes(),
                     np.ascontiguousarray(st["Phi"], np.complex128 if np.iscomplexobj(st["Phi"]) else np.float64)
                     .tobytes()])


def philox_fill(out, n: int, c0: int, c1: int, c2: int, c3: int, key: int, stream=None):
    """Fill the device uint32 tensor ``out`` (4n words) with the library's Philox4x32-10."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    _check(load_library().afqmc_philox_fill(out.data_ptr(), int(n), c0, c1, c2, c3, int(key), s.cuda_stream))
