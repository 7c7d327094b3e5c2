"""GB300 (sm_103a) library for phaseless AFQMC with a stochastically sampled
trial wave function: CUDA kernels behind the C ABI in include/afqmc.h, with a
thin ctypes binding (``paper_2505_18519_gb300.afqmc``)."""

from .afqmc import (AfqmcConfig, AfqmcError, Context, load_library, make_config, pack_state, philox_fill,  # noqa: F401
                    unpack_state, workspace_bytes)
