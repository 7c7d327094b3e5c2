"""CPU oracle (test infrastructure only).

A plain, slow, FP64 numpy implementation of the sampled-trial phaseless AFQMC
step and of its counter-based random numbers.  Only ``tests/``, the smoke check
and the CPU-baseline leg of ``bench.py`` may import it; the CUDA library never
does, and the two share no code.
"""
from . import philox, afqmc, mlp  # noqa: F401
