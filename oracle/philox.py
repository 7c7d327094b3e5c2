"""Counter-based random numbers for the oracle: Philox4x32-10.

ORACLE / TEST INFRASTRUCTURE ONLY: only tests, the smoke check and the CPU
baseline leg of the benchmark may import this package.  The CUDA library has
its own, separately written generator; the two must agree bit for bit.

Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4 x 32-bit counter and a 2 x 32-bit
key go through ten rounds; each round multiplies counter words 0 and 2 by two
fixed odd constants, forms the 64-bit products' high and low halves, and
recombines them with words 1 and 3 and the round key by exclusive-or; the key is
advanced by two Weyl constants between rounds.

Stream layout shared with the CUDA side (the paper only says that the fields
and the Metropolis proposals are Gaussian draws, Eq. (4) and Sec. III A; the
layout is this code's own):
    key     = (seed mod 2^32, seed >> 32)
    counter = (block, entity, step, (tag << 24) | sweep)
where ``entity`` is a walker index (fields, initial walkers) or a pair index
w * P + p (paths, proposals, accept/reject draws) and ``block`` numbers the
successive 4-word outputs of one draw.  Each block gives two doubles with 53
random bits: u0 from words (0, 1), u1 from words (2, 3), as
(w_hi * 2^21 + (w_lo >> 11)) * 2^-53 in [0, 1).  Normal deviates use the
Box-Muller transform of one block: r = sqrt(-2 ln(1 - u0)), z0 = r cos(2 pi u1),
z1 = r sin(2 pi u1), so normal number 2j and 2j+1 of a draw come from block j.
"""

from __future__ import annotations

import numpy as np

__all__ = ["philox4x32_10", "uniforms", "normals", "TAG_INIT_WALKER", "TAG_INIT_PATH",
           "TAG_FIELD", "TAG_PROPOSE", "TAG_ACCEPT", "TAG_BURN_PROPOSE", "TAG_BURN_ACCEPT", "TAG_COMB",
           "TAG_MEAS_PROPOSE", "TAG_MEAS_ACCEPT"]

TAG_INIT_WALKER = 1
TAG_INIT_PATH = 2
TAG_FIELD = 3
TAG_PROPOSE = 4
TAG_ACCEPT = 5
TAG_BURN_PROPOSE = 6
TAG_BURN_ACCEPT = 7
TAG_COMB = 10          # one uniform per population-control comb, entity = first walker's index
TAG_MEAS_PROPOSE = 11  # measurement-only Metropolis sweeps (extra paths of the mixed estimate)
TAG_MEAS_ACCEPT = 12

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter: np.ndarray, key) -> np.ndarray:
    """Apply ten Philox4x32 rounds to ``counter`` (shape (..., 4), uint32)."""
    c = np.asarray(counter, dtype=np.uint32)
    c0, c1, c2, c3 = (c[..., i].astype(np.uint64) for i in range(4))
    k0 = np.uint32(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint32(int(key[1]) & 0xFFFFFFFF)
    for r in range(10):
        if r > 0:
            k0 = np.uint32((int(k0) + int(_W0)) & 0xFFFFFFFF)
            k1 = np.uint32((int(k1) + int(_W1)) & 0xFFFFFFFF)
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        n0 = hi1 ^ c1 ^ np.uint64(k0)
        n2 = hi0 ^ c3 ^ np.uint64(k1)
        c0, c1, c2, c3 = n0, lo1, n2, lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _blocks(seed: int, tag: int, step: int, entities, sweep: int, nblocks: int) -> np.ndarray:
    ent = np.asarray(entities, dtype=np.uint64).reshape(-1)
    ctr = np.empty((ent.size, nblocks, 4), dtype=np.uint32)
    ctr[..., 0] = np.arange(nblocks, dtype=np.uint32)[None, :]
    ctr[..., 1] = (ent & _MASK).astype(np.uint32)[:, None]
    ctr[..., 2] = np.uint32(step & 0xFFFFFFFF)
    ctr[..., 3] = np.uint32(((tag & 0xFF) << 24) | (sweep & 0xFFFFFF))
    key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    return philox4x32_10(ctr, key)


def _u53(hi: np.ndarray, lo: np.ndarray) -> np.ndarray:
    v = (hi.astype(np.uint64) << np.uint64(21)) | (lo.astype(np.uint64) >> np.uint64(11))
    return v.astype(np.float64) * (2.0 ** -53)


def uniforms(seed: int, tag: int, step: int, entities, sweep: int, count: int) -> np.ndarray:
    """(len(entities), count) uniforms in [0, 1); number 2j, 2j+1 from block j."""
    nb = (count + 1) // 2
    w = _blocks(seed, tag, step, entities, sweep, nb)
    u = np.stack([_u53(w[..., 0], w[..., 1]), _u53(w[..., 2], w[..., 3])], axis=-1)
    return u.reshape(w.shape[0], 2 * nb)[:, :count]


def normals(seed: int, tag: int, step: int, entities, sweep: int, count: int) -> np.ndarray:
    """(len(entities), count) standard normal deviates by Box-Muller."""
    nb = (count + 1) // 2
    w = _blocks(seed, tag, step, entities, sweep, nb)
    u0 = _u53(w[..., 0], w[..., 1])
    u1 = _u53(w[..., 2], w[..., 3])
    r = np.sqrt(-2.0 * np.log1p(-u0))
    t = 2.0 * np.pi * u1
    z = np.stack([r * np.cos(t), r * np.sin(t)], axis=-1)
    return z.reshape(w.shape[0], 2 * nb)[:, :count]
