"""Two CPU ranks (gloo) each run the oracle on their block of walkers; the
summed mixed-estimator sums equal those of one process running all walkers,
step by step, because every random draw is addressed by the global walker
index."""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import afqmc_inputs as ai
from oracle import afqmc as oa
from paper_2505_18519_gb300.sharding import combine_mixed, combine_paths, max_over_ranks, shard

W, P, STEPS = 10, 4, 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _setup():
    spec = ai.SystemSpec(8, 4, 4, 12, 5, False, 1000)
    s = ai.make_system(spec)
    ham = oa.prepare(s.h, s.L, s.Phi0, s.U, 4, 4, 0.01)
    cfg = oa.OracleConfig(dtau=0.01, n_walkers=W, n_paths=P, seed=77, n_burn=2)
    return ham, cfg


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ham, cfg = _setup()
    off, cnt = shard(W, world, rank)
    st = oa.init(ham, cfg, walker_index=np.arange(off, off + cnt))
    out = []
    for _ in range(STEPS):
        st, d = oa.step(ham, cfg, st)
        num, den = d["mixed"]
        out.append(combine_mixed((num, den, 0.0)))
    # extra measurement paths on each rank's walkers: their chains are addressed by the
    # global pair index too, so the combined estimate is the single process's
    r = oa.measure_paths(ham, cfg, st, rounds=2, sweeps=1)
    R = np.where(r["alive"], r["R"], 0.0)
    e_paths = combine_paths(st.weight, np.where(r["alive"], r["e_walker"], 0.0), R)
    slowest = max_over_ranks(float(rank + 1))
    if rank == 0:
        q.put((out, e_paths, slowest))
    dist.destroy_process_group()


def test_shard_blocks_cover_population():
    for total, world in ((10, 2), (11, 3), (512, 8), (3, 4)):
        blocks = [shard(total, world, r) for r in range(world)]
        assert sum(c for _, c in blocks) == total
        assert all(blocks[r][0] + blocks[r][1] == blocks[r + 1][0] for r in range(world - 1))


def test_two_gloo_ranks_reproduce_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out, e_paths, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ham, cfg = _setup()
    st = oa.init(ham, cfg)
    for k in range(STEPS):
        st, d = oa.step(ham, cfg, st)
        num, den = d["mixed"]
        e_mix, sum_w, _ = out[k]
        assert abs(e_mix - num / den) < 1e-12 * abs(num / den)
        assert abs(sum_w - den) < 1e-12 * den
    ref = oa.measure_paths(ham, cfg, st, rounds=2, sweeps=1)["e_mix"]
    assert abs(e_paths - ref) < 1e-12 * abs(ref)
    assert slowest == 2.0
