"""Sharding over ranks: LPT partition and the end-of-mining gather, run as two
gloo ranks on CPU (the per-rank miner here is the oracle; on GPUs it is the
CUDA path, which needs no collective)."""
import os
import socket

import numpy as np
import pytest

from paper_1512_01641_gb300 import shard, synth


def test_lpt_covers_every_pair_once_and_balances():
    rng = np.random.default_rng(0)
    cost = np.concatenate([rng.lognormal(8, 1.5, size=997), [2.5e7] * 3])
    for world in (1, 2, 3, 8):
        parts = shard.lpt_partition(cost, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(cost)))
        loads = np.array([cost[p].sum() for p in parts])
        lower = max(cost.sum() / world, cost.max())
        assert loads.max() <= 4 / 3 * lower + 1e-6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        batch = synth.make_batch(41, 23, v_src=800, v_tgt=800, size_median=12, size_hi=60)
        idx, sub = shard.shard_of(batch, rank, world)
        r = oracle.mine(sub, [4, 4, -2, 1], -3.0, 0.3, 0.5, n_threads=1)
        links = [[(i, j) for i, j, _ in l] for l in r["links"]]
        res = shard.gather_results(idx, r["score"], links)
        if rank == 0:
            full = oracle.mine(batch, [4, 4, -2, 1], -3.0, 0.3, 0.5, n_threads=1)
            ok = (np.allclose(res[0], full["score"], rtol=0, atol=0) and
                  res[1] == [[(i, j) for i, j, _ in l] for l in full["links"]])
            q.put(bool(ok))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_mine_shards_and_gather():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    assert q.get(timeout=5) is True
