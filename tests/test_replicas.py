"""Replica parallelism on CPU with two gloo ranks: sources are sharded with
no overlap or gap, the max-over-ranks timing and the sum of partial
superposition gathers (each rank superposes the events of its own sources,
Sec. IV) reproduce the single-process results."""
import os
import socket

import numpy as np
import pytest

from paper_1705_04874_gb300 import replicas, synth


def test_shard_covers_every_item_once():
    for n in (0, 1, 7, 64, 301):
        for world in (1, 2, 3, 8):
            got = [list(replicas.shard(n, world, r)) for r in range(world)]
            assert sum(got, []) == list(range(n))
            sizes = [len(g) for g in got]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(5, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, tr, ev, amps, t0s, dt, n_out, out_q):
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = replicas.shard(tr.shape[0], world, rank)
    sel, local = replicas.events_of_rank(ev, mine)
    part = oracle.superpose(tr[mine.start:mine.stop], local, amps[sel], t0s[sel], dt, n_out) \
        if len(mine) else np.zeros((4, tr.shape[2], n_out))
    full = replicas.merge_gathers(dist, part.astype(np.float32))
    t = replicas.max_over_ranks(dist, 1.5 + rank)
    total = replicas.sum_over_ranks(dist, float(len(mine)))
    if rank == 0:
        out_q.put((full, t, total))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_merge_superposition(world, orc):
    import torch.multiprocessing as mp
    rng = synth.SplitMix64(8)
    tr = rng.normal(7 * 4 * 3 * 60).reshape(7, 4, 3, 60)
    ev, amps, t0s = synth.events(rng, 40, 7, t_span=0.05)
    amps, t0s = amps.astype(np.float64), t0s.astype(np.float64)
    dt, n_out = 1e-3, 120
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, tr, ev, amps, t0s, dt, n_out, q)) for r in range(world)]
    for p in procs:
        p.start()
    full, t, total = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = orc.superpose(tr, ev, amps, t0s, dt, n_out)
    assert np.abs(full - ref).max() <= 1e-5 * np.abs(ref).max()
    assert t == 1.5 + world - 1
    assert total == 7.0
