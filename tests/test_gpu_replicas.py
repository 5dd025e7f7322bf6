"""Replica parallelism through the product: two gloo ranks (processes), each
with its own copy of the model, simulate their shards of the sources with
the batched solver (es_run) and superpose their own events (es_superpose);
the summed partial gathers equal one process's superposition of all events
and the oracle's superposition of the same traces (Sec. III-A: sources on
separate GPUs; Sec. IV: superposition).  Both ranks share the one GPU of this
run; their kernels never wait on one another."""
import os
import socket

import numpy as np
import pytest

from paper_1705_04874_gb300 import replicas, synth

pytestmark = pytest.mark.gpu

SHAPE = (32, 32, 48)
NT, PML, N_SRC, N_EV, N_OUT = 150, 4, 7, 60, 260


def _problem():
    rho, cp, cs = synth.marine_model(shape=SHAPE, seed=9)
    dt = 0.3 * 10.0 / float(np.max(cp))  # Eq. (5), CFL 0.3
    rng = synth.SplitMix64(31)
    pos = synth.random_positions(rng, synth.reservoir_box(SHAPE, PML), N_SRC)
    mts = np.array([synth.random_dc(rng) for _ in range(N_SRC)])
    wav = np.stack([synth.ricker(NT, dt, 30.0)] * N_SRC)
    ev, amps, t0s = synth.events(rng, N_EV, N_SRC, t_span=0.05)
    return rho, cp, cs, dt, pos, mts, wav, ev, amps, t0s


def _simulate(es, rho, cp, cs, dt, pos, mts, wav):
    with es.Model(rho, cp, cs, dx=10.0, pml=PML) as m:
        rcv = m.seabed_receivers(3, 3)
        m.batch_set(pos, mts, wav)
        tr = m.run(NT, dt, rcv)
    return tr.reshape((len(pos),) + tr.shape[-3:])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_q):
    import torch
    import torch.distributed as dist
    from paper_1705_04874_gb300 import es
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    rho, cp, cs, dt, pos, mts, wav, ev, amps, t0s = _problem()
    mine = replicas.shard(N_SRC, world, rank)
    tr = _simulate(es, rho, cp, cs, dt, pos[mine.start:mine.stop], mts[mine.start:mine.stop],
                   wav[mine.start:mine.stop])
    sel, local = replicas.events_of_rank(ev, mine)
    part = es.es_superpose(tr, local, amps[sel], t0s[sel], dt, N_OUT)
    full = replicas.merge_gathers(dist, part)
    blocks = [None] * world
    dist.all_gather_object(blocks, tr)
    n = replicas.sum_over_ranks(dist, float(len(mine)))
    if rank == 0:
        out_q.put((full, np.concatenate(blocks), n))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_run_and_superpose_through_the_product(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import torch.multiprocessing as mp
    from paper_1705_04874_gb300 import es
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    full, traces, n = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert n == N_SRC
    rho, cp, cs, dt, pos, mts, wav, ev, amps, t0s = _problem()
    one = _simulate(es, rho, cp, cs, dt, pos, mts, wav)
    assert np.array_equal(traces, one)  # shards of a batch = the whole batch, bit for bit
    single = es.es_superpose(one, ev, amps, t0s, dt, N_OUT)
    scale = np.abs(single).max()
    assert scale > 0
    assert np.abs(full - single).max() <= 1e-6 * scale
    ref = orc.superpose(one.astype(np.float64), ev, amps.astype(np.float64), t0s.astype(np.float64), dt, N_OUT)
    assert np.abs(full - ref).max() <= 1e-5 * np.abs(ref).max()
