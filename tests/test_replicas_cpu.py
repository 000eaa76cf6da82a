"""Multi-rank (replica) path of bench.py on CPU: two gloo ranks, each with its
own range of sample ids; together they must give exactly the samples of one
process over the union of the ranges (counter-based draws, Alg. 1), and the
timing reduction must take the slowest rank. The GPU kernel reproduces the
oracle's samples bit for bit (the -m gpu parity tests), so the oracle stands
in for it here."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import workloads as W
from oracle import circuit as OC
from oracle import sampler as OS

N_SAMPLES, WARMUP, STEPS = 6, 1, 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spec = W.random_qaoa(6, 2, seed=91)
    ops = OC.qaoa_circuit(spec)
    first = bench.replica_first(rank, N_SAMPLES, WARMUP, STEPS)
    ids = [first + i for i in range((WARMUP + STEPS) * N_SAMPLES)]
    bits, _ = OS.sample_sv(spec.n, ops, 5, ids)
    slowest = bench.max_over_ranks(10.0 + rank, world)
    got = [None] * world
    dist.all_gather_object(got, (ids, np.asarray(bits).tolist(), slowest))
    if rank == 0:
        q.put(got)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_match_one_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ids0, bits0, slow0 = got[0]
    ids1, bits1, slow1 = got[1]
    assert not set(ids0) & set(ids1)                 # disjoint sample ranges
    assert slow0 == slow1 == 11.0                    # max over ranks
    spec = W.random_qaoa(6, 2, seed=91)
    ops = OC.qaoa_circuit(spec)
    ref, _ = OS.sample_sv(spec.n, ops, 5, ids0 + ids1)
    assert np.array_equal(np.asarray(bits0 + bits1), np.asarray(ref))


def test_replica_ranges_are_disjoint_for_any_world():
    for world in (2, 4, 8):
        spans = [(bench.replica_first(r, 100, 3, 5), bench.replica_first(r, 100, 3, 5) + 100 * 9) for r in range(world)]
        for a in range(world):
            for b in range(a + 1, world):
                assert spans[a][1] <= spans[b][0]
