"""Multi-rank host logic on CPU with gloo, world_size 2: the max-over-ranks
timing used by the benchmark and the patch sharding (each patch on exactly
one rank, loads balanced)."""
import os
import socket

import pytest

from paper_1410_1764_gb300 import dist, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as tdist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, lr = dist.world()
    dist.barrier()
    m = dist.max_over_ranks(10.0 + 5.0 * rank)
    dims = synth.patch_dims(3)
    mine = dist.shard_patches(dims, ws)[r]
    q.put((r, ws, lr, m, mine))
    tdist.destroy_process_group()


def test_two_rank_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 15.0 for r in res)  # the max of 10 and 15 on both ranks
    allp = sorted(res[0][4] + res[1][4])
    assert allp == list(range(64))


def test_shard_balance():
    dims = synth.patch_dims(3)
    for n in (1, 2, 3, 8):
        sh = dist.shard_patches(dims, n)
        assert sorted(p for s in sh for p in s) == list(range(len(dims)))
        cost = [sum(int(a) * int(b) * int(c) for a, b, c in (dims[p] for p in s)) for s in sh]
        assert max(cost) <= 1.1 * sum(cost) / n + max(int(a) * int(b) * int(c) for a, b, c in dims)


def test_single_process_max():
    assert dist.max_over_ranks(3.5) == 3.5
