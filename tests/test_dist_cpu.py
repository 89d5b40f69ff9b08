"""Multi-rank host logic on CPU with gloo, world_size 2: the max-over-ranks
timing used by the benchmark and the patch sharding (each patch on exactly
one rank, loads balanced)."""
import os
import socket

import numpy as np
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


def _xy_periodic(a, g):
    """Periodic x/y ghosts of a padded array (test-side numpy)."""
    nx, ny = a.shape[-1] - 2 * g, a.shape[-2] - 2 * g
    ix = (np.arange(nx + 2 * g) - g) % nx + g
    iy = (np.arange(ny + 2 * g) - g) % ny + g
    return a[..., iy, :][..., ix]


def _slab_worker(rank, world, port, q):
    import torch
    import torch.distributed as tdist
    from paper_1410_1764_gb300 import slabs
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    g, (nx, ny, nz) = 2, (6, 5, 11)
    rng = np.random.default_rng(0)  # same global data on every rank
    glob = synth.pad(rng.standard_normal((2, nz, ny, nx)), g)
    full = glob.copy()
    oracle.fill_ghosts(full, g)
    z0, n = slabs.zslabs(nz, world)[rank]
    mine = np.zeros((2, n + 2 * g, ny + 2 * g, nx + 2 * g))
    mine[:, g:g + n] = glob[:, g + z0:g + z0 + n]
    t = torch.from_numpy(mine)
    slabs.DistExchange(g, rank, world)([t])
    got = _xy_periodic(t.numpy(), g)
    ok_fill = np.array_equal(got, full[:, z0:z0 + n + 2 * g])
    h = 0.1
    r_slab = oracle.wave_rhs(np.ascontiguousarray(got), g, h)[:, g:g + n, g:-g, g:-g]
    r_full = oracle.wave_rhs(full, g, h)[:, g + z0:g + z0 + n, g:-g, g:-g]
    q.put((rank, ok_fill, float(np.abs(r_slab - r_full).max())))
    tdist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_zslab_halo_exchange_gloo(world):
    """Ranks exchange z halos point to point; with periodic x/y filled, each
    slab's padded state equals the window of the periodic global state and
    its RHS equals the global RHS on its z range (bit for bit)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_slab_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=180) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert all(ok for _, ok, _ in res), res
    assert all(e == 0.0 for _, _, e in res), res


def test_zslabs_partition():
    from paper_1410_1764_gb300 import slabs
    assert slabs.zslabs(11, 3) == [(0, 4), (4, 4), (8, 3)]
    for nz, p in ((128, 8), (17, 5), (5, 5)):
        s = slabs.zslabs(nz, p)
        assert sum(n for _, n in s) == nz and s[0][0] == 0
        assert all(s[i][0] + s[i][1] == s[i + 1][0] for i in range(p - 1))
    with pytest.raises(ValueError):
        slabs.zslabs(3, 4)


def test_checkpoint_round_trip(tmp_path):
    """save_checkpoint / load_checkpoint keep the state bit for bit with its
    time, step and metadata (resume from a checkpoint)."""
    import torch
    from paper_1410_1764_gb300 import api
    x = torch.from_numpy(np.random.default_rng(0).standard_normal((2, 6, 7, 8)))
    p = tmp_path / "ck.pt"
    api.save_checkpoint(p, x, t=0.125, step=17, kind="wave", dx=0.01)
    y, t, step, meta = api.load_checkpoint(p)
    assert torch.equal(x, y) and t == 0.125 and step == 17 and meta == {"kind": "wave", "dx": 0.01}
