"""Multi-process (gloo, world size 2, CPU) checks of the replica logic that the
benchmark uses when it runs one process per GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1204_4293_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, lr = replicas.world_info()
    t = replicas.max_over_ranks(1.5 + rank)
    seed = replicas.rank_seed(7, r)
    shard = list(replicas.shard_maps(17, w, r))
    dist.barrier()
    out.put((rank, w, r, lr, t, seed, shard))
    dist.destroy_process_group()


def test_two_rank_max_and_shards():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, _, _, t0, s0, sh0), (r1, w1, _, _, t1, s1, sh1) = res
    assert w0 == w1 == 2
    assert t0 == t1 == pytest.approx(2.5)  # max over ranks
    assert s0 != s1
    assert sh0 + sh1 == list(range(17)) and abs(len(sh0) - len(sh1)) <= 1


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.weak_scaling_value(10.0, 4, 2.0) == 20.0
    assert list(replicas.shard_maps(5, 1, 0)) == list(range(5))
