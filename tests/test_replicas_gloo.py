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
    # realisations split over ranks: each rank's partial sums (here the
    # realisation indices it owns, per element) add up to the whole range's
    import torch
    own = replicas.noise_range(10, w, r)
    sums = torch.full((2, 3, 4, 4), float(sum(own)), dtype=torch.float64)
    sums = replicas.merge_noise_sums(sums)
    dist.barrier()
    out.put((rank, w, r, lr, t, seed, shard, float(sums.min()), float(sums.max()), list(own)))
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
    (r0, w0, _, _, t0, s0, sh0, lo0, hi0, own0), (r1, w1, _, _, t1, s1, sh1, lo1, hi1, own1) = res
    assert own0 + own1 == list(range(10))  # disjoint realisation ranges covering all
    assert lo0 == hi0 == lo1 == hi1 == float(sum(range(10)))  # merged sums
    assert w0 == w1 == 2
    assert t0 == t1 == pytest.approx(2.5)  # max over ranks
    assert s0 != s1
    assert sh0 + sh1 == list(range(17)) and abs(len(sh0) - len(sh1)) <= 1


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.weak_scaling_value(10.0, 4, 2.0) == 20.0
    assert list(replicas.shard_maps(5, 1, 0)) == list(range(5))
    import torch
    t = torch.ones(2, 1, 2, 2, dtype=torch.float64)
    assert replicas.merge_noise_sums(t) is t and float(t.sum()) == 8.0
