"""bench.py's multi-rank helpers at world size 2 over gloo on the CPU.  On GPUs
the same helpers run under torchrun with NCCL, one replica per GPU: a barrier
on both sides of the timed region and the maximum of the ranks' times."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, loc = bench._dist_setup()
        assert (w, r, loc) == (world, rank, rank)
        bench._barrier(w)
        out[rank] = (bench._max_over_ranks(w, 1.5 + rank), bench._sum_over_ranks(w, 1.5 + rank))
        bench._barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_ranks_barrier_and_max_over_ranks():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert dict(out) == {0: (2.5, 4.0), 1: (2.5, 4.0)}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench._max_over_ranks(1, 3.25) == 3.25
    bench._barrier(1)


def test_batched_problems_shard_over_ranks():
    """The batch's independent problems are dealt out over the ranks: every
    problem once, cell counts balanced to within the longest problem."""
    from paper_1909_08390_gb300 import workloads as W
    nx = [q["nx"] for q in W.batched_problems(0)]
    for world in (1, 2, 3, 4, 8):
        shards = [W.shard_problems(nx, r, world) for r in range(world)]
        flat = sorted(i for sh in shards for i in sh)
        assert flat == list(range(len(nx)))
        cells = [sum(nx[i] for i in sh) for sh in shards]
        assert max(cells) - min(cells) <= max(nx)
