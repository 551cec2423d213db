"""World-size-2 gloo test of the multi-GPU replica bookkeeping (CPU only)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_1008_5113_gb300 import replicas

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = replicas.walker_seeds(rank, 4)
        count, elapsed = replicas.reduce_run(count=1000 * (rank + 1), elapsed=[2.0, 3.5][rank])
        out[rank] = (seeds, count, elapsed, replicas.throughput(count, elapsed))
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_over_two_gloo_ranks():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:  # no fork of a multi-threaded process
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    (s0, c0, t0, v0), (s1, c1, t1, v1) = res[0], res[1]
    assert s0 == [1, 2, 3, 4] and s1 == [5, 6, 7, 8]      # disjoint, rank 0 = single-GPU seeds
    assert c0 == c1 == 3000.0 and t0 == t1 == 3.5          # sum of counts, max of times
    assert v0 == v1 == pytest.approx(3000.0 / 3.5)


def test_single_process_is_identity():
    from paper_1008_5113_gb300 import replicas

    assert replicas.reduce_run(7, 1.5) == (7.0, 1.5)
    with pytest.raises(ValueError):
        replicas.walker_seeds(-1, 4)
