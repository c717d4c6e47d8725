"""Replicas across processes (the multi-GPU path shards by whole jobs): two
gloo ranks on the CPU combine their timings and work the way bench.py does
on NCCL -- job time is the slowest rank's, work is summed -- and every rank
runs a different, reproducible circuit."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    from paper_2501_13237_gb300 import replicas
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, units = replicas.aggregate(10.0 * (rank + 1), 100.0 + rank, dist, "cpu")
        out.put((rank, ms, units, replicas.replica_seed(rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_time_and_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, seed in res:
        assert ms == 20.0                 # the slowest rank
        assert units == 201.0             # both ranks' work
        assert seed == rank
    assert res[0][3] != res[1][3]


def test_single_process_is_identity():
    from paper_2501_13237_gb300 import replicas
    assert replicas.aggregate(3.5, 7.0) == (3.5, 7.0)


def test_rank_workloads_differ_and_repeat():
    import workloads as wl
    from paper_2501_13237_gb300 import replicas
    a0 = wl.brickwork_circuit(8, 4, replicas.replica_seed(0))
    a1 = wl.brickwork_circuit(8, 4, replicas.replica_seed(1))
    b0 = wl.brickwork_circuit(8, 4, replicas.replica_seed(0))
    assert not np.allclose(a0.unitaries[0], a1.unitaries[0])
    assert np.array_equal(a0.unitaries[0], b0.unitaries[0])
