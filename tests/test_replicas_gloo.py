"""The multi-GPU form is replicas: every rank simulates its own event (no collective on
the data path) and the job's throughput is the deposits of all ranks over the slowest
rank's time.  Here the host side of that path runs as two gloo ranks on the CPU."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import synth
    cfg = synth.get_config("tiny")
    dep = synth.make_deposits(cfg, seed=bench.replica_seed(cfg, rank))
    n = len(dep["x"])
    ms = 10.0 + 5.0 * rank                     # the slower rank sets the job's time
    n_job, ms_job = bench.aggregate_replicas(n, ms, world)
    q.put((rank, n, n_job, ms_job, float(np.sum(dep["x"]))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_sum_deposits_and_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, n0, job0, ms0, x0), (r1, n1, job1, ms1, x1) = res
    assert (r0, r1) == (0, 1)
    assert job0 == job1 == n0 + n1
    assert ms0 == ms1 == 15.0
    assert x0 != x1                            # each rank draws its own event


def test_one_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(123, 4.5, 1) == (123.0, 4.5)
