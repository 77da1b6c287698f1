"""The multi-GPU path of bench.py is replicas only (independent solves, no
data-path collective): the whole-job rate is every rank's solves over the
slowest rank's time.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    r, w, dist = bench.dist_init(world, backend="gloo")
    assert (r, w) == (rank, world)
    rate, tmax = bench.replica_rate(1000.0 * (rank + 1), 5, w, dist, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, tmax))


def test_replica_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # rank 1 took 2000 ms: 2 ranks x 5 solves / 2 s = 5 solves/s on every rank
    assert [o[2] for o in out] == [2000.0, 2000.0]
    assert all(abs(o[1] - 5.0) < 1e-12 for o in out)


def test_single_process_needs_no_collective():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    env = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE") if k in os.environ}
    try:
        assert bench.dist_init(1) == (0, 1, None)
        assert bench.replica_rate(500.0, 5, 1, None) == (10.0, 500.0)
    finally:
        os.environ.update(env)
