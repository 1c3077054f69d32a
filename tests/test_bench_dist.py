"""The N > 1 launch of bench.py (replicas, one process per GPU) on CPU: two gloo ranks rendezvous at
127.0.0.1, pass the barrier, and agree on the maximum of their step times (the max over ranks that
the bench's whole-job value divides by)."""

import multiprocessing as mp
import os
import socket


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      HHG_BENCH_GLOO="1")
    import bench
    r, w = bench.dist_init(2)
    bench.barrier(w)
    q.put((r, w, bench.allmax(1.5 + r, w)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_gloo_two_ranks_barrier_and_max_over_ranks():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 2, 2.5), (1, 2, 2.5)]
