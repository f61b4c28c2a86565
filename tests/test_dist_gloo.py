"""The multi-process parts of bench.py on CPU with the gloo backend
(world size 2): the MAX reduction of the timed region, the barrier, and the
reference arm running on rank 0 only.  The data path itself has no
collective: each rank reconstructs its own sweep (replicas)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, local, w = bench.init_dist("gloo")
    bench.barrier()
    m = bench.max_over_ranks(10.0 * (rank + 1))
    # rank != 0 of the reference arm exits without work
    rc = bench.run_reference(bench.parse_args(["--impl", "reference", "--steps", "1",
                                               "--warmup", "0"])) if rank == 1 else 0
    q.put((rank, r, w, m, rc))
    dist.destroy_process_group()


def test_two_rank_max_and_barrier():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert [x[0] for x in res] == [0, 1]
    assert all(x[2] == 2 for x in res)
    assert all(x[3] == 20.0 for x in res)
    assert all(x[4] == 0 for x in res)


def test_single_process_reduction_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
