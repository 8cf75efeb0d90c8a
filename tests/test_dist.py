"""The N > 1 path of bench.py on CPU with the gloo backend (world size 2): the job's step time
is the largest over the ranks, and the aggregate throughput counts every rank's work
(replicas: each rank runs the whole workload, weak scaling)."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    step_ms = 3.0 + rank            # rank 1 is the slower one
    m = bench.max_over_ranks(step_ms, world, "cpu")
    q.put((rank, m, world * 1e9 / (m * 1e-3)))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo_world_size_2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [m for _, m, _ in out] == [4.0, 4.0]
    assert all(abs(v - 2 * 1e9 / 4e-3) < 1e-3 for _, _, v in out)


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
