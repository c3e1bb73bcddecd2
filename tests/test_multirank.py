"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
GPU in a real run) each step an independent replica with its own seed, the
job time is the slowest rank's and the value counts every rank's spheres.
No data-path collective exists; the only one is the max over ranks of the
timed region."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 10.0 + 5.0 * rank                 # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    q.put((rank, bench.rank_seed(2003, rank), ms_max,
           bench.job_value(world, 1_000_000, 100 * 20, ms_max)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_the_slowest_and_count_all_spheres():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    # each child imports torch first, which can take minutes on a cold,
    # loaded machine
    out = sorted(q.get(timeout=600) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, s0, m0, v0), (r1, s1, m1, v1) = out
    assert (r0, r1) == (0, 1)
    assert s0 != s1                          # independent replicas
    assert m0 == m1 == 15.0                  # the slowest rank's time
    assert v0 == v1 == 2 * 1_000_000 * 2000 / 0.015
