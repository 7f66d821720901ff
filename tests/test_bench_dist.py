"""The multi-process path of bench.py on CPU (gloo, world size 2): ranks
solve independent instances, the only exchange is the max of their step
times, the whole-job value divides it by the number of instances, and the
reference arm runs on rank 0 alone."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    dist = bench.init_dist(torch.device("cpu"))
    local_ms = 10.0 * (r + 1)
    job_ms = bench.max_over_ranks(local_ms, torch.device("cpu"))
    value = bench.whole_job_ms(job_ms / 1, w)

    class A:
        n = 8
        steps = 1
        warmup = 0
    ref = bench.run_reference(A(), r, w) if r != 0 else "rank0-skipped"
    dist.barrier()
    dist.destroy_process_group()
    q.put((r, w, local, job_ms, value, ref))


def test_two_rank_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, w, local, job_ms, value, ref = q.get(timeout=120)
        out[r] = (w, local, job_ms, value, ref)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        w, local, job_ms, value, _ = out[r]
        assert w == 2 and local == r
        assert job_ms == 20.0          # the slower rank's time
        assert value == 10.0           # two instances solved in 20 ms
    assert out[1][4] is None           # the reference arm does no work off rank 0
