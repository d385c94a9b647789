"""The multi-GPU launch of bench.py on CPU ranks (gloo, world size 2).

The method runs as independent replicas, one box per rank, with no
collective on the data path; what crosses ranks is the job's time (the
slowest rank's, agreed by a max-reduce after a barrier) and the aggregate
rate over all ranks' replicas.  The reference arm runs on rank 0 alone: the
other ranks exit without work.
"""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, root, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, root)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")   # rank 1 is slower
    dist.barrier()
    q.put((rank, ms, bench.whole_job_mlups(1000, 10, world, ms)))
    dist.destroy_process_group()


def test_replicas_report_the_slowest_rank_and_the_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, ROOT, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(ms == 15.0 for _, ms, _ in res)              # both ranks agree on the max
    # 2 replicas x 1000 cells x 10 steps in 15 ms
    assert res[0][2] == pytest.approx(2 * 1000 * 10 / 0.015 / 1e6)
    assert res[0][2] == res[1][2]


def test_one_rank_is_the_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_mlups(2 ** 24, 100, 1, 1000.0) == pytest.approx(2 ** 24 * 100 / 1e6)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""
