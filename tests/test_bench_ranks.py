"""The benchmark's multi-rank host logic on CPU with the gloo backend (world size 2): the
barrier, the maximum over ranks that sets the job's time, the whole-job throughput, and the
reference arm's non-zero ranks leaving without work.  The GPU work of each rank is an
independent replica (no collective on the data path), so the host logic is all that the
ranks share."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.rank_barrier(world)
        slowest = bench.max_over_ranks(times[rank], world, "cpu")
        bench.rank_barrier(world)
        q.put((rank, slowest, bench.job_rate(world, 1, 10, slowest)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed not available")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.25, 2.5]                        # rank 1 is the slower one
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the job advanced 2 x 10 steps in it
    assert [o[1] for o in out] == [2.5, 2.5]
    assert [o[2] for o in out] == [8.0, 8.0]


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    bench.rank_barrier(1)
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_rate(1, 32, 20, 0.5) == 1280.0


def test_reference_arm_nonzero_rank_exits_without_work():
    """Under torchrun only rank 0 runs the oracle and prints; the others exit 0 at once."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr[-500:]
    assert r.stdout.strip() == ""
