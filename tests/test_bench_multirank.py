"""The N > 1 path of bench.py on CPU: world size 2 over gloo.  Each rank is
an independent replica; the job time is the slowest rank's and the value is
the sum of the units over ranks divided by that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    own = [2.0, 5.0][rank]  # seconds this rank took
    mx = bench.max_over_ranks(own, ws)
    thr = bench.job_throughput(100.0, own, ws)
    env = bench.dist_env()
    q.put((rank, mx, thr, env))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, thr, env in res:
        assert mx == 5.0
        assert thr == pytest.approx(2 * 100.0 / 5.0)
        assert env == (2, rank, rank)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10.0, 2.0, 1) == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun with N > 1 the reference arm (the oracle on the host)
    runs and prints on rank 0 alone; the other ranks exit 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    base = dict(os.environ, WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1",
           "--n", "256"]
    r1 = subprocess.run(cmd, cwd=root, env=dict(base, RANK="1", LOCAL_RANK="1"), capture_output=True, text=True,
                        timeout=300)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = subprocess.run(cmd, cwd=root, env=dict(base, RANK="0", LOCAL_RANK="0"), capture_output=True, text=True,
                        timeout=300)
    assert r0.returncode == 0
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
