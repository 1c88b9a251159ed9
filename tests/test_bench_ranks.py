"""The multi-process host logic of bench.py on CPU (world size 2, gloo, 127.0.0.1): replicas
share no data, so the only exchange is the timing reduction, the slowest rank's time, and the
whole-job value counts every rank's rays over that time.  The reference arm runs on rank 0 only;
the other ranks exit 0 without output."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank: int, world: int, port: int, times, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], dist, torch.device("cpu"))
        out.put((rank, t, bench.whole_job_value(1000, 10, world, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    times = [0.75, 1.5]
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, value in res:
        assert t == 1.5                                # the slowest rank's time on every rank
        assert value == pytest.approx(2 * 1000 * 10 / 1.5)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.25) == 0.25
    assert bench.whole_job_value(7, 3, 1, 0.5) == pytest.approx(42.0)


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_runs_on_rank0_only(rank):
    env = {**os.environ, "RANK": str(rank), "WORLD_SIZE": "2", "LOCAL_RANK": str(rank),
           "MASTER_ADDR": "127.0.0.1"}
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "schwarzschild_129", "--steps", "1", "--warmup", "0", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    if rank == 1:
        assert lines == []
    else:
        line = json.loads(lines[-1])
        assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
        assert line["cpu_baseline"]["kind"] == "oracle"
