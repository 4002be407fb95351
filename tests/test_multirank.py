"""The N > 1 host path of bench.py on CPU: two gloo ranks on 127.0.0.1.

The library runs one process per GPU as independent replicas (no data-path
collective); the only cross-rank steps are the barrier and the max of the
per-rank times, and the whole-job value counts every rank's updates over the
slowest rank's time.  The reference arm runs on rank 0 only.
"""
import argparse
import io
import multiprocessing as mp
import os
import socket
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(dist, times[rank], "cpu")
        q.put((rank, t, bench.job_glups(world, 1_000_000, 50, t)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.25, 0.4]
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t, glups in res:
        assert t == 0.4
        assert glups == 2 * 1_000_000 * 50 / 0.4 / 1e9


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(None, 0.3, "cpu") == 0.3
    assert bench.job_glups(1, 16_777_216, 1000, 0.39) == 16_777_216 * 1000 / 0.39 / 1e9


def test_reference_arm_runs_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench
    args = argparse.Namespace(steps=10, warmup=3, gpus=2)
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.run_reference(args, 1, 2) is None
    assert out.getvalue() == ""


def test_reference_arm_line_on_rank_zero():
    """The reference arm (the FP64 oracle on the host cores) prints one JSON
    line with the contract's keys, on the same metric and unit."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "3", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "GLUPS"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
