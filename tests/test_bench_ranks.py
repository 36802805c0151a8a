"""Host-side logic of bench.py with more than one rank, on CPU: the timing is the maximum
over ranks (two gloo processes on 127.0.0.1), the job value counts every rank's units, and
under a multi-rank launch the reference arm runs on rank 0 only (the others exit 0 at once
with no output).  The GPU replicas themselves share nothing: each rank runs its own
workload on its own device."""
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


def _worker(rank, ws, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        ms = bench._max_over_ranks(torch, 10.0 + 3.0 * rank, ws, "cpu")
        with open(os.path.join(out, f"r{rank}.txt"), "w") as f:
            f.write(repr(ms))
    finally:
        dist.destroy_process_group()


def test_timing_is_the_maximum_over_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ws, port = 2, _free_port()
    mp.spawn(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    got = [float(open(tmp_path / f"r{r}.txt").read()) for r in range(ws)]
    assert got == [13.0, 13.0]


def test_single_rank_needs_no_process_group():
    torch = pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench._max_over_ranks(torch, 4.5, 1, "cpu") == 4.5


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1", MASTER_ADDR="127.0.0.1",
               MASTER_PORT=str(_free_port()))
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                         env=env, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    assert out.stdout.strip() == ""
