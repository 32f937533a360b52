"""The multi-process path on the host: two gloo ranks on 127.0.0.1.  The bench's timing reduction (max over
ranks) and whole-job rate, and the reference arm under torchrun (rank 0 alone runs the oracle and prints one
line; the other rank exits 0 without work).  No GPU is used."""
import json
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


def _worker(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_seconds = 1.0 + rank  # rank 1 is the slower one
    m = bench.max_over_ranks(local_seconds, ws)
    rate = bench.whole_job_rate(1000.0, ws, m)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"max": m, "rate": rate}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_timing_reduction_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    for r in (0, 1):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["max"] == 2.0
        assert d["rate"] == pytest.approx(1000.0 * 2 / 2.0)


def test_single_rank_reduction_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once(tmp_path):
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle"
