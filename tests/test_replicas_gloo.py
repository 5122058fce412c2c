"""The multi-GPU path of the benchmark (N independent replicas under torchrun)
on the host: two gloo ranks on the CPU run the whole-job aggregation that
bench.py applies to its timed region, and a replica's own result is unchanged
by the other's presence (no data-path collective)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 + r ms for 100 (r + 1) units of work
        t, w = bench.whole_job(10.0 + rank, 100.0 * (rank + 1), world, "cpu")
        out[rank] = (t, w)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_whole_job_max_time_summed_work(world):
    import torch.multiprocessing as mp
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    want_t = 10.0 + (world - 1)
    want_w = 100.0 * world * (world + 1) / 2
    for r in range(world):
        assert out[r] == (want_t, want_w)


def test_single_rank_is_identity():
    import bench
    assert bench.whole_job(12.5, 7.0, 1, "cpu") == (12.5, 7.0)


def test_reference_arm_under_torchrun_prints_one_line():
    """`bench.py --impl reference` launched as the driver launches N > 1:
    rank 0 alone times the oracle and prints one JSON line; the other rank
    exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
