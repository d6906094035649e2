"""The N > 1 launch path on CPU: the bench's max-over-ranks timing and whole-job throughput
with two gloo ranks, and the reference arm under torchrun (rank 0 alone reports)."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, str(ROOT))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 14.0][rank]                       # rank 1 is the slower one
    m = bench.max_over_ranks(ms, world, "cpu")
    v = bench.job_throughput(world, 10, m / 1e3)
    dist.barrier()
    dist.destroy_process_group()
    Path(out, f"r{rank}.json").write_text(json.dumps({"max": m, "value": v}))


def test_max_over_ranks_and_job_throughput_gloo(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        d = json.loads((tmp_path / f"r{r}.json").read_text())
        assert d["max"] == 14.0                   # both ranks see the slowest rank's time
        assert d["value"] == pytest.approx(2 * 10 / 0.014)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, str(ROOT))
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.job_throughput(1, 4, 2.0) == 2.0


def test_reference_arm_under_torchrun_reports_once():
    """Two ranks launched the way the multi-GPU bench is; the reference arm (the oracle on
    host cores) runs on rank 0 only and prints one JSON line; rank 1 exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--config", "1"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the same config object as the GPU arm's line at its default launch shape
    sys.path.insert(0, str(ROOT))
    import bench
    from synth import make_scene
    assert d["config"] == bench.arm_config(make_scene(1), 16, 128, 32, 1)
