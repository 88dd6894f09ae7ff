"""N > 1 host logic of bench.py on CPU (gloo, world size 2): the timing reduction over ranks and the
reference arm launched the way the N-GPU bench is (torch.distributed.run on 127.0.0.1), where rank
0 alone runs and prints and the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out_dir):
    os.environ.update(WORLD_SIZE="2", RANK=str(rank), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    import torch.distributed as dist

    ws, r, _ = bench.dist_setup(argparse.Namespace(impl="reference"))
    got = bench.max_over_ranks(ws, 1.5 + r)  # rank 1 is the slower one
    bench.barrier(ws)
    with open(os.path.join(out_dir, f"r{r}.txt"), "w") as f:
        f.write(f"{ws} {got}")
    dist.destroy_process_group()


def test_max_over_ranks_with_gloo(tmp_path):
    import torch.multiprocessing as mp

    mp.start_processes(_worker, args=(_free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    for r in (0, 1):
        ws, got = (tmp_path / f"r{r}.txt").read_text().split()
        assert int(ws) == 2 and float(got) == 2.5


def test_reference_arm_under_torchrun():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--workload", "far64x1", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
