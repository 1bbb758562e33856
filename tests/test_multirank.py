"""The bench's multi-rank host logic on CPU (gloo, world size 2): rank setup from the launcher's
environment, the barrier, and the maximum over ranks that the timed region reports; and the
reference arm under the launcher, where rank 0 alone runs and prints one JSON line and the other
rank exits 0 without work.  (Ranks solve independent instances: there is no data-path
collective to test.)"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch

    import bench

    dist, w, r, _ = bench.dist_setup(torch)
    try:
        bench.barrier(dist, torch)
        m = bench.max_over_ranks(dist, torch, float(10 * (r + 1)))
        bench.barrier(dist, torch)
        with open(os.path.join(out, f"rank{r}.json"), "w") as f:
            json.dump({"world": w, "rank": r, "max": m, "backend": dist.get_backend()}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_maximum(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, g in enumerate(got):
        assert g == {"world": 2, "rank": r, "max": 20.0, "backend": "gloo"}


def test_reference_arm_prints_once_under_the_launcher():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
