"""The multi-rank side of bench.py on CPU (gloo, world size 2): replicas
only, so the one cross-rank step is the max over ranks of the timed region,
and only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    ms_max, value = bench.job_throughput(dist, 10.0 + 5.0 * rank, 1000, 10, ws)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"ms_max": ms_max, "value": value}, fh)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_takes_the_slowest_rank(tmp_path):
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    for r in range(ws):
        d = json.load(open(tmp_path / f"r{r}.json"))
        assert d["ms_max"] == 15.0
        # 2 replicas x 1000 nodes x 10 steps in 15 ms
        assert d["value"] == pytest.approx(1000 * 10 * 2 / 15e3)


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", MASTER_ADDR="127.0.0.1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
