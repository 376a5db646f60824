"""The multi-GPU path is replicas only (independent instances, no collective
in the data path): the benchmark's rank helpers and its reference arm under
torchrun, exercised with world_size 2 on the gloo backend (CPU)."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import gpcg_inputs as gi
    import oracle
    w, r, _ = bench._dist()
    assert (w, r) == (ws, rank)
    # each rank solves its own replica of the same QP; timing is the max
    # over ranks, the aggregate rate counts every rank's solves
    qp = gi.single_small()
    bench._barrier(w)
    res = oracle.solve(qp, tau_rel=1e-8)
    t = 0.25 * (rank + 1)  # stand-in durations that differ per rank
    tmax = bench._max_over_ranks(w, t)
    bench._barrier(w)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"tmax": tmax, "status": res.status, "q": res.stats["q"]}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_rank_helpers_gloo_world2(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    outs = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    assert all(o["status"] == 0 for o in outs)
    assert outs[0]["q"] == outs[1]["q"]  # replicas: the same result on every rank
    assert outs[0]["tmax"] == outs[1]["tmax"] == 0.5


def test_reference_arm_prints_on_rank0_only():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
