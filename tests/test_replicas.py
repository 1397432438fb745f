"""Multi-GPU form (replicas only): the round has no exchange step, so N ranks
run N independent replicas and meet only for a barrier and the max-over-ranks
timing.  Covered on CPU with world_size-2 gloo process groups; the reference
arm runs on rank 0 alone."""
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


def _rank(rank, ws, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, w, r, local = bench.dist_setup()
    assert (w, r, local) == (ws, rank, rank)
    slowest = bench.max_over_ranks(dist, times[rank])
    out[rank] = (slowest, bench.replicas_value(w, 10, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value():
    ws, port = 2, _free_port()
    times = [1.5, 2.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, port, times, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        assert res[r][0] == 2.0                 # every rank sees the slowest rank's time
        assert res[r][1] == pytest.approx(10.0)  # 2 ranks x 10 rounds / 2.0 s


def test_single_process_defaults():
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        assert k not in os.environ or os.environ[k] in ("0", "1")
    assert bench.max_over_ranks(None, 3.0) == 3.0
    assert bench.replicas_value(1, 5, 2.0) == 2.5


def test_reference_arm_only_rank0_prints(tmp_path):
    """Under torchrun the oracle arm runs on rank 0; the other rank exits 0 without work."""
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", "bench.py", "--gpus", "2", "--impl", "reference",
           "--steps", "1", "--warmup", "0", "--reference-sample-s", "1"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    import json
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["h2d_bytes_per_step"] == 0
