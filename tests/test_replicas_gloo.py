"""Host logic of the multi-process benchmark, on CPU with the gloo backend and
two ranks: the maximum over ranks, the barrier, and that a torchrun launch of
the benchmark prints exactly one JSON line (rank 0) while the other rank exits
cleanly. The solver itself has no exchange step (replicas only)."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2",
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r = bench.dist_init(None)
    assert (ws, r) == (2, rank)
    bench.barrier(ws)
    out[rank] = bench.max_over_ranks(10.0 + rank, ws)
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.skipif(torch.cuda.is_available(), reason="the gloo path is the CPU one")
def test_max_over_ranks_and_barrier():
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        assert dict(out) == {0: 11.0, 1: 11.0}


@pytest.mark.skipif(torch.cuda.is_available(), reason="the gloo path is the CPU one")
def test_torchrun_two_ranks_print_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--matrix-size", "256", "--steps", "1", "--warmup", "1"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["n_gpus"] == 2
