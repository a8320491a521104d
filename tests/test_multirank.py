"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The measured path shards by field: every rank measures its own field and the
ranks meet only at a barrier and a max-reduction of their step times (weak
scaling, no data-path collective).  These tests run that logic on two gloo
ranks, and the reference arm under torch.distributed.run, where rank 0 alone
prints the JSON line and rank 1 exits 0 without work."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(impl="reference")
    w, r, _ = bench.dist_setup(args)
    bench.barrier(w)
    worst = bench.reduce_max(10.0 + 5.0 * r, w, "cpu")   # per-rank step ms 10, 15
    field, _ = bench.field_for(r, 16)
    import torch.distributed as dist
    dist.destroy_process_group()
    out.put((r, w, worst, float(field[0, 0, 0]), float(field.std())))


def test_two_gloo_ranks_barrier_reduce_and_own_fields():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, m0, f0, s0), (r1, w1, m1, f1, s1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    # both ranks see the slowest rank's step time
    assert m0 == m1 == 15.0
    # each rank measures its own field (seed offset by rank)
    assert f0 != f1 and s0 > 0 and s1 > 0
    # whole-job throughput over 2 ranks at the slowest step
    assert np.isclose(2 * 1000.0 / m0, 133.33333333333334)


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--grid", "64"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
