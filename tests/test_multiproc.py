"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2): every rank gets
its own independent copy of the workload (weak scaling, no data exchange), the job's step time is
the slowest rank's, and the reported rate counts all ranks' entries. Only rank 0 runs the
reference arm."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    b = bench.rank_batch(rank, rays=[0])
    ms = bench.max_over_ranks(10.0 * (rank + 1), world, dist)
    ent = bench.entries(b["state"].shape[0], len(b["eps"]))
    q.put((rank, float(b["state"][:, 0].sum()), ms, bench.job_rate(ent, world, ms), ent))
    dist.barrier()
    dist.destroy_process_group()


def test_weak_scaling_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, ms0, v0, e0), (r1, s1, ms1, v1, e1) = res
    assert s0 != s1                      # independent problems per rank
    assert ms0 == ms1 == 20.0            # the slowest rank's time
    assert v0 == v1 == pytest.approx((e0 + e1) / 0.020)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), dict(gpus=2, steps=1, warmup=0))()
    out = io.StringIO()
    with redirect_stdout(out):
        assert bench.run_reference(args) == 0
    assert out.getvalue() == ""
