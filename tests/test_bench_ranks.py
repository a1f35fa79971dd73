"""bench.py's multi-rank logic on CPU (world size 2, gloo on 127.0.0.1): the timed region is the
slowest rank's, the value counts every rank's work, and the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=2)
    t = bench.max_over_ranks(1.5 + rank, 2, "cpu")        # rank 1 is the slower one
    out[rank] = (t, bench.whole_job_rate(2, 3e9, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_whole_job_rate():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    for rank in (0, 1):
        t, v = res[rank]
        assert t == 2.5                                     # both ranks see the slowest time
        assert abs(v - 2 * 3.0 / 2.5) < 1e-12               # all ranks' units over that time


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup, gpus = 1, 0, 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(A()) == 0
    assert buf.getvalue() == ""


def test_reference_arm_on_rank_zero_uses_every_core(monkeypatch):
    import json
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setattr(bench, "pick_oracle_side", lambda budget: 128)

    class A:
        steps, warmup, gpus = 1, 0, 1

    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(A()) == 0
    line = json.loads(buf.getvalue())
    assert line["impl"] == "reference" and line["value"] > 0 and line["config"]["grid"] == [128, 128]
    assert "FP64 CPU oracle" in line["config"]["workload"] and "FP32" not in line["config"]["workload"]
    assert line["cpu_baseline"]["cores"] == bench.host_cores()
    assert line["e2e"]["value"] == line["value"]
