"""Host logic of the multi-GPU benchmark run (N independent replicas, no
data-path collective), on two CPU ranks over gloo: the slowest rank's time
is taken on every rank and the whole-job rate counts every replica's work;
the reference arm prints only on rank 0."""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout
from types import SimpleNamespace

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    dist.barrier()
    ms = 100.0 + 25.0 * rank                      # rank 1 is the slowest
    ms_max = bench.max_over_ranks(ms, ws, "cpu")
    value = bench.whole_job_tflops(2.0e12, 4, ws, ms_max)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"ms": ms_max, "value": value}, f)


def test_two_replicas_max_time_and_whole_job_rate(tmp_path):
    ws, port = 2, _free_port()
    mp.start_processes(_rank, args=(ws, port, str(tmp_path)), nprocs=ws, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    for r in res:
        assert r["ms"] == 125.0                   # max over the ranks, seen by both
        # 2 replicas x 4 steps x 2 TFLOP in 125 ms
        assert abs(r["value"] - 2 * 4 * 2.0 / 0.125) < 1e-9


def test_single_rank_helpers_need_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert abs(bench.whole_job_tflops(1.0e12, 10, 1, 1000.0) - 10.0) < 1e-12


def test_reference_arm_prints_only_on_rank_zero(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(SimpleNamespace(steps=1, warmup=0))
    assert buf.getvalue() == ""
