"""The N>1 host path of the benchmark on CPU: two gloo ranks.

At N>1 every rank runs an independent replica; the reported throughput is the
units all ranks processed over the slowest rank's time, after a barrier.  The
aggregation helpers pick gloo where no GPU is visible, so the same code runs
here as world size 2.  The reference arm prints from rank 0 only.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_init()
    assert (w, r) == (world, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    units = [1000, 3000][rank]
    ms = [10.0, 40.0][rank]
    value, total, ms_max = bench.replica_throughput(w, units, ms)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"value": value, "total": total, "ms_max": ms_max}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench(tmp_path):
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:                       # every rank sees the same aggregate
        assert g["total"] == 4000.0
        assert g["ms_max"] == 40.0
        assert g["value"] == pytest.approx(4000.0 / 0.040)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(1, 500, 25.0) == (500 / 0.025, 500, 25.0)


def test_reference_arm_prints_from_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    import workloads as wl
    w = wl.WORKLOADS["tfim1d_n64_periodic"]
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                      "--warmup", "0", "--ref-gates", "8"])
    args = bench.parse()
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args, w) == 0
    assert buf.getvalue() == ""
    monkeypatch.setenv("RANK", "0")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args, w) == 0
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["config"]["workload"] == w.name
    assert line["config"]["parallelism"] == "replicas x2"
    assert line["cpu_baseline"]["kind"] == "oracle"
