"""Host logic of bench.py's multi-GPU path (replicas), on CPU: two gloo
ranks aggregate their work as the whole-job rate (units of all ranks over the
slowest rank's time); the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r processed 100 * (r + 1) units in r + 1 seconds
    rate, tmax = bench.world_rate(100.0 * (rank + 1), float(rank + 1), device="cpu")
    out[rank] = (rate, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_world_rate_two_gloo_ranks():
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        rate, tmax = out[r]
        assert tmax == 2.0 and rate == pytest.approx(300.0 / 2.0)


def test_world_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.world_rate(50.0, 2.0) == (25.0, 2.0)


def test_reference_arm_runs_on_rank_0_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload = "rmat22"
        steps = 1
        warmup = 0
    assert bench.reference_arm(Args()) == 0          # returns at once: no graph, no oracle


def test_reference_arm_line_on_a_small_graph(monkeypatch, capsys):
    """The reference arm on rank 0 (the CPU oracle on a scale-10 stand-in for
    the workload): one JSON line with the arm's fields; a step runs one BFS
    from each seeded source, or from the first k when the run would pass the
    time cap (here forced down to a single source per step)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setitem(bench.RMAT_CONFIGS, "rmat22",
                        dict(scale=10, edge_factor=16, seed=10, wmax=64, weight_seed=110))

    class Args:
        workload = "rmat22"
        steps = 2
        warmup = 1
    assert bench.reference_arm(Args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GTEPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert "16 of the 16 seeded sources per step" in line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    monkeypatch.setattr(bench, "REF_TIME_CAP_S", 0.0)
    assert bench.reference_arm(Args()) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert "1 of the 16 seeded sources per step" in line["cpu_baseline"]["sample"]
