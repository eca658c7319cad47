"""The N > 1 path of bench.py on CPU: two gloo ranks, as torchrun would start
them.  Each rank completes its own tensors (distinct seeds, same shapes); the
job's time is the slowest rank's (all-reduce MAX) and its rate counts the
units of every rank.  The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        ms, value = b.job_throughput(local_ms, 300, ws, "cpu")
        seeds = [w.seed for w in b.rank_workloads(rank)]
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(f"{ms} {value} {' '.join(map(str, seeds))}\n")
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_count_all_units(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    ws = 2
    mp.start_processes(_rank, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, start_method="spawn", join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(ws)]
    for row in rows:
        ms, value = float(row[0]), float(row[1])
        assert ms == 150.0                      # max over ranks
        assert value == pytest.approx(2 * 300 / 0.150)  # units of both ranks / slowest time
    seeds = [list(map(int, row[2:])) for row in rows]
    assert len(seeds[0]) == len(bench.OBSERVED)
    assert not set(seeds[0]) & set(seeds[1])   # each rank completes its own tensors


def test_single_rank_needs_no_process_group():
    ms, value = bench.job_throughput(250.0, 100, 1, "cpu")
    assert ms == 250.0 and value == pytest.approx(400.0)


def test_rank_workloads_share_shapes():
    a, b = bench.rank_workloads(0), bench.rank_workloads(3)
    assert [(w.n1, w.n2, w.n3, w.r, w.observed) for w in a] == [(w.n1, w.n2, w.n3, w.r, w.observed) for w in b]
    assert (a[0].n1, a[0].n2, a[0].n3, a[0].r) == (144, 288, 168, 8)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(None) is None  # returns before any work
    assert capsys.readouterr().out == ""
