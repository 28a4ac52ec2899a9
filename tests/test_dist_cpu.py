"""The multi-rank (N > 1) path of bench.py, on CPU with the gloo backend.

With several GPUs, every rank solves its own instance (weak scaling, no
collective on the data path); the job's step time is the slowest rank's and
its throughput counts one application per rank.  These tests run two gloo
ranks as spawned processes on the host; they need no GPU.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str) -> None:
    import sys

    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench

    r, w, local = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        ms = bench.max_over_ranks(1.0 + 0.5 * r, w, torch.device("cpu"))
        value = bench.job_value(ms, w)
        _, _, f_true = bench.make_inputs(seed_offset=r)
        np.save(os.path.join(out_dir, f"rank{r}.npy"), np.array([r, w, local, ms, value]))
        np.save(os.path.join(out_dir, f"img{r}.npy"), f_true)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_every_rank(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        rr, w, local, ms, value = np.load(tmp_path / f"rank{r}.npy")
        assert (rr, w, local) == (r, world, r)
        assert ms == pytest.approx(1.5)                      # the slower rank's 1.5 ms
        assert value == pytest.approx(world * 1000.0 / 1.5)  # one application per rank per step
    # weak scaling: each rank solves a different (seeded) instance of the same size
    a, b = np.load(tmp_path / "img0.npy"), np.load(tmp_path / "img1.npy")
    assert a.shape == b.shape and not np.array_equal(a, b)


def test_single_rank_needs_no_process_group():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(2.5, 1, None) == 2.5
    assert bench.job_value(2.0, 1) == pytest.approx(500.0)


def test_reference_arm_is_silent_on_other_ranks(monkeypatch, capsys):
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.reference_arm(bench.parse(["--impl", "reference", "--gpus", "2"]))
    assert capsys.readouterr().out == ""


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the GPU arm's
    metric, unit and config keys, the steps it was asked for, and a
    cpu_baseline and e2e object describing that same run."""
    import json
    import sys

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    bench.reference_arm(bench.parse(["--impl", "reference", "--steps", "1", "--warmup", "1"]))
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT and d["higher_is_better"] is True
    assert d["value"] > 0 and abs(d["value"] - 1000.0 / d["ms_per_step"]) <= 1e-6 * d["value"]
    assert d["config"]["workload"] == "vessel256_half" and d["config"]["N"] == 256
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
