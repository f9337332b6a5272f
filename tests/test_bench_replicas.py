"""bench.py's multi-GPU path is replicas only: each rank solves its own frames, and the one
collective is the MAX over ranks of the timed region.  Checked here with two gloo ranks on the
CPU.
"""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import bench as b
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        step_ms = [1.0 + rank, 2.0 + rank, 3.0 + rank]   # rank 1 is the slower replica
        v, per_step = b.whole_job_ms_per_unit(dist, "cpu", step_ms)
        v4, _ = b.whole_job_ms_per_unit(dist, "cpu", step_ms, units_per_step=4)
        seeds = [None] * world
        dist.all_gather_object(seeds, b.frame_seeds(rank, 5))
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"value": v, "per_step": per_step, "value4": v4, "seeds": seeds}, f)
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_over_all_frames(tmp_path):
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    out = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for d in out:
        # slowest rank (rank 1): 2 + 3 + 4 = 9 ms for its 3 frames; the job solved 6 frames in 9 ms
        assert d["value"] == pytest.approx(9.0 / 6)
        assert d["per_step"] == pytest.approx(3.0)
        assert d["value4"] == pytest.approx(9.0 / 24)
    s0, s1 = out[0]["seeds"]
    assert len(s0) == len(s1) == 5
    assert not set(s0) & set(s1), "replicas must solve disjoint frames"


def test_one_process_value_is_the_mean_step_time():
    v, per_step = bench.whole_job_ms_per_unit(None, "cpu", [1.0, 2.0, 4.5])
    assert v == pytest.approx(2.5) and per_step == pytest.approx(2.5)
    v, _ = bench.whole_job_ms_per_unit(None, "cpu", [3.0, 3.0], units_per_step=64)
    assert v == pytest.approx(3.0 / 64)
    with pytest.raises(ValueError):
        bench.whole_job_ms_per_unit(None, "cpu", [])
    assert bench.frame_seeds(0, 3) == [0, 1, 2]
    assert bench.frame_seeds(2, 2) == [200000, 200001]
    with pytest.raises(ValueError):
        bench.frame_seeds(0, 100001)
