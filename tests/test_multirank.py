"""The replicas-only multi-GPU path of bench.py, on CPU with two gloo ranks:
rank and world from the launcher's environment, one seed per rank, the job's
time as the slowest rank's (all-reduce MAX), the whole-job throughput over all
ranks, and the reference arm running on rank 0 only."""
import json
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    ws, r, local = bench.dist_setup(None)
    dist.init_process_group("gloo", rank=r, world_size=ws)
    # rank r timed (r + 1) * 10 ms for 3 steps of a 64 MB field
    t_ms = bench.rank_max(10.0 * (r + 1), dist, "cpu")
    gbs = bench.whole_job_gbs(64e6, ws, 3, t_ms * 1e-3)
    spec = bench.rank_spec("turb512", 1e-3, 64, r)
    dist.barrier()
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "local": local, "t_ms": t_ms, "gbs": gbs, "seed": spec.seed,
                   "dims": list(spec.dims)}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    rs = [json.load(open(tmp_path / f"rank{i}.json")) for i in range(2)]
    assert [(r["ws"], r["rank"], r["local"]) for r in rs] == [(2, 0, 0), (2, 1, 1)]
    assert [r["t_ms"] for r in rs] == [20.0, 20.0]   # both ranks see the slowest rank's time
    assert rs[0]["gbs"] == pytest.approx(64e6 * 2 * 3 / 0.020 / 1e9)
    assert rs[0]["seed"] != rs[1]["seed"]            # independent fields ...
    assert rs[0]["dims"] == rs[1]["dims"]            # ... of one workload


def test_one_rank_needs_no_process_group():
    assert bench.rank_max(12.5, None, "cpu") == 12.5
    assert bench.whole_job_gbs(4e9, 1, 2, 1.0) == pytest.approx(8.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    bench.run_reference(bench.parse_args())
    assert capsys.readouterr().out == ""
