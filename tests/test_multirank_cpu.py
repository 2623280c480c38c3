"""The benchmark's multi-rank path on CPU: two gloo ranks, as torchrun starts
them. Every ray is independent, so the path shards by rays with no exchange.
Each rank evaluates its own shard. The only collective is the max over
ranks of the timed region. The whole-job rate counts every rank's rays
against the slowest rank's time. The reference arm does its work on rank 0
alone."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch
    import torch.distributed as dist
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, _ = bench.dist_env()
    # shards: the rank's own rays; gather the first rays of every rank
    rays = bench.rank_rays(64, r)
    first = torch.from_numpy(np.stack([a[:4] for a in rays.soa()]).astype(np.float64))
    got = [torch.empty_like(first) for _ in range(ws)]
    dist.all_gather(got, first)
    # timing: a rank-dependent time, maximised over the ranks
    t_rank = 1.0 + 0.5 * r
    t_max = bench.max_over_ranks(t_rank, ws, torch.device("cpu"))
    rate = bench.whole_job_rate(1000, ws, 3, t_max)
    res = {"rank": r, "ws": ws, "t_max": t_max, "rate": rate,
           "shards_differ": bool(not torch.equal(got[0], got[1])),
           "own_shard_first": first[:, 0].tolist()}
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as fh:
        json.dump(res, fh)
    dist.barrier()
    dist.destroy_process_group()


def _reference_rank(rank, world, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import contextlib
    import io

    import bench

    class Args:
        steps, warmup = 1, 0

    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args())
    with open(os.path.join(out_dir, f"ref{rank}.txt"), "w") as fh:
        fh.write(buf.getvalue())


def test_two_gloo_ranks_shard_and_time(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["ws"] == 2
        assert r["t_max"] == 1.5                      # the slower rank's time on both
        assert r["rate"] == pytest.approx(1000 * 2 * 3 / 1.5)
        assert r["shards_differ"]
    # each rank's shard is the one its seed defines
    sys.path.insert(0, ROOT)
    import bench
    for r in range(2):
        want = np.stack([a[:1] for a in bench.rank_rays(64, r).soa()])[:, 0]
        assert np.allclose(res[r]["own_shard_first"], want)


def test_reference_arm_runs_on_rank_zero_only(tmp_path):
    import torch.multiprocessing as mp
    mp.start_processes(_reference_rank, args=(2, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    out0 = (tmp_path / "ref0.txt").read_text().strip().splitlines()
    out1 = (tmp_path / "ref1.txt").read_text().strip()
    assert out1 == ""                                 # other ranks: no work, no line
    line = json.loads(out0[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
