"""The bench's N > 1 path on CPU: world-size-2 `gloo` ranks (no GPU).  Each rank solves its own
replica, so the only cross-rank steps are the timing/throughput reductions and the per-rank
noise draw; the reference arm prints from rank 0 only."""
import json
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synthetic as S  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 10 (r + 1) H applications
        res = bench.whole_job(1.0 + rank, 10 * (rank + 1), world, torch.device("cpu"))
        with open(os.path.join(outdir, "%d.json" % rank), "w") as f:
            json.dump(res, f)
    finally:
        dist.destroy_process_group()


def test_whole_job_is_slowest_rank_time_and_all_ranks_applies(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [tuple(json.load(open(tmp_path / ("%d.json" % r)))) for r in range(world)]
    assert res[0] == res[1] == (2.0, 30.0)


def test_single_rank_needs_no_process_group():
    assert bench.whole_job(3.5, 7, 1) == (3.5, 7.0)


def test_replicas_draw_independent_noise():
    wl = S.workload("cap32")
    mask = wl["ninv"] > 0
    n0, n1, n2 = (bench.replica_noise(wl, r) for r in range(3))
    assert n0 is wl["noise"]
    for n in (n1, n2):
        assert n.shape == n0.shape
        assert np.all(n[:, ~mask] == 0)
        # unit variance after whitening by N^-1
        z = n[:, mask] * np.sqrt(wl["ninv"][mask])
        assert abs(z.var() - 1) < 0.1
    assert not np.allclose(n1, n0) and not np.allclose(n2, n1)
    np.testing.assert_array_equal(n1, bench.replica_noise(wl, 1))   # seeded


def test_reference_arm_prints_from_rank_zero_only(capsys):
    class Args:
        steps, warmup = 1, 3
    bench.run_reference(Args, rank=1, world=2)
    assert capsys.readouterr().out == ""
