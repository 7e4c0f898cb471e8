"""The multi-GPU form of the benchmark on the host: replicas that share
nothing (Sec. II works pair by pair, so pairs shard across ranks with no data
exchange).  Two gloo ranks on the CPU check the pieces bench.py's N > 1 run
uses: every rank matches its own pairs (disjoint across ranks), the timed
region's length is the slowest rank's (max over ranks), and the whole-job
value counts every rank's pixel-disparities over that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = {}
    # each rank's step time differs; every rank sees the slowest one
    res["t_max"] = bench._max_over_ranks(torch, torch.device("cpu"), 0.25 + rank, world)
    res["ids"] = {name: bench.rank_pair_ids(wl, rank) for name, wl in bench.WORKLOADS.items()}
    # the pairs a single-pair rank matches come from its own seed
    L, R, gt = bench.make_pair(bench.WORKLOADS["perlin320"], bench.rank_pair_ids(bench.WORKLOADS["perlin320"], rank)[0])
    res["first_row"] = L[0, :16, 0].tolist()
    dist.barrier()
    dist.destroy_process_group()
    out[rank] = res


def test_two_gloo_ranks_shard_pairs_and_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0]["t_max"] == res[1]["t_max"] == 1.25
    for name in res[0]["ids"]:
        a, b = set(res[0]["ids"][name]), set(res[1]["ids"][name])
        assert a and b and not (a & b), name                    # disjoint, non-empty
        assert len(a) == len(res[0]["ids"][name])               # no pair twice on a rank
    assert res[0]["first_row"] != res[1]["first_row"]           # different images per rank
    # whole-job value: every rank's work over the slowest rank's time
    import bench
    wl = bench.WORKLOADS["tissue960"]
    P = wl["W"] * wl["H"] * wl["D"]
    steps = 10
    value = world * steps * P / res[0]["t_max"] / 1e9
    assert value == pytest.approx(2 * 10 * 960 * 540 * 128 / 1.25 / 1e9)
