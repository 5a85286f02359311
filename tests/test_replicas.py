"""Host-side logic of the multi-GPU path on CPU: the sweep's shards and the
whole-job aggregation over ranks, run as two gloo processes (one process per
GPU in the real launch; the exchange is the same scalars)."""
import json
import os
import socket

import pytest

from paper_1808_05510_gb300 import replicas, synth


def test_shard_members_partition_and_balance():
    members = synth.sweep_members(126, synth.lambda_grid(), synth.fold_partition(126))
    for world in (1, 2, 3, 8):
        shards = [replicas.shard_members(members, r, world) for r in range(world)]
        ids = sorted(id(m) for s in shards for m in s)
        assert ids == sorted(id(m) for m in members)  # disjoint and complete
        sizes = [len(s) for s in shards]
        assert max(sizes) - min(sizes) <= 1
        if world > 1:  # longest first, dealt round-robin: every shard spans the lambda range
            for s in shards:
                lams = [m[0] for m in s]
                assert max(lams) >= 1e5 and min(lams) <= 10.0


def test_aggregate_single_rank():
    assert replicas.aggregate(5, 12.5, 1) == (5.0, 12.5)
    assert replicas.gather_objects({"a": 1}, 1) == [{"a": 1}]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units, ms = replicas.aggregate(rank + 1, 10.0 * (rank + 1), world)
        gathered = replicas.gather_objects({"rank": rank, "cv": [rank, 2 * rank]}, world)
        with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
            json.dump({"units": units, "ms": ms, "gathered": gathered}, f)
    finally:
        dist.destroy_process_group()


def test_aggregate_two_gloo_ranks(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        out = json.load(open(tmp_path / f"r{r}.json"))
        assert out["units"] == 3.0 and out["ms"] == 20.0  # work summed, slowest rank's time
        assert out["gathered"] == [{"rank": 0, "cv": [0, 0]}, {"rank": 1, "cv": [1, 2]}]
