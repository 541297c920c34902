"""Multi-rank host logic of bench.py on CPU: two gloo ranks check the
max-over-ranks reduction, the instance partition of the batched workload,
per-rank replica inputs, and that the reference arm runs on rank 0 only."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import sp_inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        w, r, lr = bench.rank_env()
        res["env"] = (w, r, lr)
        res["max"] = bench.max_over_ranks(1.5 + rank, world)
        res["max_none"] = bench.max_over_ranks(None, world)
        costs = [bench.instance_cost(ab.shape[0], ab.shape[1] - 1) for _, ab, _ in sp_inputs.workload(3, n=24)]
        res["parts"] = bench.shard_instances(costs, world)
        args = bench.parse(["--n", "600", "--workload", "tridiag"])
        _, ab, nu = bench.workload_band(args, rank)
        res["band_sum"] = float(np.sum(ab))
        res["nu"] = nu
        # the reference arm: rank 0 prints one JSON line, the others exit 0 without work
        args = bench.parse(["--impl", "reference", "--n", "600", "--cpu-sample-n", "96",
                            "--steps", "1", "--warmup", "1"])
        buf = io.StringIO()
        with redirect_stdout(buf):
            res["ref_rc"] = bench.run_reference(args)
        res["ref_out"] = buf.getvalue()
        dist.barrier()
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([res], dtype=object), allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / f"rank{r}.npy", allow_pickle=True)[0] for r in range(world)]
    for r in range(world):
        assert res[r]["env"] == (world, r, r)
        assert res[r]["max"] == 2.5                    # max over ranks, same on every rank
        assert res[r]["max_none"] is None
        assert res[r]["parts"] == res[0]["parts"]      # every rank computes the same partition
        assert res[r]["ref_rc"] == 0
    parts = res[0]["parts"]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(24))                     # disjoint cover of the instances
    assert all(len(p) > 0 for p in parts)
    assert res[0]["band_sum"] != res[1]["band_sum"]    # replicas draw their own inputs
    assert res[0]["nu"] == res[1]["nu"] == 300
    import json
    line = json.loads(res[0]["ref_out"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 1 and line["unit"] == "s/projector"
    assert res[1]["ref_out"] == ""                     # rank 1 prints nothing


def test_shard_balance():
    costs = [10.0, 9.0, 8.0, 1.0, 1.0, 1.0]
    parts = bench.shard_instances(costs, 2)
    loads = [sum(costs[i] for i in p) for p in parts]
    assert parts == [[0, 3, 4, 5], [1, 2]]
    assert max(loads) - min(loads) <= max(costs)
    assert bench.shard_instances(costs, 1) == [[0, 1, 2, 3, 4, 5]]
    assert bench.shard_instances([], 3) == [[], [], []]
