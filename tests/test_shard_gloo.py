"""Several ranks on independent problems (the batch of 512 uneven MaxCuts): the partition
covers every problem exactly once, balances the estimated work within the
longest-processing-time bound, and two gloo ranks on the CPU agree on it and on the
max-over-ranks timing that bench.py reports.  No GPU: the ranks exchange only host values."""
import os
import socket

import numpy as np
import pytest

from paper_2403_09133_gb300 import shard as S


def _works(count=512, seed=7):
    # the batch's shape: n ~ U[64, 2048], average degree ~ U[3, 12], entries ~ n (1 + d)
    rng = np.random.default_rng(seed)
    n = rng.integers(64, 2049, count)
    d = rng.uniform(3, 12, count)
    return [S.work_estimate(int(a), int(a * (1 + b))) for a, b in zip(n, d)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_and_balances(world):
    w = _works()
    parts = [S.shard(w, r, world) for r in range(world)]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(w)))
    loads = [sum(w[i] for i in p) for p in parts]
    # LPT: no rank exceeds the mean load by more than one problem's work
    assert max(loads) <= sum(w) / world + max(w) + 1e-9
    if world == 1:
        assert parts[0] == list(range(len(w)))


def test_partition_is_deterministic_and_rejects_bad_ranks():
    w = _works(64, seed=3)
    assert S.assign(w, 4) == S.assign(list(w), 4)
    with pytest.raises(ValueError):
        S.shard(w, 4, 4)
    with pytest.raises(ValueError):
        S.assign(w, 0)
    # equal works: round robin in index order
    assert S.assign([1.0] * 6, 3) == [0, 1, 2, 0, 1, 2]


def test_reductions_without_a_process_group():
    assert S.max_over_ranks([1.5, -2.0]) == [1.5, -2.0]
    assert S.sum_over_ranks([3.0]) == [3.0]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import json
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _works()
        mine = S.shard(w, rank, world)
        got = [None] * world
        dist.all_gather_object(got, mine)
        # a per-rank "batch time" proportional to its work, as bench.py reduces it
        t_local = sum(w[i] for i in mine) * 1e-6
        t_max = S.max_over_ranks([t_local])[0]
        total = S.sum_over_ranks([len(mine)])[0]
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"mine": mine, "all": got, "t_local": t_local, "t_max": t_max,
                       "total": total}, f)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree(tmp_path):
    import json
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    outs = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    w = _works()
    for r, o in enumerate(outs):
        assert o["mine"] == S.shard(w, r, world)
        assert o["all"] == outs[0]["all"]                 # every rank sees the same partition
        assert o["total"] == len(w)
        assert o["t_max"] == max(x["t_local"] for x in outs)
    assert sorted(outs[0]["mine"] + outs[1]["mine"]) == list(range(len(w)))
    # whole-job throughput as bench.py reports it: all problems / the slowest rank's time
    value = len(w) / outs[0]["t_max"]
    assert value > 0 and outs[0]["t_max"] >= sum(w) * 1e-6 / world - 1e-12
