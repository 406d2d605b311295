"""Multi-process path of bench.py on CPU (gloo, world size 2): the timing
reduction (slowest rank), the sums of per-rank counts, and the dealing of
independent problems to ranks (every problem exactly once).  The method's
sweeps do not shard, so several GPUs only run replicas or disjoint shares of
a batch; these helpers are all that differs from one GPU."""
import json
import os
import socket

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cpu = torch.device("cpu")
    w, r, lr = bench.rank_env()
    res = {"env": [w, r, lr],
           "max": bench.max_over_ranks(10.0 + 5.0 * rank, world, cpu),
           "sum": bench.sum_over_ranks(rank + 1, world, cpu),
           "shard": bench.shard(list(range(11)), rank, world)}
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump(res, f)


def test_rank_helpers_world_2(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r, x in enumerate(res):
        assert x["env"] == [world, r, r]
        assert x["max"] == 15.0            # the slowest rank's time
        assert x["sum"] == 3.0             # 1 + 2
    dealt = sorted(res[0]["shard"] + res[1]["shard"])
    assert dealt == list(range(11))      # every problem once
    assert not set(res[0]["shard"]) & set(res[1]["shard"])


def test_rank_helpers_single_process():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None) == 3.5
    assert bench.sum_over_ranks(4, 1, None) == 4
    assert bench.shard([1, 2, 3], 0, 1) == [1, 2, 3]
