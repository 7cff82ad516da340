"""The N > 1 bench path on CPU: two gloo ranks run the replica logic of bench.py (no GPU).

bench.py under torchrun gives every rank an independent replica (the method has no exchange
step between instances): rendezvous, barrier, the max over ranks of the timed region, and
batched instances dealt round-robin to the ranks.
"""

import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank), "LSP_BENCH_GLOO": "1"})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    # each rank "timed" a different duration; everyone must see the slowest
    t_max = bench.max_over_ranks(10.0 + 5.0 * r, w)
    mine = bench.shard(range(256), r, w)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"world": w, "rank": r, "local": local, "t_max": t_max, "mine": mine}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_logic(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert [x["rank"] for x in res] == [0, 1] and all(x["world"] == 2 for x in res)
    assert all(x["t_max"] == 15.0 for x in res)
    a, b = set(res[0]["mine"]), set(res[1]["mine"])
    assert not (a & b) and a | b == set(range(256)) and len(a) == len(b) == 128


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.shard(range(5), 0, 1) == [0, 1, 2, 3, 4]
