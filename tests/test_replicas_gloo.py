"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.
The solve does not shard, so ranks are independent replicas with a barrier
and max-over-ranks timing.  Checks the rank environment, the barrier, the
reductions, the whole-job throughput (units of all ranks over the slowest
rank's time), and that the reference arm does its work on rank 0 only."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, local = bench.dist_setup()
    bench.barrier(w)
    units = 1000.0 * (rank + 1)       # replica r processed (r + 1) thousand units
    seconds = 2.0 + rank              # and the slowest one took 3 s
    res = {
        "world": w, "rank": r, "local": local,
        "max": bench.max_over_ranks(seconds, w),
        "sum": bench.sum_over_ranks(units, w),
        "value": bench.replica_value(units, seconds, w),
    }
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        res = json.loads((tmp_path / f"rank{rank}.json").read_text())
        assert res["world"] == 2 and res["rank"] == rank and res["local"] == rank
        assert res["max"] == 3.0
        assert res["sum"] == 3000.0
        assert res["value"] == pytest.approx(1000.0)


def test_reference_arm_other_ranks_do_no_work(monkeypatch):
    """Under torchrun only rank 0 runs the oracle timing; the others return 0
    at once (checked here without starting the oracle)."""
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        warmup = 1
        steps = 1
        gpus = 2

    assert bench.reference_arm(Args(), 2, 1) == 0
