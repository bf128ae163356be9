"""Sharding one problem's slices over ranks (paper_2310_11365_gb300.shard),
on CPU: the data flow (contiguous blocks, records gathered on every rank,
the driver run redundantly, one boundary ensemble handed to the next rank
per sweep) with an oracle-backed engine, so that every sharded run can be
compared with the single-rank run and with orc_parareal bit for bit.  Two
real gloo ranks on 127.0.0.1, and the same flow in lock-step in one process
for two to five ranks."""
import json
import os
import socket
import sys

import numpy as np
import pytest

from paper_2310_11365_gb300 import shard
from paper_2310_11365_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from oracle_engine import OracleEngine  # noqa: E402


def _problem(**kw):
    base = dict(P=501, N=7, T=1.4, dt=0.02, precision="fp64", tol=1e-12, seed=31)
    base.update(kw)
    return W.cubic(1.0, 0.5, m0=0.5, s0=0.3, **base)


def test_blocks_partition_the_slices():
    for N in (1, 2, 7, 64, 129):
        for world in range(1, min(N, 9) + 1):
            blocks = [shard.slice_block(N, r, world) for r in range(world)]
            assert blocks[0][0] == 0 and blocks[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(blocks, blocks[1:]))
            sizes = [hi - lo for lo, hi in blocks]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1


def test_boundary_sends_and_receives_pair_up():
    """For every sweep a rank sends exactly when the next rank receives."""

    class Stub:
        def __init__(self, N):
            self.N = N

    for N in (3, 8, 33):
        for world in range(2, min(N, 6) + 1):
            ranks = [shard.Rank(Stub(N), r, world) for r in range(world)]
            for k in range(1, N + 1):
                for r in ranks:
                    r.k = k
                for a, b in zip(ranks, ranks[1:]):
                    assert a.sends_boundary() == b.receives_boundary(), (N, world, k)
                    # needed iff the receiver propagates its first slice lo in sweep k + 1
                    assert b.receives_boundary() == (b.lo >= k), (N, world, k)


def test_too_many_ranks_refused(orc):
    with pytest.raises(ValueError):
        shard.Rank(OracleEngine(orc, _problem(N=2)), 0, 3)


def test_single_rank_engine_is_the_oracle(orc):
    """The oracle-backed engine, run as one rank, reproduces orc_parareal's
    per-sweep moments bit for bit (so it can stand in for the oracle)."""
    p = _problem()
    got = shard.run_lockstep([OracleEngine(orc, p)])[0]
    ref = orc.parareal(p)
    assert got.shape == ref["hist"].shape
    assert np.array_equal(got, ref["hist"])


@pytest.mark.parametrize("world", [2, 3, 5])
def test_lockstep_ranks_equal_the_single_rank_run(orc, world):
    p = _problem()
    one = shard.run_lockstep([OracleEngine(orc, p)])[0]
    many = shard.run_lockstep([OracleEngine(orc, p) for _ in range(world)])
    for m in many:
        assert np.array_equal(m, one)
    assert one.shape[0] - 1 >= 3  # several sweeps, so boundaries moved


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                       "MASTER_PORT": str(port)})
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    import oracle
    from oracle_engine import OracleEngine as Engine
    from paper_2310_11365_gb300 import shard as sh

    oracle.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mom = sh.run_distributed(Engine(oracle, _problem()))
    dist.barrier()
    dist.destroy_process_group()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), mom)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"sweeps": int(mom.shape[0] - 1)}, f)


def test_two_gloo_ranks_equal_the_single_rank_run(orc, tmp_path):
    import torch.multiprocessing as mp

    p = _problem()
    one = shard.run_lockstep([OracleEngine(orc, p)])[0]
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for rank in range(2):
        got = np.load(tmp_path / f"rank{rank}.npy")
        assert np.array_equal(got, one), rank


def test_corrupted_boundary_is_caught(orc, monkeypatch):
    """Planted in the data flow: a rank that matches a perturbed copy of the
    previous rank's boundary ensemble into its first slice no longer
    reproduces the single-rank run."""
    p = _problem()
    one = shard.run_lockstep([OracleEngine(orc, p)])[0]
    monkeypatch.setattr(shard.Rank, "boundary_in",
                        lambda self, ensemble: self.engine.set_output(self.lo - 1, ensemble + 1e-6))
    many = shard.run_lockstep([OracleEngine(orc, p) for _ in range(2)])
    assert not all(np.array_equal(m, one) for m in many)
