"""Sharding one problem's slices over ranks, on one GPU: each rank is a
context of its own over the whole problem that propagates only its block
(mmp_sweep_fine), the records are gathered on every rank (mmp_get_records /
mmp_set_records), the driver runs on every rank (mmp_sweep_coarse), and the
fine output at the end of a block is handed to the next rank
(mmp_get_output / mmp_set_output).  The ranks run in lock-step in one
process, so no kernel ever waits for another rank's kernel.  Every rank's
macro states equal the single-context run bit for bit (same launch shapes,
same reductions), and the FP64 run matches the oracle to 1e-10."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import shard
from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _single(p):
    from paper_2310_11365_gb300.mmp import Solver

    s = Solver(p)
    k = s.run()
    mom = s.moments(0)
    s.close()
    return k, mom


@pytest.mark.parametrize("make,world", [
    (lambda: W.config2(P=100_003, N=12, T=1.5, precision="fp64", tol=1e-9), 2),
    (lambda: W.config2(P=100_003, N=12, T=1.5, precision="fp64", tol=1e-9), 3),
    (lambda: W.config2(P=400_003, N=16, T=2.0, precision="mixed", tol=1e-7), 4),
    (lambda: W.config3(P=60_001, N=9, T=3.0, dt=5e-3, precision="fp64", tol=1e-8), 3),
])
def test_sharded_ranks_equal_the_single_context(mmplib, orc, make, world):
    p = make()
    k1, one = _single(p)
    engines = [shard.LibraryEngine(p) for _ in range(world)]
    try:
        moms = shard.run_lockstep(engines)
        for e, m in zip(engines, moms):
            assert e.status()["sweeps"] == k1
            assert np.array_equal(m, one)
    finally:
        for e in engines:
            e.close()
    assert k1 >= 2
    if p.precision == "fp64":
        ref = orc.parareal(p)
        assert ref["sweeps"] == k1
        for n in range(p.N + 1):
            M, V = ref["hist"][-1][n]
            assert abs(one[n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V))
            assert abs(one[n, 7] - V) <= 1e-10 * V


def test_split_sweep_state_checks(mmplib):
    """The phases in the wrong order are MMP_ERR_STATE; a range outside the
    slices is MMP_ERR_INVALID_ARG; mmp_iterate waits for a pending driver."""
    from paper_2310_11365_gb300.mmp import MMPError, Solver

    p = W.config1(P=2001, N=4, T=1.0)
    s = Solver(p)
    with pytest.raises(MMPError) as e:
        mmplib.mmp_sweep_fine(s.ctx, 0, 0, 4)          # before the lift
    assert e.value.code == -7
    s.lift()
    with pytest.raises(MMPError) as e:
        mmplib.mmp_sweep_coarse(s.ctx, 0)              # no fine phase yet
    assert e.value.code == -7
    with pytest.raises(MMPError) as e:
        mmplib.mmp_sweep_fine(s.ctx, 0, 2, 5)
    assert e.value.code == -1
    mmplib.mmp_sweep_fine(s.ctx, 0, 0, 4)
    with pytest.raises(MMPError) as e:
        mmplib.mmp_sweep_fine(s.ctx, 0, 0, 4)          # its driver has not run
    assert e.value.code == -7
    with pytest.raises(MMPError) as e:
        s.iterate(1)
    assert e.value.code == -7
    mmplib.mmp_sweep_coarse(s.ctx, 0)
    s.iterate(1)
    assert s.status()["sweeps"] == 2
    s.close()
