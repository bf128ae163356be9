"""Measured launch shapes: the autotuner times the candidates it is given,
a registered shape is what the planner then uses, and results under a tuned
shape still match the oracle."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def clean_table():
    from paper_2310_11365_gb300 import tune

    tune.clear()
    yield
    tune.clear()


def test_autotune_times_each_candidate(mmplib, clean_table):
    from paper_2310_11365_gb300.mmp import mmp_autotune

    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=0.5, N=16, dt=1e-3, P=200_000, seed=3, precision="mixed")
    cands = [2, 4, 8, 13, 26]
    r = mmp_autotune(p, candidates=cands, probe_steps=16)
    assert r["best_nq"] in cands
    assert all(r["rates"][k] > 0 for k in cands)
    assert r["rates"][r["best_nq"]] == max(r["rates"].values())


def test_registered_shape_drives_the_plan(mmplib, clean_table):
    from paper_2310_11365_gb300.mmp import Solver, mmp_set_tuning

    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=0.5, N=16, dt=1e-3, P=200_000, seed=3, precision="mixed")
    base = Solver(p)
    nq0 = base.plan(0)["quads_per_thread"]
    base.close()
    want = 4 if nq0 != 4 else 8
    mmp_set_tuning("mixed", 100_000, 300_000, want)
    s = Solver(p)
    assert s.plan(0)["quads_per_thread"] == want
    s.close()
    mmp_set_tuning("mixed", 0, 0, 0)
    s = Solver(p)
    assert s.plan(0)["quads_per_thread"] == nq0
    s.close()


def test_tuned_shape_keeps_oracle_parity(mmplib, orc, clean_table):
    """FP64 run planned with a measured shape against the oracle to 1e-10 (the
    16 slices fill the GPU at either candidate, so the plan takes the measured
    one): the shape changes only the summation grouping."""
    from paper_2310_11365_gb300 import tune
    from paper_2310_11365_gb300.mmp import Solver

    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=1.6, N=16, dt=0.005, P=60_001, seed=7, precision="fp64")
    r = tune.tune(p, candidates=[1, 2], probe_steps=8)
    key = f"fp64:{int(np.floor(np.log2(p.P)))}"
    nq = r[key]["nq"]
    s = Solver(p)
    assert s.plan(0)["quads_per_thread"] == nq
    s.run()
    mom = s.moments(0)
    ref = orc.parareal(p)
    assert s.status(0)["sweeps"] == ref["sweeps"]
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert abs(mom[n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V))
        assert abs(mom[n, 7] - V) <= 1e-10 * V
    s.close()


def test_batch_cap_is_measured_and_used(mmplib, clean_table):
    """tune_batch times one batched sweep per cap candidate and registers the
    fastest; a batch created afterwards plans within that cap."""
    from paper_2310_11365_gb300 import tune
    from paper_2310_11365_gb300.mmp import Solver

    probs = W.config5(16, p_max=2e5)
    r = tune.tune_batch(probs, candidates=(8, 13), sample=8)
    assert r["nq"] in (8, 13)
    assert all(r["rates"][str(c)] > 0 for c in (8, 13))
    s = Solver(probs)
    assert max(s.plan(i)["quads_per_thread"] for i in range(len(probs))) <= r["nq"]
    s.close()
