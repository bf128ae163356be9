"""Batched sweeps (many problems, one cooperative launch per sweep): the
same results as per-problem launches with the same launch shapes, bit for
bit; parity with the oracle; and the exactness invariant per problem."""
import os

import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _batch_problems(precision="mixed", n=12, seed=3):
    """Config-5 forms (linear / double well) with uneven P and N, small."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        P = int(round(10 ** rng.uniform(3.0, 5.3)))
        N = int(rng.integers(4, 13))
        common = dict(T=0.5 * N / 4, N=N, dt=2e-3, P=P, coarse_h=0.25, seed=W.SEED_BASE + 5,
                      problem_tag=i, tol=1e-6, precision=precision, max_iter=4)
        if i % 2 == 0:
            out.append(W.linear(float(rng.uniform(0.5, 2)), float(rng.uniform(0, 1)), float(rng.uniform(0.3, 1)),
                                m0=1.0, s0=0.1, **common))
        else:
            out.append(W.double_well(0.25, 0.5, float(rng.uniform(0, 1)), float(rng.uniform(0.3, 1)),
                                     m0=0.0, s0=0.3, **common))
    return out


def _solve(problems, batch: bool):
    from paper_2310_11365_gb300.mmp import Solver

    old = os.environ.get("MMP_BATCH")
    os.environ["MMP_BATCH"] = "1" if batch else "0"
    try:
        s = Solver(problems)
    finally:
        if old is None:
            del os.environ["MMP_BATCH"]
        else:
            os.environ["MMP_BATCH"] = old
    s.run()
    moms = [s.moments(i) for i in range(len(problems))]
    sts = [s.status(i) for i in range(len(problems))]
    plans = [s.plan(i) for i in range(len(problems))]
    return s, moms, sts, plans


def test_batched_equals_per_problem_launches(mmplib):
    probs = _batch_problems()
    sb, mb, stb, pb = _solve(probs, True)
    sp, mp, stp, pp = _solve(probs, False)
    assert pb == pp
    for i in range(len(probs)):
        assert stb[i]["sweeps"] == stp[i]["sweeps"]
        assert np.array_equal(mb[i], mp[i]), i
        assert stb[i]["dev_err"] == 0
    sb.close()
    sp.close()


def test_batched_fp64_matches_oracle(mmplib, orc):
    probs = _batch_problems("fp64", n=6, seed=11)
    s, moms, sts, _ = _solve(probs, True)
    for i, p in enumerate(probs):
        ref = orc.parareal(p)
        assert sts[i]["sweeps"] == ref["sweeps"]
        for n in range(p.N + 1):
            M, V = ref["hist"][-1][n]
            assert abs(moms[i][n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V)), (i, n)
            assert abs(moms[i][n, 7] - V) <= 1e-10 * V, (i, n)
    s.close()


def test_batched_exactness_invariant(mmplib):
    """After k batched sweeps, slices 0..k of every problem equal that
    problem's serial run (same launch shape) bit for bit."""
    from paper_2310_11365_gb300.mmp import Solver

    probs = [p.scaled(max_iter=2, tol=0.0) for p in _batch_problems(n=8, seed=7)]
    s = Solver(probs)
    s.run()
    for i, p in enumerate(probs):
        mom = s.moments(i)
        ser = s.serial(i, n_end=2)
        for n in range(3):
            assert mom[n, 1] == ser[n, 1] and mom[n, 2] == ser[n, 2], (i, n)
    s.close()


def test_batched_graph_equals_direct_enqueue(mmplib):
    """Sweeps replayed from the captured CUDA graph equal the same sweeps
    enqueued directly, bit for bit, and both stop where the problems do."""
    probs = _batch_problems(n=10, seed=5)
    old = os.environ.get("MMP_BATCH_GRAPH")
    try:
        os.environ["MMP_BATCH_GRAPH"] = "0"
        sd, md, std_, _ = _solve(probs, True)
    finally:
        if old is None:
            del os.environ["MMP_BATCH_GRAPH"]
        else:
            os.environ["MMP_BATCH_GRAPH"] = old
    sg, mg, stg, _ = _solve(probs, True)
    for i in range(len(probs)):
        assert stg[i]["sweeps"] == std_[i]["sweeps"]
        assert np.array_equal(mg[i], md[i]), i
    sd.close()
    sg.close()


def test_batched_iterate_budget(mmplib):
    """iterate(k) runs exactly k batched sweeps (a graph launch runs more
    sweep slots, the device budget stops them), and 2 + 3 sweeps equal 5."""
    from paper_2310_11365_gb300.mmp import Solver

    probs = [p.scaled(tol=0.0, max_iter=12) for p in _batch_problems(n=6, seed=9)]
    a = Solver(probs)
    a.lift()
    a.iterate(2)
    assert [a.status(i)["sweeps"] for i in range(len(probs))] == [min(2, p.N) for p in probs]
    a.iterate(3)
    b = Solver(probs)
    b.lift()
    b.iterate(5)
    for i, p in enumerate(probs):
        assert a.status(i)["sweeps"] == b.status(i)["sweeps"] == min(5, p.N)
        assert np.array_equal(a.moments(i), b.moments(i)), i
    a.close()
    b.close()


def test_batched_sweeps_replay_a_graph(mmplib):
    """A batched context captures its sweeps once and replays the graph
    (the cooperative launch is accepted inside stream capture)."""
    from paper_2310_11365_gb300.mmp import Solver, mmp_batch_info

    s = Solver(_batch_problems(n=4, seed=13))
    s.run()
    info = mmp_batch_info(s.ctx)
    s.close()
    assert info["batched"] and info["graph"]
