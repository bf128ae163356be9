"""Checkpoint and resume: a run saved after some sweeps and resumed in a new
context (another workspace) ends bit for bit where the uninterrupted run
ends, for one problem and for a batch; a checkpoint of other problems is
refused."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _resume_equals_uninterrupted(problems, k_save):
    from paper_2310_11365_gb300.mmp import Solver

    problems = problems if isinstance(problems, list) else [problems]
    a = Solver(problems)
    a.lift()
    a.iterate(k_save)
    blob = a.state()
    while not a.iterate(1):
        pass
    b = Solver(problems)  # a fresh context and workspace
    b.restore(blob)
    while not b.iterate(1):
        pass
    for i in range(len(problems)):
        assert a.status(i)["sweeps"] == b.status(i)["sweeps"]
        assert np.array_equal(a.moments(i), b.moments(i)), i
    a.close()
    b.close()


def test_resume_one_problem(mmplib):
    p = W.config2(P=50_000, N=8, T=1.0, precision="mixed", tol=1e-7)
    _resume_equals_uninterrupted(p, 3)


def test_resume_a_batch(mmplib):
    probs = [W.config1(N=6, T=1.5, problem_tag=1),
             W.config3(N=6, T=1.5, dt=5e-3, P=4001, precision="fp64", problem_tag=2)]
    _resume_equals_uninterrupted(probs, 2)


def test_checkpoint_of_other_problems_is_refused(mmplib):
    from paper_2310_11365_gb300.mmp import MMPError, Solver

    a = Solver(W.config1(N=4, T=1.0))
    a.lift()
    blob = a.state()
    b = Solver(W.config1(N=4, T=1.0, kappa=0.6))
    with pytest.raises(MMPError) as e:
        b.restore(blob)
    assert "STATE" in str(e.value)
    a.close()
    b.close()
