"""The seeded workload records against the recipes they state: model
coefficients from each model's parameters, sizes, seeds, and the draws of
the 512-problem batch.  Records only: no arithmetic of the method."""
import math

import numpy as np

from paper_2310_11365_gb300 import workloads as W


def _nf(p):
    return math.ceil(p.T / p.N / p.dt - 1e-9)


def test_model_constructors():
    lin = W.linear(1.0, 0.5, 0.5)
    assert (lin.c3, lin.c1, lin.kappa, lin.c0, lin.B0) == (0.0, -1.5, 0.5, 0.0, 0.5)  # -theta X + kappa (m - X)
    cub = W.cubic(1.0, 0.5)
    assert (cub.c3, cub.c1, cub.kappa, cub.B0) == (1.0, -1.0, 1.0, 0.5)               # -X^3 + kappa (m - X)
    dw = W.double_well(0.25, 0.5, 0.1, 0.7)
    assert (dw.c3, dw.c1, dw.kappa, dw.B0) == (1.0, 1.0 - 0.1, 0.1, 0.7)              # -V'(X) + kappa (m - X)
    assert all(p.family == W.POLY for p in (lin, cub, dw))


def test_the_five_configurations():
    c1, c2, c3, c4 = W.config1(), W.config2(), W.config3(), W.config4()
    assert (c1.P, c1.N, c1.T, _nf(c1), c1.precision, c1.tol) == (2000, 16, 4.0, 125, "fp64", 1e-8)
    assert (c1.m0, c1.s0) == (1.0, 0.1)
    assert (c2.P, c2.N, c2.T, _nf(c2), c2.precision, c2.tol) == (1_000_000, 64, 8.0, 125, "mixed", 1e-6)
    assert (c2.m0, c2.s0) == (0.5, 0.2)
    assert (c3.P, c3.N, c3.T, _nf(c3), c3.n_regions, c3.threshold, c3.variant) == (
        4_000_000, 128, 20.0, 313, 2, 0.0, W.LEARNING)
    assert (c4.P, c4.N, c4.T, _nf(c4), c4.n_regions) == (1_000_000, 64, 20.0, 313, 1)
    assert [p.seed - W.SEED_BASE for p in (c1, c2, c3, c4)] == [1, 2, 3, 4]
    assert W.config2(P=10).P == 10 and W.config2().P == 1_000_000  # overrides return copies


def test_the_batch_recipe():
    """512 problems: even ones of the linear form, odd ones of the two-region
    learning double well; theta in [0.5, 2], kappa in [0, 1], sigma in
    [0.3, 1], P log-uniform in [1e4, 2e6], N in 16..128, T = 8, dt = 1e-3,
    mixed, problem tag = index, one seed; the same list on every call."""
    b = W.config5()
    assert len(b) == 512 and b == W.config5()
    for i, p in enumerate(b):
        assert p.problem_tag == i and p.seed == W.SEED_BASE + 5
        assert (p.T, p.dt, p.precision, p.tol) == (8.0, 1e-3, "mixed", 1e-6)
        assert 16 <= p.N <= 128 and 10_000 <= p.P <= 2_000_000
        assert 0.0 <= p.kappa <= 1.0 and 0.3 <= p.B0 <= 1.0
        if i % 2 == 0:
            theta = -p.c1 - p.kappa
            assert p.c3 == 0.0 and 0.5 <= theta <= 2.0 and p.n_regions == 1 and (p.m0, p.s0) == (1.0, 0.1)
        else:
            assert p.c3 == 1.0 and p.n_regions == 2 and p.variant == W.LEARNING and (p.m0, p.s0) == (0.0, 0.3)
    logp = np.log10([p.P for p in b])
    assert abs(logp.mean() - (4.0 + math.log10(2e6)) / 2) < 0.1  # log-uniform
    total = sum(p.P for p in b)
    assert 1.5e8 < total < 2.5e8


def test_the_paper_examples():
    g = W.gbm()
    s = 0.5 * math.sqrt(0.5)
    assert (g.c1, g.kappa, g.c0, g.B, g.BE, g.B0, g.m0, g.s0, g.N) == (-0.5, 0.8, 1.0 / 3.0, s, s, 1.0 / 6.0, 1.0, 0.5, 10)
    r = W.plane_rotator()
    assert r.family == W.ROTATOR and (r.K, r.g, r.T, r.dt, r.P, r.N) == (1.0, 1.0, 10.0, 1e-3, 100_000, 10)
    assert r.m0 == math.pi / 4 and abs(r.s0 ** 2 - 3 * math.pi / 4) < 1e-15 and abs(r.B0 ** 2 - 0.5) < 1e-15
