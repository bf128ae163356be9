"""Pins of the oracle with more than two regions (Def. 3.2 with I = 3, 4;
Sec. 3.6's rate model of the fractions): region lookup and restriction
against numpy, the matrix exponential and its derivative against scipy, the
rate fit on noiseless data made with scipy's expm, the two-region reduction
of the rate model to App. H's form, and whole runs (Property 3.3 bit for
bit, matching never moving a particle across a region boundary)."""
import numpy as np
import pytest
import scipy.linalg

from paper_2310_11365_gb300 import workloads as W

THR3 = dict(n_regions=3, threshold=-0.5, threshold2=0.5)
THR4 = dict(n_regions=4, threshold=-1.0, threshold2=0.0, threshold3=1.0)


def _bounds(p):
    return [p.threshold, p.threshold2, p.threshold3][: p.n_regions - 1]


def _well(variant, regions, **kw):
    base = dict(m0=0.0, s0=0.6, T=2.0, N=6, dt=0.01, P=2001, seed=41, variant=variant, tol=0.0)
    base.update(kw)
    return W.double_well(0.25, 0.5, 0.1, 0.7, **base, **regions)


@pytest.mark.parametrize("regions", [THR3, THR4])
def test_region_and_restriction_against_numpy(orc, regions):
    p = _well(W.MULTIMODAL, regions)
    rng = np.random.default_rng(3)
    u = rng.normal(0.0, 1.2, size=5001)
    b = _bounds(p)
    u[: 2 * len(b)] = b + b  # particles exactly on the boundaries
    r = np.searchsorted(np.array(_bounds(p)), u, side="right")   # x >= t_i lies in D_i
    st = orc.restrict(p.scaled(P=len(u)), u)
    for i in range(p.n_regions):
        x = u[r == i]
        assert st["count"][i] == len(x)
        assert st["mean"][i] == pytest.approx(x.mean(), rel=1e-13)
        assert st["var"][i] == pytest.approx(x.var(), rel=1e-11)
        assert st["min"][i] == x.min() and st["max"][i] == x.max()


@pytest.mark.parametrize("n", [2, 3, 4, 8])
def test_expm_and_derivative_against_scipy(orc, n):
    rng = np.random.default_rng(n)
    for scale in (0.1, 3.0):  # the second needs scaling and squaring
        X = rng.normal(size=(n, n)) * scale
        D = rng.normal(size=(n, n))
        E, dE = orc.expm(X, D)
        ref = scipy.linalg.expm(X)
        assert np.max(np.abs(E - ref)) <= 1e-13 * np.max(np.abs(ref))
        # the Frechet derivative is the upper-right block of expm([[X, D], [0, X]])
        big = scipy.linalg.expm(np.block([[X, D], [np.zeros((n, n)), X]]))[:n, n:]
        assert np.max(np.abs(dE - big)) <= 1e-11 * np.max(np.abs(big))


def test_rate_generator_and_two_region_form(orc):
    om = np.array([0.3, 0.1, 0.05, 0.2, 0.4, 0.15])
    A = orc.rate_generator(3, om)
    assert np.allclose(A.sum(axis=0), 0.0, atol=1e-15)
    assert A[1, 0] == 0.3 and A[2, 0] == 0.1 and A[0, 1] == 0.05 and A[2, 1] == 0.2
    assert A[0, 2] == 0.4 and A[1, 2] == 0.15
    # I = 2: P_0(t) = beta + (P_0(0) - beta) e^{alpha t}, alpha = -(w01 + w10), beta = w10 / (w01 + w10)
    w01, w10, dT = 0.7, 0.3, 0.25
    alpha, beta = -(w01 + w10), w10 / (w01 + w10)
    for m in (1, 3, 10):
        p = orc.rate_propagate(2, [w01, w10], dT, [0.9, 0.1], m)
        assert p[0] == pytest.approx(beta + (0.9 - beta) * np.exp(alpha * m * dT), rel=1e-13)
        assert p.sum() == pytest.approx(1.0, rel=1e-15)


def _series(orc, I, k, dT=0.25):
    """Noiseless fractions of the rate model, propagated with scipy's expm."""
    rng = np.random.default_rng(10 * I + k)
    om = rng.uniform(0.05, 0.6, size=I * (I - 1))
    A = np.zeros((I, I))
    for i in range(I):
        for j in range(I):
            if i != j:
                w = om[i * (I - 1) + (j if j < i else j - 1)]
                A[j, i] += w
                A[i, i] -= w
    Phi = scipy.linalg.expm(A * dT)
    fr = [rng.dirichlet(np.ones(I))]
    for _ in range(k + 4):
        fr.append(Phi @ fr[-1])
    return om, np.array(fr), dT


@pytest.mark.parametrize("I,k", [(3, 12), (4, 12)])
def test_rate_fit_recovers_noiseless_rates(orc, I, k):
    om, fr, dT = _series(orc, I, k)
    rc, fit = orc.rate_fit(fr[: k + 1], dT)
    assert rc == 0
    assert np.max(np.abs(fit - om) / om) < 1e-9, (fit, om)
    rc, _ = orc.rate_fit(fr[:I], dT)  # k = I - 1: too few points
    assert rc == -1


@pytest.mark.parametrize("I,k", [(3, 3), (3, 6), (4, 4), (4, 8)])
def test_rate_fit_on_short_series_predicts(orc, I, k):
    """With few points the rates are only weakly determined, but the fitted
    model reproduces the series and extrapolates it (Def. 3.4's use)."""
    om, fr, dT = _series(orc, I, k)
    rc, fit = orc.rate_fit(fr[: k + 1], dT)
    assert rc == 0 and np.all(fit >= 0.0)
    for n in range(1, k + 5):
        pred = orc.rate_propagate(I, fit, dT, fr[0], n)
        assert np.max(np.abs(pred - fr[n])) < (1e-5 if n <= k else 1e-4), n
        assert pred.sum() == pytest.approx(1.0, abs=1e-14)


@pytest.mark.parametrize("variant", [W.MULTIMODAL, W.LEARNING])
@pytest.mark.parametrize("regions", [THR3, THR4])
def test_property_3_3_bitwise(orc, variant, regions):
    """After k sweeps the iterate equals the serial fine run on slices 0..k:
    particles bit for bit, each region's (fraction, mean, variance) bit for
    bit, and the global moments (a mixture of the regions') to rounding."""
    p = _well(variant, regions)
    ser = orc.fine_serial(p, want_parts=True)
    for k in (3, p.N):
        r = orc.parareal(p.scaled(max_iter=k), want_parts=True)
        assert r["sweeps"] == k
        for n in range(k + 1):
            assert np.array_equal(r["parts"][n], ser["parts"][n]), (k, n)
            st = ser["stats"][n]
            for i in range(p.n_regions):
                assert r["frac"][n][i] == st["count"][i] / p.P
                if st["count"][i] > 0:
                    assert r["mean"][n][i] == st["mean"][i] and r["var"][n][i] == st["var"][i]
            M, V = r["hist"][k, n]
            assert abs(M - ser["gmean"][n]) < 1e-14 and abs(V - ser["gvar"][n]) < 1e-13


@pytest.mark.parametrize("regions", [THR3, THR4])
def test_matching_keeps_every_particle_in_its_region(orc, regions):
    """Def. 3.2: a region is moved only if none of its particles leaves it,
    so the fractions of every matched iterate are those of the fine outputs
    it was made from; with a middle region both of its boundaries bind and
    some updates are refused."""
    p = _well(W.MULTIMODAL, regions, max_iter=2)
    r = orc.parareal(p, want_parts=True)
    assert r["sweeps"] == 2 and r["accepted"] > 0 and r["rejected"] > 0
    bounds = np.array(_bounds(p))
    for n in range(1, p.N + 1):
        counts = np.bincount(np.searchsorted(bounds, r["parts"][n], side="right"), minlength=p.n_regions)
        assert np.array_equal(counts / p.P, r["frac"][n][: p.n_regions]), n


def test_learning_with_three_regions_moves_the_iterates(orc):
    """The rate model is fitted from sweep k = I on and changes the global
    moments beyond t_k, without touching the exact slices."""
    base = dict(N=8, T=4.0, max_iter=4)
    lrn = orc.parareal(_well(W.LEARNING, THR3, **base))
    mm = orc.parareal(_well(W.MULTIMODAL, THR3, **base))
    k = 3
    assert np.array_equal(lrn["hist"][k - 1], mm["hist"][k - 1])  # no fit before k = I
    assert not np.allclose(lrn["hist"][k][k + 1:], mm["hist"][k][k + 1:], rtol=1e-12, atol=0)
    assert np.array_equal(lrn["hist"][k][: k + 1], mm["hist"][k][: k + 1])
