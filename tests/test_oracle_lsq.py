"""Pins of the fraction-learning fit (Sec. 3.6, App. H)."""
import math

import numpy as np


def test_noiseless_exponential_recovered(orc):
    """Data from P(t) = beta + (P0 - beta) e^{alpha t} (App. H closed form)
    are fitted back to (alpha, beta) within 1e-10."""
    for alpha, beta, p0 in [(-0.3, 0.42, 0.9), (-1.7, 0.05, 0.5), (-0.05, 0.6, 0.1)]:
        dT = 0.25
        t = dT * np.arange(1, 9)
        y = beta + (p0 - beta) * np.exp(alpha * t)
        rc, a, b = orc.lsq_fit(t, y, p0, dT)
        assert rc == 0
        assert abs(a - alpha) < 1e-10 * max(1, abs(alpha))
        assert abs(b - beta) < 1e-10


def test_model_solves_van_kampen_ode():
    """App. H: P(t) = beta + (P0 - beta) e^{alpha t} solves
    dP/dt = alpha (P - beta), the two-state rate equation with
    alpha = -(1/tau12 + 1/tau21)."""
    alpha, beta, p0 = -0.8, 0.3, 0.7
    f = lambda t: beta + (p0 - beta) * math.exp(alpha * t)
    for t in (0.1, 1.0, 3.0):
        d = (f(t + 1e-6) - f(t - 1e-6)) / 2e-6
        assert abs(d - alpha * (f(t) - beta)) < 1e-8


def test_extrapolate(orc):
    """H(P_k, 0, theta) = P_k exactly; H -> beta as t -> infinity;
    H matches the closed form otherwise."""
    assert orc.extrapolate(0.37, -0.5, 0.2, 0.0) == 0.37
    assert abs(orc.extrapolate(0.37, -0.5, 0.2, 200.0) - 0.2) < 1e-15
    v = orc.extrapolate(0.37, -0.5, 0.2, 1.5)
    assert abs(v - (0.2 + (0.37 - 0.2) * math.exp(-0.75))) < 1e-15


def test_fit_rejects_growth(orc):
    """A fit that gives alpha >= 0 or beta outside [0, 1] is refused
    (no learning for that sweep)."""
    t = 0.25 * np.arange(1, 6)
    y = 0.1 * np.exp(0.5 * t)
    rc, _, _ = orc.lsq_fit(t, y, 0.1, 0.25)
    assert rc != 0
    assert orc.lsq_fit(t[:1], y[:1], 0.1, 0.25)[0] != 0


def test_noisy_fit_is_least_squares(orc):
    """With noise the result is a stationary point of the cost: the gradient
    of sum r^2 vanishes (checked by central differences)."""
    rng = np.random.default_rng(3)
    alpha, beta, p0, dT = -0.6, 0.35, 0.8, 0.2
    t = dT * np.arange(1, 12)
    y = beta + (p0 - beta) * np.exp(alpha * t) + rng.normal(0, 2e-3, t.size)
    rc, a, b = orc.lsq_fit(t, y, p0, dT)
    assert rc == 0
    cost = lambda a, b: np.sum((y - (b + (p0 - b) * np.exp(a * t))) ** 2)
    e = 1e-6
    ga = (cost(a + e, b) - cost(a - e, b)) / (2 * e)
    gb = (cost(a, b + e) - cost(a, b - e)) / (2 * e)
    assert abs(ga) < 1e-8 and abs(gb) < 1e-8
