"""Pins of the oracle's fine propagator (Euler-Maruyama with mean field,
Sec. 1.2 Eq. Euler_Maruyama) against closed forms that do not reuse its code.
"""
import math

import numpy as np

from paper_2310_11365_gb300 import workloads as W


def _normals(orc, p, n, j):
    return np.array([orc.normal(p, 0, j, n, i) for i in range(p.P)])


def test_fine_step_count(orc):
    """n_f = ceil(T/(N dt)) equal steps that end exactly on the slice end."""
    assert orc.fine_steps(W.config1()) == 125
    assert orc.fine_steps(W.config2()) == 125
    p3 = W.config3()
    assert orc.fine_steps(p3) == 313
    assert abs(orc.fine_h(p3) * 313 - p3.T / p3.N) < 1e-15
    assert orc.fine_steps(W.config1(dt=0.25 / 7)) == 7


def test_linear_sample_path_identities(orc):
    """Linear model, same draws: the ensemble mean obeys
    m_{j+1} = (1 - theta h) m_j + sigma sqrt(h) mean_p(xi_j) and the
    deviations d = x - m obey d_{j+1} = (1 - (theta+kappa) h) d_j
    + sigma sqrt(h) (xi_j - mean(xi_j)) (exact algebra of Lemma 2.1's SDE)."""
    theta, kappa, sigma = 1.0, 0.5, 0.5
    p = W.linear(theta, kappa, sigma, m0=1.0, s0=0.1, T=0.1, N=1, dt=0.01, P=37, seed=99)
    u0 = orc.initial(p)
    nf, h = orc.fine_steps(p), orc.fine_h(p)
    out, means = orc.fine(p, 0, u0, return_means=True)
    m = u0.mean()
    d = u0 - m
    for j in range(nf):
        xi = _normals(orc, p, 0, j)
        assert abs(means[j] - m) < 1e-14
        m = (1 - theta * h) * m + sigma * math.sqrt(h) * xi.mean()
        d = (1 - (theta + kappa) * h) * d + sigma * math.sqrt(h) * (xi - xi.mean())
    assert np.allclose(out, m + d, rtol=0, atol=1e-13)
    assert abs(means[nf] - m) < 1e-14


def test_linear_ensemble_average_over_seeds(orc):
    """Averaged over independent seeds, E m_j = m0 (1 - theta h)^j and
    E V_{j+1} = c^2 E V_j + sigma^2 h (P-1)/P with c = 1 - (theta+kappa) h
    (population variance); within 4 standard errors."""
    theta, kappa, sigma = 1.0, 0.5, 0.5
    P, S = 64, 300
    base = W.linear(theta, kappa, sigma, m0=1.0, s0=0.1, T=0.4, N=1, dt=0.02, P=P)
    nf, h = orc.fine_steps(base), orc.fine_h(base)
    ms, vs = [], []
    for s in range(S):
        p = base.scaled(seed=1000 + s)
        out = orc.fine(p, 0, orc.initial(p))
        ms.append(out.mean())
        vs.append(out.var())
    ms, vs = np.array(ms), np.array(vs)
    c = 1 - (theta + kappa) * h
    ev = base.s0**2 * (P - 1) / P  # E of the initial population variance
    for _ in range(nf):
        ev = c * c * ev + sigma**2 * h * (P - 1) / P
    em = base.m0 * (1 - theta * h) ** nf
    # the initial mean itself is random: Var = s0^2/P, then the noise adds up
    assert abs(ms.mean() - em) < 4 * ms.std(ddof=1) / math.sqrt(S)
    assert abs(vs.mean() - ev) < 4 * vs.std(ddof=1) / math.sqrt(S)


def test_cubic_drift_against_ode_solution(orc):
    """sigma = 0 and one particle: EM integrates dx/dt = -x^3 (cubic model,
    kappa terms cancel since m = x); exact x(t) = x0 / sqrt(1 + 2 x0^2 t).
    First-order convergence in h pins the sign and power of the cubic."""
    errs = []
    for dt in (1e-3, 5e-4):
        p = W.cubic(1.0, 0.0, m0=1.3, s0=0.0, T=1.0, N=1, dt=dt, P=1)
        x1 = orc.fine(p, 0, np.array([1.3]))[0]
        exact = 1.3 / math.sqrt(1 + 2 * 1.3**2 * 1.0)
        errs.append(abs(x1 - exact))
    assert errs[0] < 2e-3
    assert 1.7 < errs[0] / errs[1] < 2.3


def test_double_well_drift_against_ode_solution(orc):
    """sigma = 0, one particle in V = x^4/4 - x^2/2: dx/dt = x - x^3, whose
    solution is x(t) = x0 e^t / sqrt(1 + x0^2 (e^{2t} - 1))."""
    x0 = 0.2
    p = W.double_well(0.25, 0.5, 0.3, 0.0, m0=x0, T=2.0, N=1, dt=1e-4, P=1)
    x1 = orc.fine(p, 0, np.array([x0]))[0]
    e = math.exp(2.0)
    exact = x0 * math.exp(2.0) / math.sqrt(1 + x0 * x0 * (e * e - 1))
    assert abs(x1 - exact) < 1e-3


def test_multiplicative_noise_one_step_variance(orc):
    """One EM step with b = B x + BE m + B0: Var(X_1) = (1 + h c1)^2 Var(X_0)
    + h E[b^2], E[b^2] = B^2 v0 + (B m0 + BE m0 + B0)^2 (to O(1/P))."""
    P = 200_000
    p = W.Problem(c1=-0.7, kappa=0.2, B=0.6, BE=-0.3, B0=0.4, m0=0.8, s0=0.5, T=0.05, N=1,
                  dt=0.05, P=P, seed=5)
    u0 = orc.initial(p)
    h = orc.fine_h(p)
    out = orc.fine(p, 0, u0)
    v0, m0 = u0.var(), u0.mean()
    eb2 = p.B**2 * v0 + (p.B * m0 + p.BE * m0 + p.B0) ** 2
    expect = (1 + h * p.c1) ** 2 * v0 + h * eb2
    se = expect * math.sqrt(2.0 / P) * 2
    assert abs(out.var() - expect) < 4 * se


def test_mean_field_couples_particles(orc):
    """Moving one particle changes the others' next step through m_j
    (kappa h / P per unit moved), and nothing else does."""
    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=0.001, N=1, dt=0.001, P=9, seed=3)
    u0 = orc.initial(p)
    u1 = u0.copy()
    u1[4] += 0.9
    a = orc.fine(p, 0, u0)
    b = orc.fine(p, 0, u1)
    h = orc.fine_h(p)
    others = np.arange(9) != 4
    assert np.allclose(b[others] - a[others], p.kappa * h * 0.9 / 9, rtol=1e-9, atol=0)
