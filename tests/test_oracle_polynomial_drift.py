"""Pins of the polynomial-drift example (App. C, after Son Doan et al.):
dX = (alpha X + E[X] - X E[X^2]) dt + X dW, X(0) = 1.

The appendix shows that the Taylor moment model (Eq. moment_model_class_1)
is exact for this SDE: with S = E[X^2] it reproduces the exact moment system
dM/dt = (alpha + 1) M - M S, dS/dt = (2 alpha + 1) S + 2 M^2 - 2 S^2.  The
oracle carries the example's coupling to E[X^2] as the drift term
-q2 x E[X^2].  Checked here:

* every coarse model of the oracle, at any (M, Sigma), equals the exact
  system (written out from the appendix, converted with S = Sigma + M^2);
* one Euler-Maruyama step of the oracle, re-derived by hand for three
  particles from the oracle's own draws;
* exact sample-path identities of the fine propagator: the ensemble mean and
  second moment after a step, from those before it and the draws' averages;
* the Monte Carlo moments of a fine run against the exact system solved by
  scipy, within their statistical and time-step errors;
* the Parareal iteration with the Taylor and closure coarse models:
  Property 3.3 bit for bit.
"""
import numpy as np
import pytest
import scipy.integrate

from paper_2310_11365_gb300 import workloads as W

ALPHA = -0.5


def exact_rhs(alpha, M, S):
    return (alpha + 1.0) * M - M * S, (2 * alpha + 1.0) * S + 2 * M * M - 2 * S * S


@pytest.mark.parametrize("model", [W.CLOSURE, W.TAYLOR, W.SIGMA2, W.SIGMA3, W.TAYLOR1])
def test_every_coarse_model_is_the_exact_moment_system(orc, model):
    p = W.polynomial_drift(ALPHA, coarse_model=model)
    rng = np.random.default_rng(5)
    for _ in range(20):
        M, V = rng.uniform(-2, 2), rng.uniform(0.0, 3.0)
        dm, dv = orc.coarse_rhs(p, [1.0], [M], [V])
        dM, dS = exact_rhs(ALPHA, M, V + M * M)
        assert dm[0] == pytest.approx(dM, rel=1e-13, abs=1e-13)
        assert dv[0] + 2 * M * dm[0] == pytest.approx(dS, rel=1e-13, abs=1e-13)


def test_coupling_term_is_needed(orc):
    """Without the -X E[X^2] term the model is no longer the exact system."""
    p = W.polynomial_drift(ALPHA, q2=0.0)
    dm, dv = orc.coarse_rhs(p, [1.0], [0.7], [0.4])
    dM, dS = exact_rhs(ALPHA, 0.7, 0.4 + 0.49)
    assert abs(dm[0] - dM) > 0.1


def test_one_step_by_hand(orc):
    """x' = x + h (alpha x + m - x s) + sqrt(h) x xi with m, s the ensemble
    mean and mean square before the step, for three particles."""
    p = W.polynomial_drift(ALPHA, P=3, N=1, T=1e-2, dt=1e-2)
    u = np.array([0.9, 1.3, -0.4])
    out = orc.fine(p, 0, u)
    h = orc.fine_h(p)
    m, s = u.mean(), (u * u).mean()
    xi = np.array([orc.normal(p, 0, 0, 0, q) for q in range(3)])
    want = u + h * (ALPHA * u + m - u * s) + np.sqrt(h) * u * xi
    assert np.max(np.abs(out - want)) < 1e-15


def test_sample_path_identities(orc):
    """After one step, exactly (to rounding): m' = m + h ((alpha + 1) m - m s)
    + sqrt(h) <x xi>, and s' = <(x + h a + sqrt(h) x xi)^2> expanded:
    s' = s + 2 h <x a> + h^2 <a^2> + h <x^2 xi^2> + 2 sqrt(h) <x^2 xi> + 2 h^1.5 <a x xi>,
    where <x a> = alpha s + m^2 - s^2 (no particle-wise quantity but the draws)."""
    p = W.polynomial_drift(ALPHA, P=4001, N=1, T=1e-3, dt=1e-3)
    rng = np.random.default_rng(9)
    u = rng.normal(0.8, 0.5, p.P)
    out = orc.fine(p, 0, u)
    h = orc.fine_h(p)
    xi = np.array([orc.normal(p, 0, 0, 0, q) for q in range(p.P)])
    m, s = u.mean(), (u * u).mean()
    a = ALPHA * u + m - u * s
    m1 = m + h * ((ALPHA + 1) * m - m * s) + np.sqrt(h) * (u * xi).mean()
    assert abs(out.mean() - m1) < 1e-14
    xa = ALPHA * s + m * m - s * s
    s1 = (s + 2 * h * xa + h * h * (a * a).mean() + h * (u * u * xi * xi).mean()
          + 2 * np.sqrt(h) * (u * u * xi).mean() + 2 * h ** 1.5 * (a * u * xi).mean())
    assert abs((out * out).mean() - s1) < 1e-13


def test_monte_carlo_moments_follow_the_exact_system(orc):
    """The fine run's mean and second moment against the exact moment system
    (scipy, rtol 1e-12): within 5 standard errors plus the Euler-Maruyama
    bias, which is first order in h (the run with half the step halves it)."""
    p = W.polynomial_drift(ALPHA, P=40_000, N=4, T=0.8, dt=2e-3)
    ser = orc.fine_serial(p, want_parts=True)
    sol = scipy.integrate.solve_ivp(lambda t, y: exact_rhs(ALPHA, *y), (0.0, p.T), [1.0, 1.0],
                                    t_eval=np.linspace(0.0, p.T, p.N + 1), rtol=1e-12, atol=1e-14)
    for n in range(1, p.N + 1):
        x = ser["parts"][n]
        M, S = sol.y[0, n], sol.y[1, n]
        se_m = x.std() / np.sqrt(p.P)
        se_s = (x * x).std() / np.sqrt(p.P)
        assert abs(x.mean() - M) < 5 * se_m + 0.02 * p.dt * 10, (n, x.mean(), M)
        assert abs((x * x).mean() - S) < 5 * se_s + 0.02 * p.dt * 10, (n, (x * x).mean(), S)


@pytest.mark.parametrize("model", [W.TAYLOR, W.CLOSURE])
def test_parareal_is_exact_on_converged_slices(orc, model):
    """Property 3.3 with the coupling: after k sweeps the slice ends
    t_0..t_k equal the serial fine run bit for bit; at k = N everything does."""
    p = W.polynomial_drift(ALPHA, P=2001, N=5, T=0.5, dt=5e-3, coarse_model=model, tol=0.0)
    ser = orc.fine_serial(p, want_parts=True)
    for k in (2, p.N):
        r = orc.parareal(p.scaled(max_iter=k), want_parts=True)
        for n in range(k + 1):
            assert np.array_equal(r["parts"][n], ser["parts"][n]), (k, n)


def test_library_refuses_the_coupling(orc):
    from paper_2310_11365_gb300 import mmp

    with pytest.raises(mmp.MMPError):
        mmp.desc(W.polynomial_drift())
