"""Pins of the rate fit where the method uses it: on Monte-Carlo-noisy
fractions (Sec. 3.6, Eq. generalised_model_multimodal_PFs; Def. 3.4).

With three or four regions the learning variant fits the rates omega_ij of
dP/dt = A P (A_ji = omega_ij, A_ii = -sum_j omega_ij) to the fractions of the
exact slice ends t_0..t_k by least squares, P(t_n) = expm(A dT)^n P(t_0),
over the box 0 <= omega <= 20 / dT (rates are non-negative, and beyond
omega dT = 20 the slice-end fractions cannot tell rates apart).  On noisy
data the result has no closed form; what fixes it is that it minimises the
cost.  These tests check that with code of their own (the generator written
out, scipy's expm, finite differences, scipy's least_squares), on the
fractions of real double-well runs of the oracle and on multinomial draws
from the model:

* the gradient of the cost vanishes in every rate strictly inside the box;
* at a bound, moving the rate into the box does not lower the cost;
* no Gauss-Newton step of an independent Jacobian on the free rates lowers
  the cost;
* scipy's bounded trust-region solver started there finds no lower cost.

The fit reports whether it converged (0) or stopped at its iteration cap
(1): on a few very noisy series the cost has a long flat valley that
Levenberg-Marquardt follows slowly.  Every fit that reports convergence must
pass the checks; the cap may be reached only rarely, and a fit stopped there
must still have lowered the cost below that of its start.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from paper_2310_11365_gb300 import workloads as W

THR = {3: dict(n_regions=3, threshold=-0.5, threshold2=0.5),
       4: dict(n_regions=4, threshold=-1.0, threshold2=0.0, threshold3=1.0)}


def generator(I, om):
    A = np.zeros((I, I))
    for i in range(I):
        others = [j for j in range(I) if j != i]
        for t, j in enumerate(others):
            w = om[i * (I - 1) + t]
            A[j, i] += w
            A[i, i] -= w
    return A


def residuals(I, theta, fr, dT):
    Phi = scipy.linalg.expm(generator(I, theta * theta) * dT)
    p = fr[0].copy()
    out = []
    for n in range(1, fr.shape[0]):
        p = Phi @ p
        out.append(fr[n] - p)
    return np.concatenate(out)


def cost(I, theta, fr, dT):
    r = residuals(I, theta, fr, dT)
    return float(r @ r)


def run_fractions(orc, I, N, seed):
    """Fractions of a double-well serial fine run (P = 2001): the data the
    learning variant fits after its sweeps."""
    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.0, s0=0.6, T=0.25 * N, N=N, dt=0.01, P=2001,
                      seed=seed, variant=W.LEARNING, tol=0.0, **THR[I])
    ser = orc.fine_serial(p)
    return np.array([[st["count"][i] / p.P for i in range(I)] for st in ser["stats"]]), 0.25


def model_fractions(I, k, seed, P=4000):
    """Multinomial draws of P particles from the rate model's fractions."""
    rng = np.random.default_rng(seed)
    om = rng.uniform(0.05, 0.8, size=I * (I - 1))
    dT = 0.25
    Phi = scipy.linalg.expm(generator(I, om) * dT)
    p = rng.dirichlet(np.ones(I) * 2)
    fr = [p]
    for _ in range(k):
        p = Phi @ p
        fr.append(rng.multinomial(P, p / p.sum()) / P)
    return np.array(fr), dT


def om_residuals(I, om, fr, dT):
    return residuals(I, np.sqrt(np.maximum(om, 0.0)), fr, dT)


def om_cost(I, om, fr, dT):
    r = om_residuals(I, om, fr, dT)
    return float(r @ r)


def check_minimum(orc, fr, dT):
    I = fr.shape[1]
    rc, om = orc.rate_fit(fr, dT)
    om_max = 20.0 / dT
    assert rc == 0 and np.all(np.isfinite(om)) and np.all(om >= 0.0) and np.all(om <= om_max)
    check_point(om, fr, dT)
    return om


def check_point(om, fr, dT):
    I = fr.shape[1]
    om_max = 20.0 / dT
    c0 = om_cost(I, om, fr, dT)
    floor = 1e-26  # an exact fit (k = I) leaves a cost at rounding level
    lower = om == 0.0
    upper = om == om_max
    inside = ~(lower | upper)
    # (1) inside the box the gradient vanishes: by central differences, a
    #     relative change of 1e-3 of any rate moves the cost, to first order,
    #     by < 1e-8 of it
    for q in np.where(inside)[0]:
        e = 1e-6 * om[q]
        up, dn = om.copy(), om.copy()
        up[q] += e
        dn[q] -= e
        gq = (om_cost(I, up, fr, dT) - om_cost(I, dn, fr, dT)) / (2 * e)
        assert abs(gq) * om[q] * 1e-3 <= 1e-8 * c0 + floor, (q, gq, om, c0)
    # (2) at a bound the cost does not fall into the box (one-sided differences)
    for q in np.where(lower | upper)[0]:
        e = 1e-7 * max(om[q], 1e-2)
        mv = om.copy()
        mv[q] += e if lower[q] else -e
        assert om_cost(I, mv, fr, dT) >= c0 * (1 - 1e-12) - floor, (q, om)
    # (3) the Gauss-Newton step of a finite-difference Jacobian on the free
    #     rates gains nothing
    r0 = om_residuals(I, om, fr, dT)
    free = np.where(inside)[0]
    if free.size:
        J = np.zeros((r0.size, free.size))
        for t, q in enumerate(free):
            e = 1e-7 * om[q]
            up, dn = om.copy(), om.copy()
            up[q] += e
            dn[q] -= e
            J[:, t] = (om_residuals(I, up, fr, dT) - om_residuals(I, dn, fr, dT)) / (2 * e)
        step = np.linalg.lstsq(J, -r0, rcond=1e-12)[0]
        predicted = float(np.sum((J @ step) ** 2))
        assert predicted <= 1e-8 * c0 + floor, (predicted, c0)
    # (4) scipy's bounded trust-region reflective solver from the returned
    #     point finds no lower cost in the box
    x0 = np.clip(om, 1e-12, om_max * (1 - 1e-12))
    ls = scipy.optimize.least_squares(lambda w: om_residuals(I, w, fr, dT), x0, bounds=(0.0, om_max),
                                      method="trf", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert 2 * ls.cost >= c0 * (1 - 1e-9) - floor, (2 * ls.cost, c0)


@pytest.mark.parametrize("I", [3, 4])
def test_fit_on_run_fractions_is_a_minimum(orc, I):
    """Fractions of an oracle run, fitted at k = I, 2I and 12 (Def. 3.4 fits
    after every sweep from k = I on)."""
    fr, dT = run_fractions(orc, I, 12, seed=77 + I)
    for k in (I, 2 * I, 12):
        check_minimum(orc, fr[: k + 1], dT)


def survey_series(orc):
    """Series like the ones the learning variant fits: fractions of oracle
    runs (P = 2001) and multinomial draws of P = 4e3, 2e4 and 1e5 particles
    from the rate model, each cut at k = I, 2I and 12."""
    out = []
    for I in (3, 4):
        for seed in range(1, 5):
            fr, dT = run_fractions(orc, I, 12, seed=500 + seed)
            out += [(fr[: k + 1], dT) for k in (I, 2 * I, 12)]
        for P in (4000, 20000, 100000):
            for seed in range(1, 4):
                fr, dT = model_fractions(I, 12, seed=1000 * I + seed, P=P)
                out += [(fr[: k + 1], dT) for k in (I, 2 * I, 12)]
    return out


def test_converged_fits_are_minima(orc):
    series = survey_series(orc)
    capped = 0
    for fr, dT in series:
        rc, om = orc.rate_fit(fr, dT)
        assert rc in (0, 1)
        if rc == 0:
            check_point(om, fr, dT)
        else:
            capped += 1
            # a capped fit still descended from its start (the rates are used)
            assert om_cost(fr.shape[1], om, fr, dT) < 0.5 * om_cost(fr.shape[1], start_rates(fr, dT), fr, dT)
    assert capped <= len(series) // 20, (capped, len(series))


def start_rates(fr, dT):
    """The fit's start, restated: the one-step regression, floored at
    1e-3 / (k dT) and capped at 1 / dT."""
    I = fr.shape[1]
    k = fr.shape[0] - 1
    X, Y = fr[:-1], fr[1:]
    Phi0 = np.linalg.solve(X.T @ X, X.T @ Y).T
    om = np.zeros(I * (I - 1))
    for i in range(I):
        for t, j in enumerate([j for j in range(I) if j != i]):
            w = Phi0[j, i] / dT
            om[i * (I - 1) + t] = min(w, 1.0 / dT) if np.isfinite(w) and w > 1e-3 / (k * dT) else 1e-3 / (k * dT)
    return om


@pytest.mark.parametrize("I", [3, 4])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_fit_on_multinomial_fractions_is_a_minimum(orc, I, seed):
    fr, dT = model_fractions(I, 12, seed=100 * I + seed)
    for k in (I, 2 * I, 12):
        rc, om = orc.rate_fit(fr[: k + 1], dT)
        if rc == 0:
            check_point(om, fr[: k + 1], dT)


def test_planted_mistakes_are_caught(orc):
    """The checks above see a fit that stops short of the minimum: rates
    moved by 1e-3 relative from the returned ones (as an early stop or a
    wrong Jacobian leaves them) fail them, and a bounded solver started
    there does find a lower cost."""
    fr, dT = run_fractions(orc, 4, 12, seed=81)
    rc, om = orc.rate_fit(fr, dT)
    assert rc == 0
    c0 = om_cost(4, om, fr, dT)
    bad = om * (1 + 1e-3 * np.linspace(-1, 1, om.size))
    cb = om_cost(4, bad, fr, dT)
    assert cb > c0
    x0 = np.clip(bad, 1e-12, None)
    ls = scipy.optimize.least_squares(lambda w: om_residuals(4, w, fr, dT), x0, bounds=(0.0, 20.0 / dT),
                                      method="trf", xtol=1e-15, ftol=1e-15, gtol=1e-15)
    assert 2 * ls.cost < cb * (1 - 1e-9)
    with pytest.raises(AssertionError):
        check_point(bad, fr, dT)
