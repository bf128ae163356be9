"""Pins of the oracle's plane rotator (Sec. 5, Example "Unimodal plane
rotator", Eq. SDE_plane_rotator, Eq. plane_rotator_third_order): the fine
step against the paper's pairwise sum written out, exact sample-path
identities (two particles; pure noise), rotation equivariance, the wrapped
normal law, the coarse models against quadrature and closed forms, and
Property 3.3 of the whole iteration."""
import math

import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

TWO_PI = 2.0 * math.pi


def _circ(a, b):
    """Distance on the circle of circumference 2 pi."""
    d = np.abs(np.asarray(a) - np.asarray(b)) % TWO_PI
    return np.minimum(d, TWO_PI - d)


def _draws(orc, p, j, n):
    return np.array([orc.normal(p, 0, j, n, q) for q in range(p.P)])


def test_wrap_is_a_shift_into_the_centred_interval(orc):
    """x - wrap(x) is a whole number of turns and wrap(x) lies in [-pi, pi]
    (reading: centred on the stable point 0 of -sin x); the initial ensemble
    is wrapped too."""
    xs = [-50.0, -TWO_PI, -math.pi - 1e-15, -math.pi, -1e-17, 0.0, 1e-17, 1.0, math.pi - 1e-15, math.pi,
          TWO_PI, 7.0, 1234.5]
    for x in xs:
        w = orc.wrap(x)
        assert -math.pi <= w <= math.pi, x
        turns = (x - w) / TWO_PI
        assert abs(turns - round(turns)) < 1e-12, x
    assert orc.wrap(1.0) == 1.0 and orc.wrap(-1.0) == -1.0
    assert orc.wrap(1.0 + TWO_PI) == pytest.approx(1.0, abs=1e-15)
    assert orc.wrap(4.0) == pytest.approx(4.0 - TWO_PI, abs=1e-15)
    p = W.plane_rotator(P=5000)
    u0 = orc.initial(p)
    assert u0.min() >= -math.pi and u0.max() <= math.pi
    raw = p.m0 + p.s0 * np.array([orc.normal(p, 1, 0, 0, q) for q in range(200)])
    assert np.max(_circ(u0[:200], raw)) < 1e-14
    assert np.any(raw > math.pi)  # the wrap did move some particles


@pytest.mark.parametrize("n", [0, 1])
def test_fine_steps_equal_the_pairwise_sum(orc, n):
    """Brute force on a tiny ensemble: each Euler-Maruyama step with the
    paper's (K/P) sum_q sin(X_q - X_p) summed pair by pair, then the shift
    modulo 2 pi, on the oracle's draws of slice n."""
    p = W.plane_rotator(P=7, N=2, T=0.02, dt=0.004, K=1.3, g=0.8, B0=0.9)
    nf, h = orc.fine_steps(p), orc.fine_h(p)
    assert nf == 3
    u0 = orc.initial(p)
    x = u0.copy()
    for j in range(nf):
        z = _draws(orc, p, j, n)
        coup = np.array([p.K / p.P * sum(math.sin(x[q] - x[i]) for q in range(p.P)) for i in range(p.P)])
        x = x + (coup - p.g * np.sin(x)) * h + p.B0 * math.sqrt(h) * z
        x = x - TWO_PI * np.floor((x + math.pi) / TWO_PI)
    assert np.max(_circ(orc.fine(p, n, u0), x)) < 1e-13


def test_two_particles_without_noise(orc):
    """P = 2, g = 0, no noise: the increments of the two particles cancel, so
    X_1 + X_2 stays fixed (mod 2 pi), and the difference d follows
    d_{j+1} = d_j - h K sin d_j exactly (up to rounding)."""
    p = W.plane_rotator(P=2, N=3, T=0.6, dt=0.01, K=2.0, g=0.0, B0=0.0)
    nf, h = orc.fine_steps(p), orc.fine_h(p)
    parts = orc.fine_serial(p, want_parts=True)["parts"]
    s0 = parts[0, 0] + parts[0, 1]
    d = parts[0, 0] - parts[0, 1]
    for n in range(1, p.N + 1):
        for _ in range(nf):
            d = d - h * p.K * math.sin(d)
        assert _circ(parts[n, 0] + parts[n, 1], s0) < 1e-13, n
        assert _circ(parts[n, 0] - parts[n, 1], d) < 1e-13, n
    assert abs(math.sin(d)) < abs(math.sin(parts[0, 0] - parts[0, 1]))  # they approach each other


def test_rotation_equivariance_without_pinning(orc):
    """With g = 0 the drift depends on differences only: rotating the initial
    ensemble by c rotates the result by c (same draws).  The pinning term
    -g sin x breaks it."""
    c = 0.7
    p = W.plane_rotator(P=501, N=1, T=0.2, dt=0.004, K=1.5, g=0.0, B0=0.5)
    u0 = orc.initial(p)
    u0c = np.array([orc.wrap(x + c) for x in u0])
    a = orc.fine(p, 0, u0)
    b = orc.fine(p, 0, u0c)
    assert np.max(_circ(b, a + c)) < 1e-11
    q = p.scaled(g=1.0)
    assert np.max(_circ(orc.fine(q, 0, u0c), orc.fine(q, 0, u0) + c)) > 1e-3


def test_pure_noise_path_and_wrapped_normal_law(orc):
    """K = g = 0: X_n = wrap(X_0 + B0 sqrt(h) sum_j xi_j) path by path, and the
    ensemble is a sample of the wrapped normal law WN(m0, s0^2 + B0^2 t) on
    [-pi, pi]: its mean and variance (by image sums) within 5 standard errors.
    With m0 = 2.5 about a quarter of the law lies beyond pi, so the interval
    convention matters."""
    p = W.plane_rotator(P=4, N=2, T=0.1, dt=0.01, K=0.0, g=0.0, B0=0.8)
    nf, h = orc.fine_steps(p), orc.fine_h(p)
    parts = orc.fine_serial(p, want_parts=True)["parts"]
    x = parts[0].copy()
    for n in range(p.N):
        for j in range(nf):
            x = x + p.B0 * math.sqrt(h) * _draws(orc, p, j, n)
        assert np.max(_circ(parts[n + 1], x)) < 1e-13

    big = W.plane_rotator(P=40_000, N=1, T=0.5, dt=0.05, K=0.0, g=0.0, B0=1.0, m0=2.5, s0=0.5)
    u = orc.fine(big, 0, orc.initial(big))
    s2 = big.s0 ** 2 + big.B0 ** 2 * big.T
    xg = np.linspace(-math.pi, math.pi, 200_001)
    dens = sum(np.exp(-(xg - big.m0 + TWO_PI * k) ** 2 / (2 * s2)) for k in range(-8, 9)) / math.sqrt(2 * math.pi * s2)
    mass = np.trapezoid(dens, xg)
    mean = np.trapezoid(xg * dens, xg)
    var = np.trapezoid((xg - mean) ** 2 * dens, xg)
    assert abs(mass - 1.0) < 1e-9
    se_m = math.sqrt(var / big.P)
    fourth = np.trapezoid((xg - mean) ** 4 * dens, xg)
    se_v = math.sqrt((fourth - var ** 2) / big.P)
    assert abs(u.mean() - mean) < 5 * se_m
    assert abs(u.var() - var) < 5 * se_v


@pytest.mark.parametrize("m,v", [(0.3, 0.05), (1.2, 0.4), (2.9, 1.1), (4.0, 2.5), (5.9, 0.01)])
def test_closure_against_gauss_hermite(orc, m, v):
    """Gaussian closure: dm = E[a(X)], dv = 2 E[(X - m) a(X)] + B0^2 under
    X ~ N(m, v), with S = E sin X and C = E cos X under the same law, by
    120-point Gauss-Hermite quadrature."""
    p = W.plane_rotator(K=1.4, g=0.9, B0=0.6, coarse_model=W.CLOSURE)
    t, w = np.polynomial.hermite_e.hermegauss(120)
    w = w / math.sqrt(2 * math.pi)
    X = m + math.sqrt(v) * t
    S, C = np.sum(w * np.sin(X)), np.sum(w * np.cos(X))
    a = p.K * (S * np.cos(X) - C * np.sin(X)) - p.g * np.sin(X)
    dm, dv = orc.coarse_rhs(p, [1.0], [m], [v])
    assert abs(dm[0] - np.sum(w * a)) < 1e-13
    assert abs(dv[0] - (2 * np.sum(w * (X - m) * a) + p.B0 ** 2)) < 1e-13


@pytest.mark.parametrize("m,v", [(0.3, 0.05), (1.2, 0.4), (2.9, 1.1), (4.0, 2.5)])
def test_sigma_point_rules_in_closed_form(orc, m, v):
    """The 2- and 3-point rules applied to every expectation, S and C
    included, reduce to closed forms: with d the offset and c the rule's
    mean of cos(offset) (cos d; 2/3 + cos d / 3), a(m +- d) = -+K c sin d -
    g sin(m +- d), so dm = -g c sin m and
    dv = -4 w d sin d (K c + g cos m) + B0^2 with w the outer weight (1/2; 1/6)."""
    p = W.plane_rotator(K=1.4, g=0.9, B0=0.6)
    for model, d, c, w in ((W.SIGMA2, math.sqrt(v), math.cos(math.sqrt(v)), 0.5),
                           (W.SIGMA3, math.sqrt(3 * v), 2 / 3 + math.cos(math.sqrt(3 * v)) / 3, 1 / 6)):
        dm, dv = orc.coarse_rhs(p.scaled(coarse_model=model), [1.0], [m], [v])
        assert abs(dm[0] - (-p.g * c * math.sin(m))) < 1e-14, model
        want = -4 * w * d * math.sin(d) * (p.K * c + p.g * math.cos(m)) + p.B0 ** 2
        assert abs(dv[0] - want) < 1e-14, model


@pytest.mark.parametrize("m,v", [(0.3, 0.05), (2.0, 0.7), (4.5, 1.3)])
def test_taylor_models_against_the_paper(orc, m, v):
    """Eq. plane_rotator_third_order (g = 1): dM = -sin M + (Sigma/2) sin M and,
    read with the sign of Eq. moment_model_class_1,
    dSigma = 2 (-K - cos M) Sigma + B0^2; the first coarse model of the example
    drops the Sigma term of the mean."""
    p = W.plane_rotator(K=1.7, g=1.0, B0=0.6)
    dm, dv = orc.coarse_rhs(p.scaled(coarse_model=W.TAYLOR), [1.0], [m], [v])
    assert abs(dm[0] - (-math.sin(m) + 0.5 * v * math.sin(m))) < 1e-15
    assert abs(dv[0] - (2 * (-p.K - math.cos(m)) * v + p.B0 ** 2)) < 1e-14
    dm1, dv1 = orc.coarse_rhs(p.scaled(coarse_model=W.TAYLOR1), [1.0], [m], [v])
    assert abs(dm1[0] + math.sin(m)) < 1e-15 and dv1[0] == dv[0]


def test_taylor_is_the_small_variance_limit_of_the_closure(orc):
    """The closure's right-hand side minus the Taylor model's is O(v^2) at
    fixed m (the Taylor model expands the Gaussian expectations to first
    order in v)."""
    p = W.plane_rotator(K=1.2, g=0.8, B0=0.5)
    m = 1.1
    errs = []
    for v in (0.02, 0.01, 0.005):
        a = np.array(orc.coarse_rhs(p.scaled(coarse_model=W.CLOSURE), [1.0], [m], [v]))[:, 0]
        b = np.array(orc.coarse_rhs(p.scaled(coarse_model=W.TAYLOR), [1.0], [m], [v]))[:, 0]
        errs.append(np.abs(a - b))
    ratios = errs[0] / errs[1], errs[1] / errs[2]
    for r in ratios:
        assert np.all((r > 3.6) & (r < 4.4)), ratios


@pytest.mark.parametrize("model", [W.CLOSURE, W.TAYLOR, W.TAYLOR1, W.SIGMA2, W.SIGMA3])
def test_property_3_3_with_the_rotator(orc, model):
    """After k sweeps the slice ends t_0..t_k equal the serial fine run bit
    for bit, for each coarse model; at k = N all of them do.  Only fine
    outputs are shifted into [-pi, pi]: the matching T is affine and is not
    followed by a shift (that would break S(T(rho, u)) = rho, Lemma 3.1), so
    a matched iterate beyond t_k may leave the interval until its next fine
    step."""
    p = W.plane_rotator(P=1001, N=4, T=1.0, dt=0.01, coarse_model=model, tol=0.0)
    serial = orc.fine_serial(p, want_parts=True)["parts"]
    assert serial.min() >= -math.pi and serial.max() <= math.pi
    for k in (1, 2, p.N):
        res = orc.parareal(p.scaled(max_iter=k), want_parts=True)
        assert res["sweeps"] == k
        for n in range(k + 1):
            assert np.array_equal(res["parts"][n], serial[n]), (k, n)


def test_rotator_limits_are_refused(orc):
    """The rotator has one region and no adjoint in the oracle."""
    with pytest.raises(ValueError):
        orc.parareal(W.plane_rotator(P=101, N=2, T=0.1, n_regions=2, variant=W.MULTIMODAL))
    with pytest.raises(ValueError):
        orc.adjoint(W.plane_rotator(P=101, N=2, T=0.1), np.ones(2), np.ones(2))


def test_reaches_the_statistical_error_in_a_few_sweeps(orc):
    """The example's finding: with each of its four coarse solvers (Taylor
    without the Sigma term of the mean, Taylor, 2 and 3 sigma points) the
    iteration reaches the statistical error in a few sweeps.  Here, on the
    same draws as the serial fine run (the iteration's limit), the error of
    the global mean and variance after two sweeps is below one statistical
    unit (sqrt(V/P) and V sqrt(2/P)), while the coarse-only iterate k = 0 is
    above it.  P = 2000, dt = 1e-2, otherwise the example's sizes."""
    for model in (W.TAYLOR1, W.TAYLOR, W.SIGMA2, W.SIGMA3):
        p = W.plane_rotator(P=2000, dt=1e-2, coarse_model=model, tol=0.0)
        ser = orc.fine_serial(p)
        M, V = ser["gmean"], ser["gvar"]
        hist = orc.parareal(p.scaled(max_iter=2))["hist"]
        sm, sv = math.sqrt(V.max() / p.P), V.max() * math.sqrt(2.0 / p.P)
        err = [max(np.max(np.abs(h[:, 0] - M)) / sm, np.max(np.abs(h[:, 1] - V)) / sv) for h in hist]
        assert err[0] > 1.0 and err[2] < 1.0, (model, err)
        assert V[-1] < 0.5  # unimodal: the ensemble gathers around the stable point
