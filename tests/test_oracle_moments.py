"""Pins of restriction, matching, mixture and the coarse moment ODEs."""
import math

import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W


def test_restriction_and_mixture_identity(orc):
    """Eq. (mixture_of_distributions_mean_variance) with population variances
    reproduces the direct whole-ensemble moments; fractions sum to one."""
    p = W.config3(P=5001)
    u = orc.initial(p) * 3.0 + 0.4
    st = orc.restrict(p, u)
    assert st["count"][0] + st["count"][1] == p.P
    assert st["count"][0] == int(np.sum(u < 0.0))
    frac = [c / p.P for c in st["count"]]
    M, V = orc.mixture(p, frac, st["mean"], st["var"])
    assert abs(M - u.mean()) < 1e-13
    assert abs(V - u.var()) < 1e-12
    assert abs(st["gmean"] - u.mean()) < 1e-14 and abs(st["gvar"] - u.var()) < 1e-13
    assert st["min"][1] >= 0.0 > st["max"][0]
    assert st["min"][0] == u.min() and st["max"][1] == u.max()


def test_lemma_3_1_T_of_S_is_identity_bitwise(orc):
    """Lemma 3.1 (i): T(S u, u) = u, bit for bit, per region."""
    for p in (W.config1(P=333), W.config3(P=777)):
        u = orc.initial(p)
        st = orc.restrict(p, u)
        out = orc.match(p, 1, st["mean"], st["var"], [1, 1], u)
        assert np.array_equal(out, u)


def test_lemma_3_1_S_of_T(orc):
    """Lemma 3.1 (ii): S(T(rho, u)) = rho for positive target variance."""
    p = W.config1(P=1001)
    u = orc.initial(p)
    out = orc.match(p, 2, [0.3, 0.0], [0.07, 0.0], [1, 0], u)
    st = orc.restrict(p, out)
    assert abs(st["mean"][0] - 0.3) < 1e-14
    assert abs(st["var"][0] - 0.07) < 1e-14


def test_matching_zero_variance_branch(orc):
    """T([mu, sigma], u) with V[u] = 0 draws sqrt(sigma) xi + mu (tag 2);
    T(S u, u) = u still holds (sigma = 0)."""
    p = W.config1(P=20_000, s0=0.0)
    u = np.full(p.P, 0.75)
    st = orc.restrict(p, u)
    assert st["var"][0] == 0.0
    assert np.array_equal(orc.match(p, 3, st["mean"], st["var"], [1, 0], u), u)
    out = orc.match(p, 3, [1.5, 0.0], [0.04, 0.0], [1, 0], u)
    assert out[11] == 1.5 + 0.2 * orc.normal(p, 2, 0, 3, 11)
    assert abs(out.mean() - 1.5) < 5 * 0.2 / math.sqrt(p.P)
    assert abs(out.var() - 0.04) < 5 * 0.04 * math.sqrt(2 / p.P)


def test_matching_only_selected_region(orc):
    p = W.config3(P=3000)
    u = orc.initial(p) * 2
    st = orc.restrict(p, u)
    out = orc.match(p, 1, [st["mean"][0] - 0.1, 0.0], [st["var"][0] * 0.5, 0.0], [1, 0], u)
    assert np.array_equal(out[u >= 0], u[u >= 0])
    assert not np.array_equal(out[u < 0], u[u < 0])


def _gh_expect(f, m, v, n=80):
    x, w = np.polynomial.hermite_e.hermegauss(n)
    return float(np.sum(w * f(m + math.sqrt(v) * x)) / math.sqrt(2 * math.pi))


def test_gaussian_closure_against_quadrature(orc):
    """Gaussian-assumed-density moment model, Eq. (Gaussian_model_McK_V_SDE)
    read with the Ito variance equation dV = 2E[(X-M)a] + E[b^2]: the
    closed forms must equal Gauss-Hermite quadrature of N(m, v)."""
    p = W.Problem(c3=1.3, c1=0.4, kappa=0.7, c0=-0.2, B=0.3, BE=0.5, B0=0.6)
    for (m, v) in [(0.5, 0.04), (-1.2, 0.3), (0.0, 1.1)]:
        a = lambda x: -p.c3 * x**3 + p.c1 * x + p.kappa * m + p.c0
        b = lambda x: p.B * x + p.BE * m + p.B0
        dm_q = _gh_expect(a, m, v)
        dv_q = 2 * _gh_expect(lambda x: (x - m) * a(x), m, v) + _gh_expect(lambda x: b(x) ** 2, m, v)
        dm, dv = orc.coarse_rhs(p, [1.0], [m], [v])
        assert abs(dm[0] - dm_q) < 1e-12 * (1 + abs(dm_q))
        assert abs(dv[0] - dv_q) < 1e-12 * (1 + abs(dv_q))


@pytest.mark.parametrize("regions", [2, 3, 4])
def test_multimodal_region_rhs_uses_global_mean(orc, regions):
    """Per-region model, Eq. (moment_model_Taylor_multimodal): each region's
    drift feels the mixture mean M = sum P_i m_i through kappa (two to four
    regions; Gauss-Hermite quadrature of each region's N(m_i, v_i))."""
    p = W.double_well(0.25, 0.5, 0.3, 0.7, n_regions=regions, threshold=-0.5, threshold2=0.0, threshold3=0.5)
    frac = {2: [0.3, 0.7], 3: [0.3, 0.3, 0.4], 4: [0.1, 0.2, 0.3, 0.4]}[regions]
    mean, var = [-0.9, 1.1, 0.2, -0.4][:regions], [0.05, 0.08, 0.12, 0.03][:regions]
    M = sum(f * m for f, m in zip(frac, mean))
    dm, dv = orc.coarse_rhs(p, frac, mean, var)
    for i in range(regions):
        a = lambda x: -p.c3 * x**3 + p.c1 * x + p.kappa * M
        assert abs(dm[i] - _gh_expect(a, mean[i], var[i])) < 1e-12
        dvq = 2 * _gh_expect(lambda x: (x - mean[i]) * a(x), mean[i], var[i]) + p.B0**2
        assert abs(dv[i] - dvq) < 1e-12


def test_property_2_2_linear_multimodal_equals_unimodal(orc):
    """Property 2.2: for a linear SDE, the per-region moment ODEs combined by
    the mixture identity (constant fractions) give the unimodal ODE's vector
    field at the mixture state."""
    theta, kappa, sigma = 0.8, 0.4, 0.6
    p1 = W.linear(theta, kappa, sigma)
    p2 = W.linear(theta, kappa, sigma, n_regions=2)
    frac, mean, var = [0.35, 0.65], [-0.7, 1.3], [0.2, 0.05]
    M, V = orc.mixture(p2, frac, mean, var)
    dm2, dv2 = orc.coarse_rhs(p2, frac, mean, var)
    dM = sum(f * d for f, d in zip(frac, dm2))
    dV = sum(f * (2 * m * d + e) for f, m, d, e in zip(frac, mean, dm2, dv2)) - 2 * M * dM
    dm1, dv1 = orc.coarse_rhs(p1, [1.0], [M], [V])
    assert abs(dM - dm1[0]) < 1e-13
    assert abs(dV - dv1[0]) < 1e-13


def test_coarse_forward_euler_closed_form(orc):
    """Linear model, forward Euler with step h_c: m_j = m0 (1 - theta h_c)^j,
    v_j = v_inf + (v0 - v_inf)(1 - 2 (theta + kappa) h_c)^j (exact algebra)."""
    theta, kappa, sigma = 1.0, 0.5, 0.5
    p = W.linear(theta, kappa, sigma, T=4.0, N=4, coarse_h=0.25)
    hc = 1.0 / orc.coarse_steps(p)
    assert orc.coarse_steps(p) == 4
    m, v = 1.0, 0.01
    _, mm, vv = orc.coarse(p, [1.0], [m], [v])
    vinf = sigma**2 / (2 * (theta + kappa))
    assert abs(mm[0] - (1 - theta * hc) ** 4) < 1e-15
    assert abs(vv[0] - (vinf + (v - vinf) * (1 - 2 * (theta + kappa) * hc) ** 4)) < 1e-15


def test_coarse_converges_to_lemma_2_1_solution(orc):
    """Lemma 2.1: for the linear SDE the moment model is exact; with a small
    coarse step it reproduces m(t) = m0 e^{-theta t} and
    v(t) = v_inf + (v0 - v_inf) e^{-2 (theta+kappa) t}."""
    theta, kappa, sigma = 1.0, 0.5, 0.5
    p = W.linear(theta, kappa, sigma, T=1.0, N=1, coarse_h=1e-5)
    _, mm, vv = orc.coarse(p, [1.0], [1.0], [0.01])
    vinf = sigma**2 / (2 * (theta + kappa))
    assert abs(mm[0] - math.exp(-theta)) < 1e-5
    assert abs(vv[0] - (vinf + (0.01 - vinf) * math.exp(-2 * (theta + kappa)))) < 1e-5


def test_coarse_keeps_fractions(orc):
    """Def. 3.2: the coarse propagator does not update the fractions."""
    p = W.config3()
    fr, _, _ = orc.coarse(p, [0.4, 0.6], [-1.0, 1.0], [0.1, 0.1])
    assert fr[:2] == [0.4, 0.6]
