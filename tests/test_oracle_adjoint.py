"""Pins of the oracle's adjoint of the serial fine propagator: central
differences with common random numbers (additive, state-proportional and
mean-field diffusion), the Taylor remainder, and closed forms of the linear
model's mean."""
import math

import numpy as np

from paper_2310_11365_gb300 import workloads as W

PARAMS = ("c3", "c1", "kappa", "c0", "B0", "B", "BE")


def _loss(orc, p, m_tgt, v_tgt):
    ser = orc.fine_serial(p)
    return float(np.sum((ser["gmean"][1:] - m_tgt) ** 2 + (ser["gvar"][1:] - v_tgt) ** 2))


def _check_central_differences(orc, p, ref):
    st = orc.fine_serial(ref)
    m_tgt, v_tgt = st["gmean"][1:], st["gvar"][1:]
    L, g = orc.adjoint_loss(p, m_tgt, v_tgt)
    assert abs(L - _loss(orc, p, m_tgt, v_tgt)) < 1e-14
    for k, name in enumerate(PARAMS):
        h = 1e-5
        plus = p.scaled(**{name: getattr(p, name) + h})
        minus = p.scaled(**{name: getattr(p, name) - h})
        fd = (_loss(orc, plus, m_tgt, v_tgt) - _loss(orc, minus, m_tgt, v_tgt)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1e-8), (name, g[k], fd)


def test_adjoint_matches_central_differences(orc):
    """Double-well model with additive noise, same draws in every
    evaluation: the adjoint gradient of L = sum (M-m*)^2 + (V-v*)^2 equals
    central differences (h = 1e-5) to 1e-6 relative in every coefficient,
    the diffusion's B and BE (zero here) included."""
    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.2, s0=0.5, T=1.0, N=4, dt=0.01, P=301, seed=17)
    ref = W.double_well(0.25, 0.5, 0.15, 0.65, m0=0.2, s0=0.5, T=1.0, N=4, dt=0.01, P=301, seed=18)
    _check_central_differences(orc, p, ref)


def test_adjoint_general_diffusion_central_differences(orc):
    """Cubic drift with b = B x + BE E[X] + B0 (state-proportional and
    mean-field noise, Sec. 2's general diffusion): the reverse recursion's
    noise terms (sqrt(h) B xi on the diagonal, sqrt(h) BE xi / P in the
    mean-field column) agree with central differences in all seven
    coefficients."""
    p = W.Problem(c3=0.6, c1=-0.4, kappa=0.5, c0=0.1, B=0.3, BE=-0.25, B0=0.35, m0=0.4, s0=0.3,
                  T=1.0, N=4, dt=0.01, P=257, seed=29)
    ref = p.scaled(kappa=0.7, B=0.2, BE=0.1, seed=30)
    _check_central_differences(orc, p, ref)


def test_adjoint_taylor_remainder(orc):
    """L(theta + eps d) - L(theta) - eps grad.d shrinks like eps^2."""
    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=1.0, N=4, dt=0.01, P=257, seed=5).scaled(B=0.2, BE=0.1)
    m_tgt = np.full(p.N, 0.3)
    v_tgt = np.full(p.N, 0.05)
    L0, g = orc.adjoint_loss(p, m_tgt, v_tgt)
    d = np.array([0.3, -0.7, 0.5, 0.2, -0.4, 0.25, -0.35])
    rem = []
    for eps in (1e-2, 5e-3):
        q = p.scaled(**{name: getattr(p, name) + eps * d[k] for k, name in enumerate(PARAMS)})
        L1 = _loss(orc, q, m_tgt, v_tgt)
        rem.append(abs(L1 - L0 - eps * g @ d))
    assert 3.0 < rem[0] / rem[1] < 5.0


def test_adjoint_linear_mean_closed_form(orc):
    """Linear model, cotangent 1 on M_N only: the mean obeys
    M_{j+1} = r M_j + h c0 + B0 sqrt(h) xibar_j with r = 1 + h (c1 + kappa), so
    dM_N/dc0 = h sum_{i<J} r^i and dM_N/dB0 = sqrt(h) sum_j xibar_j r^{J-1-j}."""
    p = W.linear(1.0, 0.5, 0.5, m0=1.0, s0=0.1, T=0.5, N=2, dt=0.05, P=9, seed=3)
    gm = np.zeros(p.N)
    gm[-1] = 1.0
    g, mom = orc.adjoint(p, gm, np.zeros(p.N))
    nf, h = orc.fine_steps(p), orc.fine_h(p)
    J = p.N * nf
    r = 1 + h * (p.c1 + p.kappa)
    assert abs(g[3] - h * sum(r**i for i in range(J))) < 1e-14
    xibar = [np.mean([orc.normal(p, 0, j % nf, j // nf, q) for q in range(p.P)]) for j in range(J)]
    dB0 = math.sqrt(h) * sum(xibar[j] * r ** (J - 1 - j) for j in range(J))
    assert abs(g[4] - dB0) < 1e-14
    # dM_N/dc3 at c3 = 0 is the propagated sensitivity to a small cubic term:
    # -h sum_j r^{J-1-j} mean_p(x_j^3) along the same (linear) path, whose
    # states are rebuilt here step by step from the same draws
    states = []
    u = orc.initial(p)
    for n in range(p.N):
        for j in range(nf):
            states.append(u.copy())
            xi = np.array([orc.normal(p, 0, j, n, k) for k in range(p.P)])
            u = u + h * (p.c1 * u + p.kappa * u.mean() + p.c0) + p.B0 * math.sqrt(h) * xi
    dc3 = -h * sum(r ** (J - 1 - j) * np.mean(states[j] ** 3) for j in range(J))
    assert abs(g[0] - dc3) < 1e-12 * max(1.0, abs(dc3))


def test_adjoint_variance_cotangent_linear(orc):
    """Linear model, cotangent 1 on V_N: deviations obey
    d_{j+1} = c d_j + B0 sqrt(h)(xi - xibar), c = 1 + h c1, so
    V_N = c^{2J} V_0 + ... and dV_N/dc0 = 0, dV_N/dkappa = 0."""
    p = W.linear(1.0, 0.5, 0.5, m0=1.0, s0=0.1, T=0.5, N=2, dt=0.05, P=13, seed=4)
    gv = np.zeros(p.N)
    gv[-1] = 1.0
    g, _ = orc.adjoint(p, np.zeros(p.N), gv)
    assert abs(g[3]) < 1e-14 and abs(g[2]) < 1e-14
