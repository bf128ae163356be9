"""Brute force at tiny sizes: the MC-moments Parareal iteration written out
by hand in plain Python (lists and scalar arithmetic, nothing shared with
the oracle's C), for P in {2, 3}, N in {1, 2, 3} and at most three fine
steps per slice, against the oracle.  Only the random draws (tag-0 noise,
tag-1 initial ensemble) come from the oracle's generator, which has its
own pins; everything the method computes from them is re-derived here:

  fine      X_{j+1} = X_j + a(X_j, m_j) h + b(X_j, m_j) sqrt(h) xi_j,  m_j = mean of X_j
            a(x, m) = -c3 x^3 + c1 x + kappa m + c0,  b(x, m) = B x + BE m + B0   (Sec. 1.2)
  restrict  population mean and variance (Sec. 3.4)
  coarse    forward Euler on the Gaussian-closure moment ODE (Sec. 2.1-2.2)
  iterate   alpha = R(F(u^k_n)) + (C(rho^{k+1}_n) - C(rho^k_n)), accepted if its variance
            is >= 0; matching T(rho, u) = x + (mu - m) + (s - 1)(x - m), s = sqrt(sigma / v)
            (Defs. 3.1, Eq. mM_parareal_other_k_NEW)
"""
import math

import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W


def _stats(x):
    P = len(x)
    m = sum(x) / P
    return m, sum((xi - m) * (xi - m) for xi in x) / P


def _brute_parareal(p, orc):
    P, N = p.P, p.N
    dT = p.T / N
    nf = math.ceil(dT / p.dt - 1e-9)
    h = dT / nf
    nc = math.ceil(dT / p.coarse_h - 1e-9)
    hc = dT / nc

    def z(j, n, q):
        return orc.normal(p, 0, j, n, q)

    def fine(n, u):
        x = list(u)
        for j in range(nf):
            m = sum(x) / P
            x = [x[q] + (-p.c3 * x[q] ** 3 + p.c1 * x[q] + p.kappa * m + p.c0) * h
                 + (p.B * x[q] + p.BE * m + p.B0) * math.sqrt(h) * z(j, n, q) for q in range(P)]
        return x

    def coarse(mv):
        m, v = mv
        for _ in range(nc):
            eb = p.B * m + p.BE * m + p.B0
            dm = -p.c3 * (m ** 3 + 3 * m * v) + p.c1 * m + p.kappa * m + p.c0
            dv = 2 * (-p.c3 * 3 * v * (m * m + v) + p.c1 * v) + p.B * p.B * v + eb * eb
            m, v = m + hc * dm, v + hc * dv
        return m, v

    def match(x, mu, sigma, m, v):
        s = math.sqrt(sigma / v)
        return [xi + (mu - m) + (s - 1) * (xi - m) for xi in x]

    u0 = [p.m0 + p.s0 * orc.normal(p, 1, 0, 0, q) for q in range(P)]
    st0 = _stats(u0)
    rho = [st0]
    cache = []
    for n in range(N):
        rho.append(coarse(rho[n]))
        cache.append(rho[n + 1])
    U = [u0] + [match(u0, rho[n][0], rho[n][1], *st0) if rho[n][1] >= 0 else list(u0) for n in range(1, N + 1)]
    hist = [list(rho)]
    for k in range(1, N + 1):
        Bf = [fine(n, U[n]) for n in range(N)]
        new = [rho[0]]
        Unew = [u0]
        for n in range(N):
            a = coarse(new[n])
            bm, bv = _stats(Bf[n])
            am, av = bm + (a[0] - cache[n][0]), bv + (a[1] - cache[n][1])
            if av >= 0:
                new.append((am, av))
                Unew.append(match(Bf[n], am, av, bm, bv))
            else:
                new.append((bm, bv))
                Unew.append(Bf[n])
            cache[n] = a
        rho, U = new, Unew
        hist.append(list(rho))
    serial = [u0]
    for n in range(N):
        serial.append(fine(n, serial[-1]))
    return hist, [_stats(x) for x in serial]


CASES = []
for P in (2, 3):
    for N in (1, 2, 3):
        for form in ("linear", "cubic", "multiplicative"):
            CASES.append((P, N, form))


@pytest.mark.parametrize("P,N,form", CASES)
def test_tiny_parareal_by_hand(orc, P, N, form):
    nf = 1 + (P + N) % 3  # 1..3 fine steps per slice
    common = dict(T=0.6 * N, N=N, dt=0.6 / nf, P=P, coarse_h=0.25, seed=W.SEED_BASE + 41 + 7 * P + N,
                  tol=0.0, max_iter=N, precision="fp64", m0=0.3, s0=0.7)
    if form == "linear":
        p = W.Problem(c1=-1.2, kappa=0.4, c0=0.1, B0=0.6, **common)
    elif form == "cubic":
        p = W.Problem(c3=1.0, c1=0.5, kappa=0.3, c0=-0.05, B0=0.5, **common)
    else:
        p = W.Problem(c3=0.5, c1=-0.4, kappa=0.2, c0=0.02, B=0.3, BE=-0.1, B0=0.4, **common)
    hist, serial = _brute_parareal(p, orc)
    ref = orc.parareal(p)
    assert ref["sweeps"] == N
    for k in range(N + 1):
        for n in range(N + 1):
            M, V = ref["hist"][k][n]
            m, v = hist[k][n]
            assert abs(M - m) <= 1e-13 * max(1.0, abs(m)), (k, n)
            assert abs(V - v) <= 1e-13 * max(1.0, abs(v)), (k, n)
    # and the serial fine run the iteration ends on (Property 3.3 at k = N)
    st = orc.fine_serial(p)
    for n in range(N + 1):
        assert abs(st["gmean"][n] - serial[n][0]) <= 1e-13 * max(1.0, abs(serial[n][0]))
        assert abs(st["gvar"][n] - serial[n][1]) <= 1e-13 * max(1.0, serial[n][1])
        assert abs(hist[N][n][0] - serial[n][0]) <= 1e-12 * max(1.0, abs(serial[n][0]))
