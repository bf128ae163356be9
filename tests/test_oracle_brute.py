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


# ---- several regions (Def. 3.2), written out the same way ------------------

def _regions_brute(p, orc):
    """The multimodal iteration by hand: per-region restriction with extremes,
    per-region closure with the mixture mean field and frozen fractions, the
    iterator per region (alpha_V >= 0, V(b) > 0, the transformed extremes
    inside [t_i, t_{i+1})), an empty region carrying the coarse prediction,
    fractions from the fine outputs; lifting redraws a region of variance 0
    from the tag-2 stream of that region."""
    P, N, I = p.P, p.N, p.n_regions
    bounds = [p.threshold, p.threshold2, p.threshold3][: I - 1]
    dT = p.T / N
    nf = math.ceil(dT / p.dt - 1e-9)
    h = dT / nf
    nc = math.ceil(dT / p.coarse_h - 1e-9)
    hc = dT / nc

    def region(x):
        for i, t in enumerate(bounds):
            if x < t:
                return i
        return I - 1

    def restrict(x):
        out = []
        for i in range(I):
            xs = [v for v in x if region(v) == i]
            if xs:
                m, v = _stats(xs)
                out.append((len(xs), m, v, min(xs), max(xs)))
            else:
                out.append((0, 0.0, 0.0, math.inf, -math.inf))
        return out

    def mixture(rho):
        fr, mean, var = rho
        M = sum(f * m for f, m in zip(fr, mean))
        return M, sum(f * (m * m + v) for f, m, v in zip(fr, mean, var)) - M * M

    def coarse(rho):
        fr, mean, var = list(rho[0]), list(rho[1]), list(rho[2])
        for _ in range(nc):
            M = sum(f * m for f, m in zip(fr, mean))
            new_m, new_v = [], []
            for m, v in zip(mean, var):
                eb = p.B * m + p.BE * M + p.B0
                dm = -p.c3 * (m ** 3 + 3 * m * v) + p.c1 * m + p.kappa * M + p.c0
                dv = 2 * (-p.c3 * 3 * v * (m * m + v) + p.c1 * v) + p.B * p.B * v + eb * eb
                new_m.append(m + hc * dm)
                new_v.append(v + hc * dv)
            mean, var = new_m, new_v
        return fr, mean, var

    def fine(n, u):
        x = list(u)
        for j in range(nf):
            m = sum(x) / P
            x = [x[q] + (-p.c3 * x[q] ** 3 + p.c1 * x[q] + p.kappa * m + p.c0) * h
                 + (p.B * x[q] + p.BE * m + p.B0) * math.sqrt(h) * orc.normal(p, 0, j, n, q) for q in range(P)]
        return x

    def transformed(x, mu, sigma, m, v):
        return x + (mu - m) + (math.sqrt(sigma / v) - 1) * (x - m)

    def match(x, n, mu, sigma, doit, st):
        out = []
        for q, xq in enumerate(x):
            i = region(xq)
            if doit[i]:
                m, v = st[i][1], st[i][2]
                if v == 0.0:
                    xq = mu[i] + math.sqrt(sigma[i]) * orc.normal(p, 2, i, n, q)
                else:
                    xq = transformed(xq, mu[i], sigma[i], m, v)
            out.append(xq)
        return out

    u0 = [p.m0 + p.s0 * orc.normal(p, 1, 0, 0, q) for q in range(P)]
    st0 = restrict(u0)
    rho = [([c / P for c, *_ in st0], [s[1] for s in st0], [s[2] for s in st0])]
    cache = []
    for n in range(N):
        rho.append(coarse(rho[n]))
        cache.append(rho[n + 1])
    U = [u0]
    for n in range(1, N + 1):
        doit = [st0[i][0] > 0 and rho[n][2][i] >= 0 for i in range(I)]
        U.append(match(u0, n, rho[n][1], rho[n][2], doit, st0))
    hist = [[mixture(r) for r in rho]]
    for k in range(1, N + 1):
        Bf = [fine(n, U[n]) for n in range(N)]
        rst = [restrict(b) for b in Bf]
        fr = [rho[0][0]] + [[s[0] / P for s in rst[n]] for n in range(N)]
        new = [rho[0]]
        Unew = [u0]
        for n in range(N):
            cur = (fr[n], new[n][1], new[n][2])
            new[n] = cur
            a = coarse(cur)
            b = rst[n]
            mean, var, doit = [], [], []
            for i in range(I):
                cnt, bm, bv, lo, hi = b[i]
                if cnt == 0:
                    mean.append(a[1][i])
                    var.append(a[2][i])
                    doit.append(False)
                    continue
                am = bm + (a[1][i] - cache[n][1][i])
                av = bv + (a[2][i] - cache[n][2][i])
                accept = av >= 0
                if accept:
                    if bv == 0.0:
                        accept = False
                    else:
                        if i > 0:
                            accept = transformed(lo, am, av, bm, bv) >= bounds[i - 1]
                        if accept and i < I - 1:
                            accept = transformed(hi, am, av, bm, bv) < bounds[i]
                mean.append(am if accept else bm)
                var.append(av if accept else bv)
                doit.append(accept)
            new.append((fr[n + 1], mean, var))
            Unew.append(match(Bf[n], n + 1, mean, var, doit, b))
            cache[n] = a
        rho, U = new, Unew
        hist.append([mixture(r) for r in rho])
    return hist, rho


# (regions, boundaries): two, three, three with a narrow middle region (often
# empty at these sizes) and four
BOUNDS = {
    2: dict(n_regions=2, threshold=0.0),
    3: dict(n_regions=3, threshold=-0.3, threshold2=0.3),
    "3n": dict(n_regions=3, threshold=-0.06, threshold2=0.06),
    4: dict(n_regions=4, threshold=-0.6, threshold2=0.0, threshold3=0.6),
}
REGION_CASES = [(I, P, N) for I in (2, 3, "3n", 4) for P in (5, 7) for N in (2, 3)] + [(4, 16, 3), (4, 23, 3)]


@pytest.mark.parametrize("I,P,N", REGION_CASES)
def test_tiny_multimodal_parareal_by_hand(orc, I, P, N):
    nf = 1 + (P + N) % 3
    bounds = BOUNDS[I]
    p = W.double_well(0.25, 0.5, 0.3, 0.6, T=0.6 * N, N=N, dt=0.6 / nf, P=P, coarse_h=0.25,
                      seed=W.SEED_BASE + 71 + 5 * P + N + 11 * bounds["n_regions"], tol=0.0, max_iter=N,
                      precision="fp64", m0=0.1, s0=0.8, variant=W.MULTIMODAL, **bounds)
    I = p.n_regions
    hist, rho = _regions_brute(p, orc)
    ref = orc.parareal(p)
    assert ref["sweeps"] == N
    for k in range(N + 1):
        for n in range(N + 1):
            M, V = ref["hist"][k][n]
            m, v = hist[k][n]
            assert abs(M - m) <= 1e-12 * max(1.0, abs(m)), (k, n, M, m)
            assert abs(V - v) <= 1e-12 * max(1.0, abs(v)), (k, n, V, v)
    for n in range(N + 1):
        for i in range(I):
            # empty regions too: they carry the coarse prediction (reading of Defs. 3.2/3.4)
            assert ref["frac"][n][i] == rho[n][0][i], (n, i)
            assert abs(ref["mean"][n][i] - rho[n][1][i]) <= 1e-12 * max(1.0, abs(rho[n][1][i])), (n, i)
            assert abs(ref["var"][n][i] - rho[n][2][i]) <= 1e-12 * max(1.0, abs(rho[n][2][i])), (n, i)
    assert ref["accepted"] > 0 or N == 1
