"""Pins of the oracle's Parareal drivers: classical Parareal (Sec. 3.1,
Sec. 4.4 Dahlquist), the noisy-fine bounds of Lemma 4.2, and Property 3.3
(exactness of MC-moments Parareal) against the serial fine run."""
import math

import numpy as np
import pytest
from scipy.special import comb

from paper_2310_11365_gb300 import workloads as W


def test_classical_parareal_dahlquist_error_recursion(orc):
    """Dahlquist lambda = -4, coarse model error eps = 0.1 (Sec. 4.4): the
    iterates obey e^{k+1}_{n+1} = (F - G) e^k_n + G e^{k+1}_n (Lemma 4.1 with
    no noise), and u^k_n = u_n for k >= n (exactness)."""
    lam, eps, T, N = -4.0, 0.1, 2.0, 10
    dT = T / N
    F, G = math.exp(dT * lam), math.exp(dT * lam * (1 + eps))
    K = N
    it = orc.parareal_scalar(N, K, 1.0, F, 0.0, G, 0.0)
    exact = np.array([F**n for n in range(N + 1)])
    e = it - exact
    for k in range(K):
        for n in range(N):
            assert abs(e[k + 1, n + 1] - ((F - G) * e[k, n] + G * e[k + 1, n])) < 1e-15
    for k in range(K + 1):
        assert np.allclose(it[k, : k + 1], exact[: k + 1], rtol=0, atol=1e-15)
    # affine propagators (Lemma 4.1 allows f_n, g_n): exactness still holds
    it2 = orc.parareal_scalar(N, K, 0.3, F, 0.2, G, 0.1)
    ex2 = [0.3]
    for _ in range(N):
        ex2.append(F * ex2[-1] + 0.2)
    for k in range(K + 1):
        assert np.allclose(it2[k, : k + 1], ex2[: k + 1], rtol=0, atol=1e-15)


def test_lemma_4_2_bounds_with_noise(orc):
    """Lemma 4.2: with a noisy fine propagator (E|eps| <= varepsilon), the
    mean error max_n E|u^k_n - u_n| stays under the linear and superlinear
    bounds (Sec. 4.2 example)."""
    rng = np.random.default_rng(11)
    N, K, beta = 10, 6, 1e-2
    F, G = 0.5, 0.45
    ref = orc.parareal_scalar(N, N, 1.0, F, 0.0, G, 0.0)[N]  # noise-free fine = serial
    R = 400
    err = np.zeros((K + 1, N + 1))
    for _ in range(R):
        noise = rng.uniform(-2 * beta, 2 * beta, size=(K + 1, N + 1))  # E|eps| = beta
        it = orc.parareal_scalar(N, K, 1.0, F, 0.0, G, 0.0, noise)
        err += np.abs(it - ref)
    err /= R
    xi0 = err[0].max()
    q = abs(F - G) / (1 - abs(G))
    for k in range(1, K + 1):
        lin = q**k * xi0 + beta / (1 - abs(G)) * sum(q**j for j in range(k))
        sup = (abs(F - G) ** k / math.factorial(k) * np.prod([N - j for j in range(1, k + 1)]) * xi0
               + beta * (1 - abs(G) ** N) / (1 - abs(G))
               * sum(abs(F - G) ** j * comb(N - 1, j) for j in range(k)))
        assert err[k].max() <= min(lin, sup) * 1.05


def _small_unimodal():
    return W.config1(N=6, P=301, T=1.5)


def _small_multimodal(variant):
    # all mass starts in one well and relaxes into the other, so the region
    # fractions follow the two-state model of App. H and the fit is accepted
    return W.config3(N=8, P=6001, T=6.0, dt=5e-3, variant=variant, s0=0.3, m0=1.0, B0=1.0)


@pytest.mark.parametrize("make", [
    _small_unimodal,
    lambda: W.config2(N=6, P=250, T=1.5, dt=5e-3, precision="fp64"),
    lambda: _small_multimodal(W.MULTIMODAL),
    lambda: _small_multimodal(W.LEARNING),
])
def test_property_3_3_exactness_bitwise(orc, make):
    """Property 3.3: with the same draws in every iteration, after k sweeps
    the iterate equals the serial fine run on slices 0..k, particles and
    moments, bit for bit (with alpha = R(b) + (a - c) and the matching
    written as x + (mu - m) + (s - 1)(x - m))."""
    p = make()
    ser = orc.fine_serial(p, want_parts=True)
    for k in (1, 2, 3, p.N):
        q = p.scaled(max_iter=k, tol=0.0)
        r = orc.parareal(q, want_parts=True)
        assert r["sweeps"] == k
        for n in range(k + 1):
            assert np.array_equal(r["parts"][n], ser["parts"][n]), (k, n)
            M, V = r["hist"][k, n]
            assert M == ser["gmean"][n] or abs(M - ser["gmean"][n]) < 1e-14
            assert abs(V - ser["gvar"][n]) < 1e-13


def test_consistency_rho_equals_restriction(orc):
    """Micro-macro consistency (Property 3.3): rho^k_n = R(u^k_n) up to the
    rounding of S(T(alpha, b)) = alpha (Lemma 3.1 ii)."""
    p = _small_unimodal().scaled(max_iter=2, tol=0.0)
    r = orc.parareal(p, want_parts=True)
    for n in range(p.N + 1):
        st = orc.restrict(p, r["parts"][n])
        assert abs(r["mean"][n][0] - st["mean"][0]) < 1e-12
        assert abs(r["var"][n][0] - st["var"][0]) < 1e-12


def test_unimodal_linear_error_reaches_statistical_level(orc):
    """Config-1 form (Sec. 4.2-4.3): one sweep brings the error on (M, V)
    below the Monte-Carlo level sqrt(V/P); the iteration then contracts to
    the serial run and is exact at k = N (Property 3.3)."""
    p = W.config1(P=400, tol=0.0)
    r = orc.parareal(p)
    assert r["sweeps"] == p.N and r["converged"]
    ser = orc.fine_serial(p)
    h = r["hist"]
    err = [max(np.max(np.abs(h[k, :, 0] - ser["gmean"])), np.max(np.abs(h[k, :, 1] - ser["gvar"])))
           for k in range(p.N + 1)]
    mc_level = math.sqrt(ser["gvar"].max() / p.P)
    assert err[1] < mc_level < err[0]
    assert err[p.N] == 0.0
    assert err[p.N // 2] < err[1]


def test_multimodal_fractions_follow_fine(orc):
    """Def. 3.2: fractions of rho^{k}_{n+1} are those of F_n(u^{k-1}_n); the
    matching never changes them (Remark on particle fractions)."""
    p = _small_multimodal(W.MULTIMODAL).scaled(max_iter=3, tol=0.0)
    r = orc.parareal(p, want_parts=True)
    for n in range(p.N + 1):
        st = orc.restrict(p, r["parts"][n])
        assert r["frac"][n][0] == st["count"][0] / p.P
        assert r["frac"][n][0] + r["frac"][n][1] == 1.0


def test_learning_changes_only_extrapolated_fractions(orc):
    """Def. 3.4: learning replaces fractions beyond the exact slices only, so
    slices 0..k are identical with and without learning."""
    pm = _small_multimodal(W.MULTIMODAL).scaled(max_iter=3, tol=0.0)
    pl = _small_multimodal(W.LEARNING).scaled(max_iter=3, tol=0.0)
    rm = orc.parareal(pm)
    rl = orc.parareal(pl)
    assert np.array_equal(rm["hist"][3, :4], rl["hist"][3, :4])
    assert not np.array_equal(rm["frac"][5:], rl["frac"][5:])
    # the extrapolated fractions follow the fitted relaxation towards beta
    ser = orc.fine_serial(pl)
    fr = [st["count"][0] / pl.P for st in ser["stats"]]
    dT = pl.T / pl.N
    rc, alpha, beta = orc.lsq_fit(dT * np.arange(1, 4), np.array(fr[1:4]), fr[0], dT)
    assert rc == 0 and alpha < 0 and 0 <= beta <= 1
    for n in range(4, pl.N + 1):
        assert abs(rl["frac"][n][0] - orc.extrapolate(fr[3], alpha, beta, (n - 3) * dT)) < 1e-15
