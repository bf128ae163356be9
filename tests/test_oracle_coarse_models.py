"""The coarse moment models besides the Gaussian closure (Sec. 2): the
Taylor model (Eq. moment_model_class_1) and the Gaussian-assumed density
(Eq. Gaussian_model_McK_V_SDE) with 2- and 3-point sigma-point rules.  For
the drift a = -c3 x^3 + c1 x + kappa M + c0 and diffusion b = B x + BE M + B0
their right-hand sides differ from the closure in closed form:

  linear drift (c3 = 0): all four equal (the moment ODE is exact, Lemma 2.1);
  3-point rule: exact for polynomials of degree <= 5, so equal to the closure;
  2-point rule: exact to degree 3; dV differs by +4 c3 V^2;
  Taylor: a(M) + a_XX V / 2 and (2 a_X + b_X^2) V + b(M)^2; dV differs by +6 c3 V^2.

The MC-moments Parareal iteration ends on the serial fine run whatever the
coarse model (Property 3.3), and the models do change the iterates before."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

MODELS = (W.CLOSURE, W.TAYLOR, W.SIGMA2, W.SIGMA3)


def _rhs(orc, p, model, frac, mean, var):
    return orc.coarse_rhs(p.scaled(coarse_model=model), frac, mean, var)


BOUNDS = dict(threshold=-0.5, threshold2=0.0, threshold3=0.5)
FRAC = {1: [1.0], 2: [0.4, 0.6], 3: [0.3, 0.3, 0.4], 4: [0.2, 0.3, 0.1, 0.4]}
MEAN = [-0.7, 0.9, 1.3, -1.1]
VAR = [0.3, 0.5, 0.2, 0.45]


@pytest.mark.parametrize("regions", [1, 2, 3, 4])
def test_linear_drift_all_models_agree(orc, regions):
    p = W.Problem(c1=-1.3, kappa=0.4, c0=0.2, B=0.3, BE=0.1, B0=0.5, n_regions=regions,
                  variant=W.MULTIMODAL if regions > 1 else W.UNIMODAL, **BOUNDS)
    frac, mean, var = FRAC[regions], MEAN[:regions], VAR[:regions]
    ref = _rhs(orc, p, W.CLOSURE, frac, mean, var)
    for model in MODELS[1:]:
        got = _rhs(orc, p, model, frac, mean, var)
        for i in range(regions):
            assert got[0][i] == pytest.approx(ref[0][i], rel=1e-14, abs=1e-15)
            assert got[1][i] == pytest.approx(ref[1][i], rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("regions", [1, 2, 3, 4])
def test_cubic_drift_closed_form_differences(orc, regions):
    c3 = 0.8
    p = W.Problem(c3=c3, c1=0.6, kappa=0.3, c0=-0.1, B=0.25, BE=-0.2, B0=0.4, n_regions=regions,
                  variant=W.MULTIMODAL if regions > 1 else W.UNIMODAL, **BOUNDS)
    frac, mean, var = FRAC[regions], MEAN[:regions], VAR[:regions]
    cl = _rhs(orc, p, W.CLOSURE, frac, mean, var)
    s3 = _rhs(orc, p, W.SIGMA3, frac, mean, var)
    s2 = _rhs(orc, p, W.SIGMA2, frac, mean, var)
    ta = _rhs(orc, p, W.TAYLOR, frac, mean, var)
    for i in range(regions):
        v = var[i]
        for got in (s3, s2, ta):
            assert got[0][i] == pytest.approx(cl[0][i], rel=1e-13)
        assert s3[1][i] == pytest.approx(cl[1][i], rel=1e-13)
        assert s2[1][i] == pytest.approx(cl[1][i] + 4 * c3 * v * v, rel=1e-13)
        assert ta[1][i] == pytest.approx(cl[1][i] + 6 * c3 * v * v, rel=1e-13)


@pytest.mark.parametrize("model", MODELS)
def test_parareal_ends_on_the_serial_run(orc, model):
    p = W.double_well(0.25, 0.5, 0.2, 0.6, m0=0.1, s0=0.5, T=2.0, N=5, dt=0.02, P=301, seed=19,
                      tol=0.0, max_iter=5, coarse_model=model)
    ref = orc.parareal(p)
    st = orc.fine_serial(p)
    assert ref["sweeps"] == p.N
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert M == st["gmean"][n] and V == st["gvar"][n], n


def test_models_change_the_iterates(orc):
    base = dict(T=2.0, N=5, dt=0.02, P=301, seed=19, tol=0.0, max_iter=2, m0=0.1, s0=0.5)
    first = {}
    for model in MODELS:
        p = W.double_well(0.25, 0.5, 0.2, 0.6, coarse_model=model, **base)
        first[model] = orc.parareal(p)["hist"][1]
    # sigma3 reproduces the closure; the others move the first iterate
    assert np.allclose(first[W.SIGMA3], first[W.CLOSURE], rtol=1e-12, atol=1e-14)
    assert not np.allclose(first[W.SIGMA2], first[W.CLOSURE], rtol=1e-9)
    assert not np.allclose(first[W.TAYLOR], first[W.CLOSURE], rtol=1e-9)


def test_gbm_every_model_the_same_and_one_sweep_reaches_the_mc_level(orc):
    """The modified geometric Brownian motion (Sec. 5.1) has drift and
    diffusion linear in X and E[X], state- and mean-dependent noise
    included, so every coarse model is the same moment ODE (Lemma 2.1) and
    gives the same iterates; with that model one sweep brings the iterate to
    the Monte Carlo level of the serial fine run (within two statistical
    units, sqrt(V/P) for the mean and V sqrt(2/P) for the variance)."""
    hists = {}
    for model in MODELS:
        p = W.gbm(P=2000, dt=1e-2, coarse_model=model, tol=0.0)
        hists[model] = orc.parareal(p.scaled(max_iter=2))["hist"]
    for model in MODELS[1:]:
        assert np.allclose(hists[model], hists[W.CLOSURE], rtol=1e-12, atol=1e-14), model
    p = W.gbm(P=2000, dt=1e-2, tol=0.0)
    ser = orc.fine_serial(p)
    M, V = ser["gmean"], ser["gvar"]
    sm, sv = np.sqrt(V.max() / p.P), V.max() * np.sqrt(2.0 / p.P)
    h = hists[W.CLOSURE][1]
    assert np.max(np.abs(h[:, 0] - M)) < 2 * sm
    assert np.max(np.abs(h[:, 1] - V)) < 2 * sv
