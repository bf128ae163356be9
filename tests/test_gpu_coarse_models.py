"""GPU Parareal with each coarse moment model (closure, Taylor, 2- and
3-point sigma-point rules) against the FP64 oracle to 1e-10 relative, on a
unimodal cubic problem, (all but Taylor) a two-region double well and the
paper's modified geometric Brownian motion; an unknown model is refused
before any launch.  The Taylor model has no
Sigma^2 term, so its variance grows exponentially in a region whose mean
sits near the barrier top (a_X > 0): its lifting prediction for the
two-region well overflows in the oracle as on the GPU."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MODELS = (W.CLOSURE, W.TAYLOR, W.SIGMA2, W.SIGMA3)


def _problems(model):
    out = [W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=2.0, N=8, dt=0.01, P=4001, seed=5, precision="fp64",
                   tol=1e-9, coarse_model=model)]
    if model != W.TAYLOR:
        out.append(W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.0, s0=0.4, T=4.0, N=8, dt=0.01, P=6001, seed=6,
                                 n_regions=2, threshold=0.0, variant=W.MULTIMODAL, precision="fp64",
                                 tol=1e-9, coarse_model=model))
    return out


@pytest.mark.parametrize("model", MODELS)
def test_coarse_model_matches_oracle(mmplib, orc, model):
    from paper_2310_11365_gb300.mmp import Solver

    for p in _problems(model):
        s = Solver(p)
        k = s.run()
        mom = s.moments(0)
        ref = orc.parareal(p)
        assert k == ref["sweeps"], (model, k, ref["sweeps"])
        for n in range(p.N + 1):
            M, V = ref["hist"][-1][n]
            assert abs(mom[n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V)), (model, n)
            assert abs(mom[n, 7] - V) <= 1e-10 * V, (model, n)
        s.close()


@pytest.mark.parametrize("model", MODELS)
def test_gbm_matches_oracle(mmplib, orc, model):
    """The paper's modified geometric Brownian motion (linear drift,
    state-proportional and mean-field noise), solved through mmp.run with
    each coarse model: the slice-end moments equal the oracle's to 1e-10.
    For linear coefficients the four models are the same moment ODE
    (Lemma 2.1), so they also agree with each other to rounding."""
    from paper_2310_11365_gb300 import mmp

    p = W.gbm(P=4001, dt=0.01, coarse_model=model)
    res = mmp.run(p)[0]
    ref = orc.parareal(p)
    assert res["sweeps"] == ref["sweeps"] and res["dev_err"] == 0
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert abs(res["moments"][n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V)), (model, n)
        assert abs(res["moments"][n, 7] - V) <= 1e-10 * V, (model, n)
    base = orc.parareal(p.scaled(coarse_model=W.CLOSURE))
    assert np.allclose(ref["hist"][1], base["hist"][1], rtol=1e-12, atol=1e-14)


def test_unknown_coarse_model_is_refused(mmplib):
    from paper_2310_11365_gb300.mmp import MMPError, Solver

    with pytest.raises(MMPError) as e:
        Solver(W.config1(N=4, T=1.0, coarse_model=7))
    assert "INVALID_ARG" in str(e.value)
