"""Full MC-moments Parareal on the GPU against the oracle, and the
exactness invariant (Property 3.3) of the GPU path against its own serial
reference run."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _gpu_run(p, max_iter=None):
    from paper_2310_11365_gb300.mmp import Solver

    q = p if max_iter is None else p.scaled(max_iter=max_iter, tol=0.0)
    s = Solver(q)
    k = s.run()
    mom = s.moments()
    st = s.status()
    return s, k, mom, st


def _assert_moments_close(mom, orc_res, rtol=1e-10):
    """rho^K_n per region and globally, tolerance relative to the natural
    scale: sqrt(v) for means, v for variances.  Fractions counted from
    particles match exactly; fractions extrapolated by the learned model
    (Def. 3.4, an iterative LM fit) match to rtol."""
    N1 = mom.shape[0]
    I = 2 if np.any(orc_res["frac"][:, 1] != 0) else 1
    for n in range(N1):
        for i in range(I):
            fo, mo, vo = orc_res["frac"][n][i], orc_res["mean"][n][i], orc_res["var"][n][i]
            f, m, v = mom[n, 3 * i], mom[n, 3 * i + 1], mom[n, 3 * i + 2]
            assert abs(f - fo) <= rtol, (n, i, f, fo)
            if fo == 0 and I > 1:
                continue
            assert abs(m - mo) <= rtol * max(abs(mo), np.sqrt(abs(vo))), (n, i, m, mo)
            assert abs(v - vo) <= rtol * max(abs(vo), 1e-300), (n, i, v, vo)
        M, V = orc_res["hist"][-1][n]
        assert abs(mom[n, 6] - M) <= rtol * max(abs(M), np.sqrt(abs(V))), n
        assert abs(mom[n, 7] - V) <= rtol * abs(V), n


def test_config1_full_matches_oracle(mmplib, orc):
    """Config 1 (linear, P = 2000, N = 16, FP64) to tolerance: same sweep
    count and moments within 1e-10 relative."""
    p = W.config1()
    s, k, mom, st = _gpu_run(p)
    ref = orc.parareal(p)
    assert k == ref["sweeps"]
    assert st["converged"] == ref["converged"]
    _assert_moments_close(mom, ref)
    s.close()


@pytest.mark.parametrize("kmax", [1, 2, 5])
def test_intermediate_iterates_match_oracle(mmplib, orc, kmax):
    p = W.config2(P=3001, N=8, T=2.0, dt=4e-3, precision="fp64")
    s, k, mom, st = _gpu_run(p, kmax)
    ref = orc.parareal(p.scaled(max_iter=kmax, tol=0.0))
    assert k == kmax == ref["sweeps"]
    _assert_moments_close(mom, ref)
    s.close()


@pytest.mark.parametrize("variant", [W.MULTIMODAL, W.LEARNING])
def test_multimodal_matches_oracle(mmplib, orc, variant):
    p = W.config3(N=8, P=6001, T=6.0, dt=5e-3, variant=variant, s0=0.3, m0=1.0, B0=1.0, precision="fp64",
                  max_iter=5, tol=0.0)
    s, k, mom, st = _gpu_run(p)
    ref = orc.parareal(p)
    assert k == ref["sweeps"]
    _assert_moments_close(mom, ref)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("make", [
    lambda prec: W.config1(N=8, P=1001, T=2.0, precision=prec),
    lambda prec: W.config3(N=8, P=6001, T=4.0, dt=5e-3, s0=0.6, m0=0.2, precision=prec),
])
def test_property_3_3_gpu_bitwise(mmplib, make, prec):
    """After k sweeps slices 0..k of the GPU iterate equal the GPU serial
    run bit for bit, moments and particles."""
    import torch

    p = make(prec)
    from paper_2310_11365_gb300.mmp import Solver

    ref = Solver(p)
    ser = ref.serial()
    for kmax in (1, 3):
        s, k, mom, st = _gpu_run(p, kmax)
        for n in range(kmax + 1):
            if p.n_regions == 1:
                assert mom[n, 1] == ser[n, 1] and mom[n, 2] == ser[n, 2], (kmax, n)
            else:
                for i in range(2):
                    assert mom[n, 3 * i] == ser[n, 5 * i] / p.P
                    if ser[n, 5 * i] > 0:
                        assert mom[n, 3 * i + 1] == ser[n, 5 * i + 1]
                        assert mom[n, 3 * i + 2] == ser[n, 5 * i + 2]
        # the particles of the last exact slice end
        _, last = ref.serial(n_end=kmax, want_last=True)
        got = s.particles(kmax)
        assert torch.equal(got, last)
        s.close()
    ref.close()


def test_mixed_config2_small_against_oracle(mmplib, orc):
    """Mixed precision on the config-2 model vs the FP64 oracle on the same
    draws after a fixed number of sweeps: moments within the stated bounds
    (means 1.2e-6 of max(|m|, sd), variances 3e-6 relative; about twice the
    errors measured on a GB300, 5.3e-7 and 1.15e-6)."""
    p = W.config2(P=20_000, N=8, T=1.0, precision="mixed", max_iter=3, tol=0.0)
    s, k, mom, st = _gpu_run(p)
    ref = orc.parareal(p.scaled(precision="fp64"))
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert abs(mom[n, 6] - M) < 1.2e-6 * max(abs(M), np.sqrt(V)), n
        assert abs(mom[n, 7] - V) < 3e-6 * V, n
    s.close()


def test_edge_cases(mmplib, orc):
    """P = 1 (zero variance: redraw branch), N = 1, s0 = 0."""
    for p in (W.config1(P=1, N=4, T=1.0), W.config1(N=1, T=0.25, P=37),
              W.config1(P=64, N=4, T=1.0, s0=0.0)):
        s, k, mom, st = _gpu_run(p)
        ref = orc.parareal(p)
        assert k == ref["sweeps"]
        _assert_moments_close(mom, ref)  # 1e-10, as every other FP64 parity test
        assert st["dev_err"] == 0
        s.close()


def test_full_size_config2_invariant(mmplib):
    """Config 2 at full size (P = 1e6, N = 64, mixed), in the launch shape
    the benchmark uses: two sweeps reproduce the serial run exactly on the
    first two slice ends."""
    p = W.config2()
    s, k, mom, st = _gpu_run(p, 2)
    ser = s.serial(n_end=2)
    for n in range(3):
        assert mom[n, 1] == ser[n, 1] and mom[n, 2] == ser[n, 2]
    assert st["dev_err"] == 0
    s.close()
