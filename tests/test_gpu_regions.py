"""Three and four regions on the GPU (Def. 3.2 on intervals split at
t_1 < t_2 < t_3; Def. 3.4 with the rate model of Sec. 3.6): the fused
restriction per region against the oracle, whole MC-moments Parareal runs
(multimodal and learning) against the oracle, Property 3.3 bit for bit
against the GPU's own serial run, mixed precision within its bounds, and a
batch of three- and four-region problems."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THR3 = dict(n_regions=3, threshold=-0.5, threshold2=0.5)
THR4 = dict(n_regions=4, threshold=-1.0, threshold2=0.0, threshold3=1.0)


def _well(variant, regions, precision="fp64", **kw):
    base = dict(m0=0.0, s0=0.6, T=2.0, N=6, dt=0.01, P=6001, seed=41, variant=variant, tol=0.0,
                precision=precision)
    base.update(kw)
    return W.double_well(0.25, 0.5, 0.1, 0.7, **base, **regions)


def _compare(p, mom, ref, rtol):
    """Per region (fraction, mean, variance) and the global (M, V) of the
    final iterate, each against its natural scale."""
    from paper_2310_11365_gb300.mmp import moment_region

    for n in range(p.N + 1):
        for i in range(p.n_regions):
            o = moment_region(i)
            fo, mo, vo = ref["frac"][n][i], ref["mean"][n][i], ref["var"][n][i]
            assert abs(mom[n, o] - fo) <= rtol, (n, i, mom[n, o], fo)
            if fo == 0:
                continue
            assert abs(mom[n, o + 1] - mo) <= rtol * max(abs(mo), np.sqrt(abs(vo))), (n, i)
            assert abs(mom[n, o + 2] - vo) <= rtol * max(abs(vo), 1e-300), (n, i)
        for i in range(p.n_regions, 4):
            o = moment_region(i)
            assert mom[n, o] == 0 and mom[n, o + 1] == 0 and mom[n, o + 2] == 0
        M, V = ref["hist"][-1][n]
        assert abs(mom[n, 6] - M) <= rtol * max(abs(M), np.sqrt(abs(V))), n
        assert abs(mom[n, 7] - V) <= rtol * abs(V), n


@pytest.mark.parametrize("regions", [THR3, THR4])
def test_serial_restriction_per_region(mmplib, orc, regions):
    """The fused restriction of the serial fine run, per region: counts
    exact, means and variances to 1e-10, extremes exact (FP64)."""
    from paper_2310_11365_gb300.mmp import Solver, stat_region

    p = _well(W.MULTIMODAL, regions)
    s = Solver(p)
    st = s.serial()
    ref = orc.fine_serial(p)
    for n in range(p.N + 1):
        r = ref["stats"][n]
        for i in range(p.n_regions):
            o = stat_region(i)
            assert st[n, o] == r["count"][i], (n, i)
            if r["count"][i] == 0:
                continue
            assert abs(st[n, o + 1] - r["mean"][i]) <= 1e-10 * max(abs(r["mean"][i]), np.sqrt(r["var"][i]))
            assert abs(st[n, o + 2] - r["var"][i]) <= 1e-10 * r["var"][i]
            assert abs(st[n, o + 3] - r["min"][i]) <= 1e-12 * max(1.0, abs(r["min"][i]))
            assert abs(st[n, o + 4] - r["max"][i]) <= 1e-12 * max(1.0, abs(r["max"][i]))
        assert abs(st[n, 10] - ref["gmean"][n]) <= 1e-12
    s.close()


@pytest.mark.parametrize("kmax", [2, 4, 6])
@pytest.mark.parametrize("variant", [W.MULTIMODAL, W.LEARNING])
@pytest.mark.parametrize("regions", [THR3, THR4])
def test_parareal_matches_oracle(mmplib, orc, regions, variant, kmax):
    """Intermediate and final iterates in FP64 to 1e-10, including sweeps
    whose fractions beyond t_k come from the fitted rate model (k >= I)."""
    from paper_2310_11365_gb300.mmp import Solver

    p = _well(variant, regions, max_iter=kmax)
    s = Solver(p)
    k = s.run()
    ref = orc.parareal(p)
    assert k == ref["sweeps"] == kmax
    assert s.status()["dev_err"] == 0
    _compare(p, s.moments(), ref, 1e-10)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("regions", [THR3, THR4])
def test_property_3_3_bitwise(mmplib, regions, prec):
    """After k sweeps slices 0..k equal the GPU serial run bit for bit, in
    every region."""
    import torch

    from paper_2310_11365_gb300.mmp import Solver, moment_region, stat_region

    p = _well(W.LEARNING, regions, precision=prec)
    ref = Solver(p)
    ser = ref.serial()
    for kmax in (1, 4):
        s = Solver(p.scaled(max_iter=kmax))
        s.run()
        mom = s.moments()
        for n in range(kmax + 1):
            for i in range(p.n_regions):
                o, so = moment_region(i), stat_region(i)
                assert mom[n, o] == ser[n, so] / p.P, (kmax, n, i)
                if ser[n, so] > 0:
                    assert mom[n, o + 1] == ser[n, so + 1] and mom[n, o + 2] == ser[n, so + 2], (kmax, n, i)
        _, last = ref.serial(n_end=kmax, want_last=True)
        assert torch.equal(s.particles(kmax), last)
        s.close()
    ref.close()


@pytest.mark.parametrize("regions", [THR3, THR4])
def test_mixed_within_bounds(mmplib, orc, regions):
    """FP32 particles with FP64 moments against the FP64 oracle after three
    sweeps: global mean to 2e-6 of its scale, variance to 1e-5 relative."""
    from paper_2310_11365_gb300.mmp import Solver

    p = _well(W.MULTIMODAL, regions, precision="mixed", max_iter=3, P=20_001)
    s = Solver(p)
    s.run()
    mom = s.moments()
    ref = orc.parareal(p.scaled(precision="fp64"))
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert abs(mom[n, 6] - M) <= 2e-6 * max(abs(M), np.sqrt(V)), n
        assert abs(mom[n, 7] - V) <= 1e-5 * V, n
    s.close()


def test_batch_of_three_and_four_regions(mmplib, orc):
    """Problems with 3 and 4 regions (and one with 2) solved as one batch:
    each matches the oracle to 1e-10."""
    from paper_2310_11365_gb300.mmp import Solver, mmp_batch_info

    batch = [_well(W.LEARNING, THR3, max_iter=5, problem_tag=1),
             _well(W.MULTIMODAL, THR4, max_iter=5, problem_tag=2, P=4001),
             _well(W.LEARNING, dict(n_regions=2, threshold=0.0), max_iter=5, problem_tag=3)]
    s = Solver(batch)
    s.run()
    assert mmp_batch_info(s.ctx)["batched"]
    for b, p in enumerate(batch):
        ref = orc.parareal(p)
        assert s.status(b)["sweeps"] == ref["sweeps"] and s.status(b)["dev_err"] == 0
        _compare(p, s.moments(b), ref, 1e-10)
    s.close()


def test_redraw_branch_with_three_regions(mmplib, orc):
    """Every initial particle at x = 0 (s0 = 0): the middle region has
    variance 0, so lifting redraws it from the tag-2 stream of region 1
    (Eq. multimodal_M's first branch); FP64 against the oracle to 1e-10."""
    from paper_2310_11365_gb300.mmp import Solver

    p = _well(W.MULTIMODAL, THR3, s0=0.0, max_iter=3)
    s = Solver(p)
    s.run()
    ref = orc.parareal(p)
    assert s.status()["sweeps"] == ref["sweeps"] and s.status()["dev_err"] == 0
    _compare(p, s.moments(), ref, 1e-10)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_regions_with_state_dependent_noise(mmplib, orc, prec):
    """Four regions with b = B x + BE E[X] + B0 (the general-form fine
    kernel): FP64 to 1e-10; mixed within its bounds on the slice ends that
    are exact after k sweeps (beyond t_k the fractions come from a fit to
    counts, and a particle near a boundary may fall on either side in FP32)."""
    from paper_2310_11365_gb300.mmp import Solver

    p = _well(W.LEARNING, THR4, precision=prec, max_iter=5, P=8001).scaled(B=0.15, BE=-0.1)
    s = Solver(p)
    s.run()
    mom = s.moments()
    ref = orc.parareal(p.scaled(precision="fp64"))
    assert s.status()["sweeps"] == ref["sweeps"] and s.status()["dev_err"] == 0
    if prec == "fp64":
        _compare(p, mom, ref, 1e-10)
    else:
        for n in range(p.max_iter + 1):
            M, V = ref["hist"][-1][n]
            assert abs(mom[n, 6] - M) <= 2e-6 * max(abs(M), np.sqrt(V)), n
            assert abs(mom[n, 7] - V) <= 1e-5 * V, n
    s.close()
