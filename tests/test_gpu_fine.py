"""GPU fine propagator (one slice, explicit ensemble) against the oracle:
particles and restriction records, FP64 to 1e-10 relative, FP32 within
stated bounds.  Sizes span one and many CTAs per slice and ragged tails."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _run_fine(mmplib, p, n, u0):
    import torch

    from paper_2310_11365_gb300.mmp import Solver

    s = Solver(p)
    dt = s.dtype()
    u_in = torch.zeros(p.P + 8, dtype=dt, device="cuda")
    u_in[: p.P] = torch.from_numpy(u0).to(dt)
    u_out = torch.zeros_like(u_in)
    st = mmplib.mmp_fine(s.ctx, 0, n, u_in.data_ptr(), u_out.data_ptr())
    out = u_out[: p.P].double().cpu().numpy()
    plan = s.plan()
    s.close()
    return out, st, plan


def _check_stats(st, ref, P, rtol):
    """Counts exact; means and variances relative to their natural scale."""
    for i in range(2):
        assert st[5 * i] == ref["count"][i]
        if ref["count"][i] == 0:
            continue
        scale_m = max(abs(ref["mean"][i]), np.sqrt(ref["var"][i]), 1e-300)
        assert abs(st[5 * i + 1] - ref["mean"][i]) <= rtol * scale_m
        assert abs(st[5 * i + 2] - ref["var"][i]) <= rtol * max(ref["var"][i], 1e-300)
    assert abs(st[10] - ref["gmean"]) <= rtol * max(abs(ref["gmean"]), np.sqrt(ref["gvar"]))
    assert abs(st[11] - ref["gvar"]) <= rtol * max(ref["gvar"], 1e-300)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 257, 1000, 4097, 50_001, 123_458, 400_002, 400_003])
def test_fine_fp64_matches_oracle(mmplib, orc, P):
    p = W.config2(P=P, N=8, T=0.4, dt=2e-3, precision="fp64", m0=0.3, s0=0.5)  # n_f = 25
    u0 = orc.initial(p)
    got, st, plan = _run_fine(mmplib, p, 3, u0)
    ref = orc.fine(p, 3, u0)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-11
    _check_stats(st, orc.restrict(p, ref), P, 1e-10)
    if P >= 400_000:
        assert plan["ctas_per_slice"] > 1  # the cross-CTA stage is exercised


def test_fine_fp64_multimodal_and_multiplicative(mmplib, orc):
    p = W.Problem(c3=1.0, c1=0.9, kappa=0.1, c0=0.05, B=0.3, BE=-0.2, B0=0.5, m0=0.1, s0=0.8, T=1.0, N=4,
                  dt=2e-3, P=70_001, n_regions=2, threshold=0.0, variant=W.MULTIMODAL, seed=77,
                  problem_tag=3, precision="fp64")
    u0 = orc.initial(p)
    got, st, _ = _run_fine(mmplib, p, 1, u0)
    ref = orc.fine(p, 1, u0)
    assert np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-11
    rs = orc.restrict(p, ref)
    _check_stats(st, rs, p.P, 1e-10)
    for k, ref in ((3, rs["min"][0]), (4, rs["max"][0]), (8, rs["min"][1]), (9, rs["max"][1])):
        assert abs(st[k] - ref) <= 1e-12 * max(1.0, abs(ref))


@pytest.mark.parametrize("P", [999, 200_001, 200_002, 200_003])
def test_fine_mixed_within_bounds(mmplib, orc, P):
    """FP32 particles on the same draws as the FP64 oracle: per-particle and
    moment errors stay inside the stated mixed-precision bounds."""
    p = W.config2(P=P, N=8, precision="mixed")  # n_f = 125
    u0 = orc.initial(p)
    got, st, _ = _run_fine(mmplib, p, 5, u0.astype(np.float32).astype(np.float64))
    ref = orc.fine(p, 5, u0)
    assert np.max(np.abs(got - ref)) < 2e-5
    rs = orc.restrict(p, ref)
    sd = np.sqrt(rs["gvar"])
    assert abs(st[10] - rs["gmean"]) < 2e-6 * max(abs(rs["gmean"]), sd)
    assert abs(st[11] - rs["gvar"]) < 1e-5 * rs["gvar"]


def test_fine_full_size_sampled(mmplib, orc):
    """Config-2 slice at full size (P = 1e6, n_f = 125) in FP64 against the
    oracle on the same draws."""
    p = W.config2(precision="fp64")
    u0 = orc.initial(p)
    got, st, plan = _run_fine(mmplib, p, 0, u0)
    ref = orc.fine(p, 0, u0)
    idx = np.arange(0, p.P, 9973)
    assert np.max(np.abs(got[idx] - ref[idx]) / np.maximum(np.abs(ref[idx]), 1.0)) < 1e-11
    _check_stats(st, orc.restrict(p, ref), p.P, 1e-10)
