"""GPU plane rotator (Sec. 5, Example "Unimodal plane rotator",
Eq. SDE_plane_rotator) against the FP64 oracle: the drift
K (S cos x - C sin x) - g sin x through the ensemble means S, C of sin X and
cos X (two group sums per step), additive noise, and every particle shifted
modulo 2 pi into [-pi, pi] after each step and in the initial ensemble.

FP64 results match the oracle to 1e-10 relative (particle values to 1e-11
absolute, as angles); the mixed form (FP32 particles, FP64 sums) stays within
the bounds stated below.  Sizes span one and many CTAs per slice and ragged
tails; every coarse model of the example is run."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _rot(**kw):
    base = dict(P=4001, N=5, T=2.0, dt=1e-2, precision="fp64", tol=1e-9)
    base.update(kw)
    return W.plane_rotator(**base)


def _angle_diff(a, b):
    """a - b taken modulo 2 pi into [-pi, pi)."""
    return np.mod(a - b + np.pi, 2 * np.pi) - np.pi


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


def test_initial_ensemble_is_shifted(mmplib, orc):
    from paper_2310_11365_gb300.mmp import Solver

    p = _rot(P=100_003)
    s = Solver(p)
    u0 = s.particles(0).double().cpu().numpy()
    s.close()
    ref = orc.initial(p)
    assert np.all(np.abs(u0) <= np.pi)
    assert np.max(np.abs(u0 - ref)) < 1e-14


@pytest.mark.parametrize("P", [1, 3, 5, 257, 4097, 60_001, 400_003])
def test_fine_fp64_matches_oracle(mmplib, orc, P):
    p = _rot(P=P, N=4, T=0.8, dt=1e-2)  # 20 steps per slice
    u0 = orc.initial(p)
    got, st, plan = _run_fine(mmplib, p, 2, u0)
    ref = orc.fine(p, 2, u0)
    assert np.all(np.abs(got) <= np.pi)
    assert np.max(np.abs(_angle_diff(got, ref))) < 1e-11
    r = orc.restrict(p, ref)
    assert st[0] == P
    assert abs(st[10] - r["gmean"]) <= 1e-10 * max(abs(r["gmean"]), np.sqrt(r["gvar"]))
    assert abs(st[11] - r["gvar"]) <= 1e-10 * max(r["gvar"], 1e-300)
    if P >= 400_000:
        assert plan["ctas_per_slice"] > 1  # the cross-CTA sums of sin and cos are exercised


def test_fine_mixed_within_bounds(mmplib, orc):
    """FP32 particles against the FP64 oracle on the same draws, 20 steps:
    every particle within 2e-5 (as an angle), the slice-end mean and variance
    within 2e-6 of their scale once the particles that the FP32 and FP64
    shifts put on opposite ends of [-pi, pi] are set aside."""
    p = _rot(P=200_003, N=4, T=0.8, dt=1e-2, precision="mixed")
    u0 = orc.initial(p.scaled(precision="fp64"))
    got, st, _ = _run_fine(mmplib, p, 1, u0.astype(np.float32).astype(np.float64))
    ref = orc.fine(p.scaled(precision="fp64"), 1, u0.astype(np.float32).astype(np.float64))
    d = _angle_diff(got, ref)
    assert np.max(np.abs(d)) < 2e-5
    same = np.abs(got - ref) < np.pi
    flips = int(np.sum(~same))
    assert flips <= 3
    r = orc.restrict(p.scaled(precision="fp64", P=int(same.sum())), ref[same])
    gm = got[same].mean()
    gv = got[same].var()
    assert abs(gm - r["gmean"]) <= 2e-6 * max(abs(r["gmean"]), np.sqrt(r["gvar"]))
    assert abs(gv - r["gvar"]) <= 2e-6 * r["gvar"]
    if flips == 0:
        assert abs(st[10] - r["gmean"]) <= 2e-6 * max(abs(r["gmean"]), np.sqrt(r["gvar"]))
        assert abs(st[11] - r["gvar"]) <= 2e-6 * r["gvar"]


@pytest.mark.parametrize("model", [W.CLOSURE, W.TAYLOR, W.TAYLOR1, W.SIGMA2, W.SIGMA3])
def test_parareal_fp64_matches_oracle(mmplib, orc, model):
    from paper_2310_11365_gb300.mmp import Solver

    p = _rot(coarse_model=model)
    s = Solver(p)
    k = s.run()
    mom = s.moments(0)
    st = s.status(0)
    s.close()
    ref = orc.parareal(p)
    assert k == ref["sweeps"] and st["dev_err"] == 0, (model, k, ref["sweeps"])
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert abs(mom[n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V)), (model, n)
        assert abs(mom[n, 7] - V) <= 1e-10 * V, (model, n)


def test_property_3_3_bitwise(mmplib, orc):
    """After k sweeps the slice ends t_0..t_k equal the serial fine run of
    the same launch shape bit for bit (the GPU against itself): the macro
    states are the serial run's restrictions and u^k_k is its ensemble."""
    import torch

    from paper_2310_11365_gb300.mmp import Solver

    k = 2
    p = _rot(P=60_001, tol=0.0, max_iter=k)
    s = Solver(p)
    s.run()
    mom = s.moments(0)
    ser, last = s.serial(0, n_end=k, want_last=True)
    for n in range(k + 1):
        assert mom[n, 1] == ser[n, 1] and mom[n, 2] == ser[n, 2], n
    assert torch.equal(s.particles(k), last)
    s.close()


def test_parareal_mixed_within_bounds(mmplib, orc):
    """The mixed form against the FP64 oracle over a whole run of the
    example's settings (scaled down): slice-end means within 2e-6 of
    max(|M|, sqrt(V)) and variances within 2e-5 relative, after the same
    number of sweeps."""
    from paper_2310_11365_gb300.mmp import Solver

    p = _rot(P=100_003, N=5, T=2.0, dt=1e-2, precision="mixed", tol=0.0, max_iter=3)
    s = Solver(p)
    s.run()
    mom = s.moments(0)
    s.close()
    ref = orc.parareal(p.scaled(precision="fp64"))
    for n in range(p.N + 1):
        M, V = ref["hist"][-1][n]
        assert abs(mom[n, 6] - M) <= 2e-6 * max(abs(M), np.sqrt(V)), n
        assert abs(mom[n, 7] - V) <= 2e-5 * V, n


def test_rotator_with_a_polynomial_problem_in_one_context(mmplib, orc):
    """A context that holds a rotator and a cubic problem runs them one by
    one (the batched kernel is the polynomial family's); each matches its
    oracle run."""
    from paper_2310_11365_gb300.mmp import Solver

    probs = [_rot(problem_tag=3), W.config2(P=4001, N=4, T=0.5, precision="fp64", problem_tag=4, tol=1e-9)]
    s = Solver(probs)
    s.run()
    for i, p in enumerate(probs):
        ref = orc.parareal(p)
        mom = s.moments(i)
        assert s.status(i)["sweeps"] == ref["sweeps"]
        for n in range(p.N + 1):
            M, V = ref["hist"][-1][n]
            assert abs(mom[n, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V)), (i, n)
    s.close()


def test_adjoint_and_parameter_switch_are_refused(mmplib):
    from paper_2310_11365_gb300.mmp import MMPError, Solver

    s = Solver(_rot(N=2))
    with pytest.raises(MMPError) as e:
        mmplib.mmp_adjoint_workspace_size(s.ctx, 0, 8)
    assert e.value.code == -3
    with pytest.raises(MMPError) as e:
        mmplib.mmp_set_params(s.ctx, 0, [0.0, 0.0, 0.0, 0.0, 0.5])
    assert e.value.code == -3
    s.close()
