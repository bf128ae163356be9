"""GPU adjoint of the serial fine propagator against the FP64 oracle adjoint
(same draws), against central differences of the GPU forward (common random
numbers), and through the torch.autograd.Function wrapper."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu

THETA = ("c3", "c1", "kappa", "c0", "B0", "B", "BE")


def _theta(p):
    return np.array([getattr(p, k) for k in THETA])


def _gpu_adjoint(p, gm, gv, ckpt_every):
    from paper_2310_11365_gb300.mmp import Adjoint, Solver

    s = Solver(p)
    adj = Adjoint(s, 0, ckpt_every)
    mom = adj.forward(_theta(p))
    grad = adj.backward(gm, gv)
    s.close()
    return grad, mom


def _general(p):
    """The same model with state-proportional and mean-field noise."""
    return p.scaled(B=0.2, BE=-0.15)


@pytest.mark.parametrize("general", [False, True])
@pytest.mark.parametrize("ckpt_every", [1, 7, 64])
def test_adjoint_fp64_matches_oracle(mmplib, orc, ckpt_every, general):
    """FP64 GPU adjoint = oracle adjoint to 1e-10 relative in all seven
    coefficients, for checkpoint intervals that do and do not divide the
    slice length, with additive noise (shift-form kernels) and with
    b = B x + BE E[X] + B0 (general-form kernels)."""
    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.2, s0=0.5, T=1.0, N=4, dt=0.01, P=3001, seed=17,
                      precision="fp64")
    if general:
        p = _general(p)
    rng = np.random.default_rng(1)
    gm, gv = rng.normal(size=p.N), rng.normal(size=p.N)
    g_ref, mom_ref = orc.adjoint(p, gm, gv)
    g, mom = _gpu_adjoint(p, gm, gv, ckpt_every)
    assert np.allclose(mom, mom_ref, rtol=1e-11, atol=1e-13)
    scale = np.maximum(np.abs(g_ref), 1e-12)
    assert np.max(np.abs(g - g_ref) / scale) < 1e-10, (g, g_ref)


@pytest.mark.parametrize("general", [False, True])
def test_adjoint_fp64_whole_gpu_shape_matches_oracle(mmplib, orc, general):
    """The reverse kernel's launch shape at a million particles (one
    512-thread CTA on every SM, three or four quads per thread, a ragged last
    quad) with a checkpoint interval that crosses slice ends: FP64 GPU
    adjoint = oracle adjoint to 1e-10 relative."""
    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.2, s0=0.5, T=0.2, N=2, dt=0.01, P=1_000_003, seed=29,
                      precision="fp64")
    if general:
        p = _general(p)
    rng = np.random.default_rng(2)
    gm, gv = rng.normal(size=p.N), rng.normal(size=p.N)
    g_ref, mom_ref = orc.adjoint(p, gm, gv)
    g, mom = _gpu_adjoint(p, gm, gv, 7)
    assert np.allclose(mom, mom_ref, rtol=1e-11, atol=1e-13)
    scale = np.maximum(np.abs(g_ref), 1e-12)
    assert np.max(np.abs(g - g_ref) / scale) < 1e-10, (g, g_ref)


def test_adjoint_fp64_config4_loss_gradient(mmplib, orc):
    """Config-4 loss L = sum (M - m*)^2 + (V - v*)^2 on the double-well model
    (targets from a run at (kappa, sigma) = (0.15, 0.65)), reduced to
    P = 1e4, T = 2, with checkpoints every 64 steps."""
    p = W.config4(P=10_000, T=2.0, N=8, precision="fp64")
    tgt = W.config4(P=10_000, T=2.0, N=8, precision="fp64", kappa=0.15, c1=1.0 - 0.15, B0=0.65,
                    seed=W.SEED_BASE + 5)
    st = orc.fine_serial(tgt)
    m_tgt, v_tgt = st["gmean"][1:], st["gvar"][1:]
    L_ref, g_ref = orc.adjoint_loss(p, m_tgt, v_tgt)
    from paper_2310_11365_gb300.mmp import Adjoint, Solver

    s = Solver(p)
    adj = Adjoint(s, 0, 64)
    mom = adj.forward(_theta(p))
    gm = 2 * (mom[1:, 0] - m_tgt)
    gv = 2 * (mom[1:, 1] - v_tgt)
    L = float(np.sum((mom[1:, 0] - m_tgt) ** 2 + (mom[1:, 1] - v_tgt) ** 2))
    g = adj.backward(gm, gv)
    s.close()
    assert abs(L - L_ref) <= 1e-10 * L_ref
    assert np.max(np.abs(g - g_ref) / np.maximum(np.abs(g_ref), 1e-12)) < 1e-9


def test_one_call_adjoint_loss(mmplib, orc):
    """mmp_adjoint (forward, loss, backward in one call) against the oracle's
    loss and gradient, FP64, general diffusion."""
    from paper_2310_11365_gb300.mmp import Adjoint, Solver

    p = _general(W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.2, s0=0.5, T=1.0, N=4, dt=0.01, P=3001, seed=17,
                               precision="fp64"))
    m_tgt, v_tgt = np.full(p.N, 0.1), np.full(p.N, 0.3)
    L_ref, g_ref = orc.adjoint_loss(p, m_tgt, v_tgt)
    s = Solver(p)
    adj = Adjoint(s, 0, 16)
    L, g = adj.loss_and_grad(_theta(p), m_tgt, v_tgt)
    s.close()
    assert abs(L - L_ref) <= 1e-10 * L_ref
    assert np.max(np.abs(g - g_ref) / np.maximum(np.abs(g_ref), 1e-12)) < 1e-10, (g, g_ref)


@pytest.mark.parametrize("general", [False, True])
def test_adjoint_mixed_close_to_oracle(mmplib, orc, general):
    """FP32 particles, FP64 accumulation: gradient within 1e-3 relative of the
    FP64 oracle on the same draws (P = 1e4), each coefficient's error
    measured against its own size or, for a coefficient whose derivative
    nearly vanishes, against 1e-3 of the largest."""
    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.0, s0=0.3, T=2.0, N=8, dt=1e-3, P=10_000, seed=23,
                      precision="mixed")
    if general:
        p = _general(p)
    rng = np.random.default_rng(5)
    gm, gv = rng.normal(size=p.N), rng.normal(size=p.N)
    g_ref, _ = orc.adjoint(p.scaled(precision="fp64"), gm, gv)
    g, _ = _gpu_adjoint(p, gm, gv, 64)
    scale = np.maximum(np.abs(g_ref), 1e-3 * np.max(np.abs(g_ref)))
    assert np.max(np.abs(g - g_ref) / scale) < 1e-3, (g, g_ref)


@pytest.mark.parametrize("general", [False, True])
def test_adjoint_matches_gpu_central_differences(mmplib, general):
    """Central differences of the GPU FP64 forward with common draws
    (h = 1e-4) agree with the GPU adjoint to 1e-6 relative in all seven
    coefficients.  From additive noise, a step in B or BE switches the
    forward to the general-form kernel (mmp_set_params with 7 values)."""
    from paper_2310_11365_gb300.mmp import Adjoint, Solver

    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=1.0, N=4, dt=0.005, P=50_001, seed=9, precision="fp64")
    if general:
        p = _general(p)
    rng = np.random.default_rng(3)
    gm, gv = rng.normal(size=p.N), rng.normal(size=p.N)
    s = Solver(p)
    adj = Adjoint(s, 0, 16)
    th = _theta(p)
    adj.forward(th)
    g = adj.backward(gm, gv)

    def objective(theta):
        mom = adj.forward(theta)
        return float(gm @ mom[1:, 0] + gv @ mom[1:, 1])

    for k in range(len(THETA)):
        h = 1e-4 * max(1.0, abs(th[k]))
        e = np.zeros(len(THETA))
        e[k] = h
        fd = (objective(th + e) - objective(th - e)) / (2 * h)
        assert abs(g[k] - fd) <= 1e-6 * max(abs(fd), 1e-6), (THETA[k], g[k], fd)
    s.close()


def test_autograd_function_double_well(mmplib, orc):
    """torch.autograd through FineMoments with the double-well
    parameterisation (kappa, sigma, a, b): the gradient equals the oracle's
    chain-ruled adjoint."""
    import torch

    from paper_2310_11365_gb300.mmp import Adjoint, Solver, double_well_theta, fine_moments

    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.1, s0=0.4, T=1.0, N=4, dt=0.01, P=4001, seed=31,
                      precision="fp64")
    s = Solver(p)
    adj = Adjoint(s, 0, 32)
    params = torch.tensor([0.1, 0.7, 0.25, 0.5], dtype=torch.float64, requires_grad=True)
    theta = double_well_theta(params[0], params[1], params[2], params[3])
    mom = fine_moments(theta, adj)
    m_tgt = torch.full((p.N,), 0.2, dtype=torch.float64)
    v_tgt = torch.full((p.N,), 0.3, dtype=torch.float64)
    loss = ((mom[1:, 0] - m_tgt) ** 2 + (mom[1:, 1] - v_tgt) ** 2).sum()
    loss.backward()
    L_ref, g_ref = orc.adjoint_loss(p, m_tgt.numpy(), v_tgt.numpy())
    # chain rule: c3 = 4a, c1 = 2b - kappa, kappa_m = kappa, B0 = sigma
    want = np.array([g_ref[2] - g_ref[1], g_ref[4], 4 * g_ref[0], 2 * g_ref[1]])
    assert abs(loss.item() - L_ref) <= 1e-10 * L_ref
    assert np.max(np.abs(params.grad.numpy() - want) / np.maximum(np.abs(want), 1e-12)) < 1e-9
    s.close()


def test_set_params_switches_form(mmplib):
    """mmp_set_params with 7 values: a single problem moves between the
    additive and general kernel forms (and back, bit for bit); a batch, whose
    problems share one form, refuses the switch and keeps its coefficients."""
    from paper_2310_11365_gb300.mmp import Adjoint, Solver, mmp_set_params

    p = W.cubic(1.0, 0.5, m0=0.5, s0=0.2, T=1.0, N=2, dt=0.01, P=20_001, seed=4, precision="fp64")
    s = Solver(p)
    adj = Adjoint(s, 0, 16)
    th = _theta(p)
    m0 = adj.forward(th)
    m1 = adj.forward(th + np.array([0, 0, 0, 0, 0, 0.3, 0.1]))
    assert not np.array_equal(m0, m1)
    m2 = adj.forward(th)
    assert np.array_equal(m0, m2)
    s.close()

    batch = [W.config1(N=4, T=1.0, problem_tag=1), W.config1(N=4, T=1.0, problem_tag=2)]
    s = Solver(batch)
    with pytest.raises(Exception):
        mmp_set_params(s.ctx, 0, np.array([0, batch[0].c1, batch[0].kappa, 0, batch[0].B0, 0.2, 0.0]))
    mmp_set_params(s.ctx, 0, np.array([0, batch[0].c1, batch[0].kappa, 0, batch[0].B0 * 1.1, 0.0, 0.0]))
    s.close()
