"""Error paths on the GPU, none of which faults, traps or hangs the device:
workspace checks, calls out of order, and non-finite values reported through
the device status word.  After each the library goes on working."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _code(mmplib, call):
    with pytest.raises(mmplib.MMPError) as e:
        call()
    return e.value.code


def _healthy(prec="fp64"):
    return W.config1(P=2001, N=4, T=1.0, precision=prec)


def test_context_workspace_too_small_or_misaligned(mmplib):
    """mmp_create refuses a workspace one 256-byte block short of the size
    mmp_workspace_size gives, and one 16 bytes off its 256-byte boundary,
    with MMP_ERR_WORKSPACE (nothing is written); the full one works."""
    import torch

    p = _healthy()
    n = mmplib.mmp_workspace_size([p])
    ws = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
    assert _code(mmplib, lambda: mmplib.mmp_create([p], ws.data_ptr(), n - 256)) == -2
    assert _code(mmplib, lambda: mmplib.mmp_create([p], ws.data_ptr() + 16, n)) == -2
    ctx = mmplib.mmp_create([p], ws.data_ptr(), n)
    mmplib.mmp_destroy(ctx)


def test_calls_before_lift(mmplib):
    """Sweeps, moments and slice-end particles before the lift are
    MMP_ERR_STATE; the same context then solves the problem."""
    from paper_2310_11365_gb300.mmp import Solver

    s = Solver(_healthy())
    for call in (lambda: s.iterate(1), s.moments, lambda: s.particles(1)):
        assert _code(mmplib, call) == -7
    assert s.run() >= 1
    assert s.status()["dev_err"] == 0
    s.close()


def test_adjoint_workspace_and_order(mmplib):
    """The adjoint: backward before any forward and backward with another
    workspace than the forward's are MMP_ERR_STATE; a short or misaligned
    workspace is MMP_ERR_WORKSPACE; a checkpoint interval of 0 is
    MMP_ERR_INVALID_ARG.  A proper forward and backward follow."""
    import torch

    from paper_2310_11365_gb300.mmp import Solver

    p = W.double_well(0.25, 0.5, 0.1, 0.7, m0=0.2, s0=0.5, T=1.0, N=4, dt=0.01, P=3001, seed=17,
                      precision="fp64")
    s = Solver(p)
    c = 8
    nb = mmplib.mmp_adjoint_workspace_size(s.ctx, 0, c)
    a = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    b = torch.empty(nb, dtype=torch.uint8, device="cuda")
    g = np.ones(p.N)
    assert _code(mmplib, lambda: mmplib.mmp_adjoint_backward(s.ctx, 0, g, g, a.data_ptr(), nb)) == -7
    assert _code(mmplib, lambda: mmplib.mmp_adjoint_forward(s.ctx, 0, c, a.data_ptr(), nb - 256, p.N)) == -2
    assert _code(mmplib, lambda: mmplib.mmp_adjoint_forward(s.ctx, 0, c, a.data_ptr() + 16, nb, p.N)) == -2
    assert _code(mmplib, lambda: mmplib.mmp_adjoint_forward(s.ctx, 0, 0, a.data_ptr(), nb, p.N)) == -1
    mom = mmplib.mmp_adjoint_forward(s.ctx, 0, c, a.data_ptr(), nb, p.N)
    assert _code(mmplib, lambda: mmplib.mmp_adjoint_backward(s.ctx, 0, g, g, b.data_ptr(), nb)) == -7
    grad = mmplib.mmp_adjoint_backward(s.ctx, 0, g, g, a.data_ptr(), nb)
    assert np.all(np.isfinite(mom)) and np.all(np.isfinite(grad))
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_non_finite_values_are_reported(mmplib, orc, prec):
    """dX = X^3 dt + 0.3 dW from X0 ~ N(1, 0.3^2) blows up before t = 1/2:
    the fine run overflows (the oracle's ensemble mean is NaN from the first
    slice end on), the sweep returns MMP_ERR_NUMERIC (-5) and the problem's
    status word keeps it.  The device stays usable: a fresh context solves a
    healthy problem with a clean status."""
    from paper_2310_11365_gb300.mmp import Solver

    p = W.Problem(c3=-1.0, B0=0.3, m0=1.0, s0=0.3, T=2.0, N=4, dt=0.01, P=1001, coarse_h=0.25,
                  seed=7, tol=1e-8, precision=prec)
    gmean = orc.fine_serial(p.scaled(precision="fp64"))["gmean"]
    assert np.isfinite(gmean[0]) and not np.any(np.isfinite(gmean[1:]))
    s = Solver(p)
    assert _code(mmplib, s.run) == -5
    assert s.status()["dev_err"] == -5
    s.close()
    ok = Solver(_healthy(prec))
    assert ok.run() >= 1
    assert ok.status()["dev_err"] == 0
    ok.close()


@pytest.mark.parametrize("channel", [0, 1])
def test_bounded_wait_runs_out_and_the_device_stays_usable(mmplib, orc, channel):
    """Failure detection of the group exchange: one CTA of a two-CTA group
    waits for a peer that never publishes (channel 0: the epoch-flag records;
    channel 1: the tagged step words of float particles).  The wait gives up
    after its 20 ms limit, sets the timeout bit and returns MMP_ERR_TIMEOUT;
    a group of one waits for nobody; the library then solves a healthy
    problem."""
    import time

    import torch

    from paper_2310_11365_gb300.mmp import Solver

    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    rc, st = mmplib.mmp_probe_wait(channel, 2, 20.0, ws.data_ptr(), ws.numel())
    waited = time.perf_counter() - t0
    assert rc == -6 and st & 1, (rc, st)
    assert 0.015 < waited < 5.0, waited
    assert mmplib.mmp_probe_wait(channel, 1, 20.0, ws.data_ptr(), ws.numel()) == (0, 0)
    # argument checks before any launch
    assert mmplib.mmp_probe_wait(2, 2, 20.0, ws.data_ptr(), ws.numel())[0] == -1
    assert mmplib.mmp_probe_wait(channel, 2, 0.5, ws.data_ptr(), ws.numel())[0] == -1
    assert mmplib.mmp_probe_wait(channel, 2, 20.0, ws.data_ptr() + 16, ws.numel())[0] == -2
    assert mmplib.mmp_probe_wait(channel, 64, 20.0, ws.data_ptr(), 1024)[0] == -2
    p = _healthy()
    s = Solver(p)
    k = s.run()
    ref = orc.parareal(p)
    assert k == ref["sweeps"] and s.status()["dev_err"] == 0
    M, V = ref["hist"][-1][p.N]
    assert abs(s.moments()[p.N, 6] - M) <= 1e-10 * max(abs(M), np.sqrt(V))
    s.close()
