"""mmp_fine_static: the fine propagation for callers that cannot allocate
device memory (code inside an application or framework that owns the GPU's
memory through its own allocator, latency-bound loops where a cudaMalloc
could stall the device).  Run in the same launch shape as mmp_fine, it must
give exactly what mmp_fine gives on the same input, call after call,
although every call reuses the library's one static scratch array (this
file is collected last on purpose; it also passes on its own)."""
import numpy as np
import pytest

from paper_2310_11365_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference(mmplib, p, n, u_in):
    """The existing entry point, mmp_fine, with a context and workspace."""
    import torch

    from paper_2310_11365_gb300.mmp import Solver

    s = Solver(p)
    out = torch.zeros_like(u_in)
    st = mmplib.mmp_fine(s.ctx, 0, n, u_in.data_ptr(), out.data_ptr())
    s.close()
    return out, st


def _static(mmplib, p, n, u_in):
    import torch

    out = torch.full_like(u_in, float("nan"))
    st = torch.full((mmplib.STAT_STRIDE,), float("nan"), dtype=torch.float64, device="cuda")
    mmplib.mmp_fine_static(p, n, u_in.data_ptr(), out.data_ptr(), st.data_ptr())
    torch.cuda.synchronize()
    return out, st.cpu().numpy()


def _inputs(orc, p):
    import torch

    dt = torch.float32 if p.precision == "mixed" else torch.float64
    u0 = torch.from_numpy(orc.initial(p)).to(dt).cuda()
    return u0


@pytest.mark.parametrize("make", [
    lambda: W.config2(P=300_001, N=8, precision="mixed"),
    lambda: W.config3(P=40_003, N=16, T=2.0, precision="fp64"),
])
def test_static_matches_mmp_fine_on_consecutive_calls(mmplib, orc, make):
    import torch

    p = make()
    u_in = _inputs(orc, p)
    ref_u, ref_st = _reference(mmplib, p, 3, u_in)
    for call in range(2):
        got_u, got_st = _static(mmplib, p, 3, u_in)
        assert got_st[14] == 0.0, call  # device status
        # the same kernel in the same launch shape on the same input: bit for bit
        assert torch.equal(got_u, ref_u), call
        for k in (0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11):
            assert got_st[k] == ref_st[k], (call, k)


def test_static_consecutive_calls_of_different_shapes(mmplib, orc):
    """A large call followed by a small one and a large one again: the state
    the first call leaves in the shared array does not leak into the next."""
    problems = [W.config2(P=600_001, N=8, precision="mixed"), W.config1(P=2000, precision="fp64"),
                W.config2(P=600_001, N=8, precision="mixed")]
    for p in problems:
        u_in = _inputs(orc, p)
        ref_u, ref_st = _reference(mmplib, p, 1, u_in)
        got_u, got_st = _static(mmplib, p, 1, u_in)
        assert got_st[14] == 0.0
        assert got_st[0] == ref_st[0]
        assert abs(got_st[10] - ref_st[10]) <= 1e-10 * max(abs(ref_st[10]), np.sqrt(ref_st[11]))
        assert abs(got_st[11] - ref_st[11]) <= 1e-10 * ref_st[11]


def test_static_rejects_oversized_problem(mmplib):
    """Problems whose launch shape needs more CTAs per slice than the static
    array serves are refused on the host.  The buffers passed hold all P
    values, so the call would stay in bounds even if it were not refused."""
    import torch

    p = W.config2(P=20_000_001, N=1, T=0.125, precision="mixed")
    u_in = torch.zeros(p.P, dtype=torch.float32, device="cuda")
    u_out = torch.empty_like(u_in)
    st = torch.full((mmplib.STAT_STRIDE,), -1.0, dtype=torch.float64, device="cuda")
    with pytest.raises(mmplib.MMPError) as e:
        mmplib.mmp_fine_static(p, 0, u_in.data_ptr(), u_out.data_ptr(), st.data_ptr())
    assert e.value.code == -3
    torch.cuda.synchronize()
    assert torch.all(st == -1.0)  # nothing ran
