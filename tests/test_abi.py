"""The C-ABI library loads and exports every symbol include/mmp.h declares;
host-side argument checks reject bad descriptors before any CUDA call."""
import ctypes as C
import os
import re

import pytest

from paper_2310_11365_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mmp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mmp_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(mmplib):
    lib = C.CDLL(mmplib.LIB_PATH)
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(mmplib.EXPORTED)


def test_strerror_and_version(mmplib):
    assert mmplib.mmp_version() >= 100
    assert mmplib.mmp_strerror(0) == "ok"
    for code in range(-7, 0):
        assert mmplib.mmp_strerror(code) not in ("ok", "unknown error")


@pytest.mark.parametrize("bad", [
    dict(N=0), dict(N=70000), dict(P=0), dict(T=-1.0), dict(dt=0.0), dict(coarse_h=0.0),
    dict(n_regions=5), dict(n_regions=0), dict(variant=7), dict(s0=-0.1), dict(c3=float("nan")),
    dict(tol=-1.0), dict(n_regions=3, threshold=0.5, threshold2=0.5),
    dict(n_regions=4, threshold=-1.0, threshold2=0.0, threshold3=-0.5),
    dict(n_regions=3, threshold=0.0, threshold2=float("inf")),
    dict(P=2**31), dict(N=1, T=1e3, dt=1e-7), dict(N=1, T=1.0, coarse_h=1e-9), dict(coarse_model=5),
    dict(B0=float("inf")), dict(precision="fp64", m0=float("nan")),
])
def test_invalid_descriptor_rejected_on_host(mmplib, bad):
    p = W.config1(**bad)
    with pytest.raises(mmplib.MMPError) as e:
        mmplib.mmp_workspace_size([p])
    assert e.value.code == -1


def test_bad_precision_rejected(mmplib):
    d = mmplib.desc(W.config1())
    d.precision = 5
    n = C.c_size_t()
    assert mmplib.load().mmp_workspace_size(C.byref(d), 1, C.byref(n)) == -1


def test_null_arguments(mmplib):
    lib = mmplib.load()
    assert lib.mmp_workspace_size(None, 1, None) == -1
    assert lib.mmp_create(None, None, 0, None, 0, None) == -1
    assert lib.mmp_lift(None) == -1
    assert lib.mmp_status(None, 0, None, None, None, None) == -1


def test_python_surface(mmplib):
    """The binding's user-facing names: the problem record, the one-call
    solve, and the autograd function over the adjoint (built on first
    access, so that importing the binding does not import torch)."""
    import torch

    assert mmplib.Problem is W.Problem
    assert callable(mmplib.run) and callable(mmplib.fine_moments)
    assert issubclass(mmplib.FineMoments, torch.autograd.Function)
    assert mmplib.FineMoments is mmplib.FineMoments
    assert mmplib.N_THETA == len(mmplib.THETA_NAMES) == 7


def test_set_params_arity(mmplib):
    lib = mmplib.load()
    theta = (C.c_double * 7)(*([0.0] * 7))
    assert lib.mmp_set_params(None, 0, theta, 7) == -1


def test_workspace_checked_before_any_device_work(mmplib):
    """A NULL or misaligned device workspace is MMP_ERR_WORKSPACE (-2), for
    the context, the adjoint and the autotuner, before any CUDA call (so it
    holds without a GPU); a missing context is MMP_ERR_INVALID_ARG."""
    lib = mmplib.load()
    d = mmplib.desc(W.config1())
    ctx = C.c_void_p()
    for ws in (None, 8, 4096 + 16):
        assert lib.mmp_create(C.byref(ctx), C.byref(d), 1, ws, 1 << 20, None) == -2
        assert not ctx.value
    best = C.c_int()
    assert lib.mmp_autotune(C.byref(d), None, 0, 0, 8, 1 << 20, None, C.byref(best), None) == -2
    assert lib.mmp_autotune(None, None, 0, 0, 4096, 1 << 20, None, C.byref(best), None) == -1
    assert lib.mmp_autotune(C.byref(d), None, 0, 0, 4096, 1 << 20, None, None, None) == -1
    n = C.c_size_t()
    v = (C.c_double * 8)()
    assert lib.mmp_adjoint_workspace_size(None, 0, 8, C.byref(n)) == -1
    assert lib.mmp_adjoint_forward(None, 0, 8, 4096, 1 << 20, v) == -1
    assert lib.mmp_adjoint_backward(None, 0, v, v, 4096, 1 << 20, v) == -1
    assert lib.mmp_adjoint(None, 0, v, v, 8, 4096, 1 << 20, v, v) == -1
    assert lib.mmp_iterate(None, 1, None) == -1
    assert lib.mmp_get_moments(None, 0, v) == -1


def test_plane_rotator_descriptors_checked_on_the_host(mmplib):
    """The plane rotator (family MMP_FAMILY_ROTATOR) has additive noise and
    one region: a state-dependent diffusion is refused as invalid, more
    regions as unsupported, an unknown family or coarse model as invalid, all
    before any device work.  The second-moment coupling of App. C is refused
    by the binding (the kernels do not carry it)."""
    lib = mmplib.load()
    n = C.c_size_t()

    def rc(p, **fields):
        d = mmplib.desc(p)
        for k, v in fields.items():
            setattr(d, k, v)
        return lib.mmp_workspace_size(C.byref(d), 1, C.byref(n))

    r = W.plane_rotator(P=1000)
    assert rc(r, B=0.5) == -1
    assert rc(r, BE=0.5) == -1
    assert rc(r, n_regions=2, threshold=0.0) == -3
    assert rc(r, family=2) == -1
    assert rc(r, coarse_model=5) == -1
    assert rc(r, K=float("nan")) == -1
    with pytest.raises(mmplib.MMPError) as e:
        mmplib.desc(W.polynomial_drift())
    assert e.value.code == -3


def test_probe_wait_arguments_checked_on_the_host(mmplib):
    """The failure-detection self-test refuses an unknown channel, a group
    size or wait limit out of range, and a NULL, misaligned or short
    scratch, before any device work."""
    lib = mmplib.load()
    assert lib.mmp_probe_wait(2, 2, 20.0, 4096, 1 << 16, None, None) == -1
    assert lib.mmp_probe_wait(0, 0, 20.0, 4096, 1 << 16, None, None) == -1
    assert lib.mmp_probe_wait(0, 1025, 20.0, 4096, 1 << 20, None, None) == -1
    assert lib.mmp_probe_wait(0, 2, 0.5, 4096, 1 << 16, None, None) == -1
    assert lib.mmp_probe_wait(0, 2, 2e4, 4096, 1 << 16, None, None) == -1
    assert lib.mmp_probe_wait(0, 2, 20.0, None, 1 << 16, None, None) == -2
    assert lib.mmp_probe_wait(0, 2, 20.0, 4096 + 16, 1 << 16, None, None) == -2
    assert lib.mmp_probe_wait(0, 2, 20.0, 4096, 2 * 548 + 3, None, None) == -2


def test_probe_step_arguments_checked_on_the_host(mmplib):
    import ctypes as C

    lib = mmplib.load()
    r = C.c_double()
    assert lib.mmp_probe_step(2, 4096, 64, None, C.byref(r)) == -1
    assert lib.mmp_probe_step(-1, 4096, 64, None, C.byref(r)) == -1
    assert lib.mmp_probe_step(0, 4096, 64, None, None) == -1
    assert lib.mmp_probe_step(1, None, 64, None, C.byref(r)) == -2
    assert lib.mmp_probe_step(1, 4096 + 16, 64, None, C.byref(r)) == -2
    assert lib.mmp_probe_step(0, 4096, 4, None, C.byref(r)) == -2


def test_normals_arguments_checked_on_the_host(mmplib):
    """mmp_normals refuses a misaligned output, an oversized count, a tag
    past 8 bits and a slice past 24 bits before any launch."""
    lib = mmplib.load()
    d = mmplib.desc(W.config1())
    assert lib.mmp_normals(C.byref(d), 0, 0, 0, 16, 4096 + 4, None) == -1   # FP64 needs 8-byte alignment
    assert lib.mmp_normals(C.byref(d), 0, 0, 0, (4 << 32) + 1, 4096, None) == -1
    assert lib.mmp_normals(C.byref(d), 256, 0, 0, 16, 4096, None) == -1
    assert lib.mmp_normals(C.byref(d), 0, 0, 1 << 24, 16, 4096, None) == -1
    assert lib.mmp_normals(C.byref(d), 0, 0, 0, 0, 4096, None) == 0        # nothing to do
