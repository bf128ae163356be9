"""ctypes wrapper around the plain FP64 C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY.  It is imported by tests/, by
__graft_entry__.smoke() and by bench.py's cpu_baseline / reference legs,
never by the product package.  It shares no code with the CUDA library:
the only thing both sides take is the problem statement (a plain record of
parameters, see paper_2310_11365_gb300/workloads.py).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

UNIMODAL, MULTIMODAL, LEARNING = 0, 1, 2
MAX_REGIONS = 4
POLY, ROTATOR = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
             "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


class OrcProblem(C.Structure):
    _fields_ = [
        ("c3", C.c_double), ("c1", C.c_double), ("kappa", C.c_double), ("c0", C.c_double),
        ("B", C.c_double), ("BE", C.c_double), ("B0", C.c_double),
        ("m0", C.c_double), ("s0", C.c_double),
        ("T", C.c_double), ("N", C.c_int), ("dt", C.c_double), ("P", C.c_longlong),
        ("coarse_h", C.c_double), ("n_regions", C.c_int), ("threshold", C.c_double),
        ("variant", C.c_int), ("seed", C.c_uint64), ("problem_tag", C.c_uint32),
        ("tol", C.c_double), ("max_iter", C.c_int), ("coarse_model", C.c_int),
        ("threshold2", C.c_double), ("threshold3", C.c_double),
        ("family", C.c_int), ("K", C.c_double), ("g", C.c_double), ("q2", C.c_double),
    ]


class OrcStats(C.Structure):
    _fields_ = [
        ("count", C.c_longlong * MAX_REGIONS), ("mean", C.c_double * MAX_REGIONS),
        ("var", C.c_double * MAX_REGIONS), ("min", C.c_double * MAX_REGIONS),
        ("max", C.c_double * MAX_REGIONS), ("gmean", C.c_double), ("gvar", C.c_double),
    ]


class OrcMacro(C.Structure):
    _fields_ = [
        ("frac", C.c_double * MAX_REGIONS), ("mean", C.c_double * MAX_REGIONS),
        ("var", C.c_double * MAX_REGIONS),
    ]


class OrcResult(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int), ("converged", C.c_int), ("last_change", C.c_double),
        ("accepted_total", C.c_int), ("rejected_total", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        d = C.POINTER(C.c_double)
        pp = C.POINTER(OrcProblem)
        _lib.orc_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        _lib.orc_uniform.argtypes = [C.c_uint32]
        _lib.orc_uniform.restype = C.c_double
        _lib.orc_normal.argtypes = [pp, C.c_int, C.c_uint32, C.c_uint32, C.c_longlong]
        _lib.orc_normal.restype = C.c_double
        _lib.orc_initial.argtypes = [pp, d]
        _lib.orc_fine_steps.argtypes = [pp]
        _lib.orc_fine_steps.restype = C.c_int
        _lib.orc_fine_h.argtypes = [pp]
        _lib.orc_fine_h.restype = C.c_double
        _lib.orc_fine.argtypes = [pp, C.c_int, d, d, d]
        _lib.orc_wrap.argtypes = [C.c_double]
        _lib.orc_wrap.restype = C.c_double
        _lib.orc_region.argtypes = [pp, C.c_double]
        _lib.orc_restrict.argtypes = [pp, d, C.POINTER(OrcStats)]
        _lib.orc_mixture.argtypes = [pp, C.POINTER(OrcMacro), d, d]
        _lib.orc_match.argtypes = [pp, C.c_int, d, d, C.POINTER(C.c_int), C.POINTER(OrcStats), d, d]
        _lib.orc_coarse_steps.argtypes = [pp]
        _lib.orc_coarse_steps.restype = C.c_int
        _lib.orc_coarse_rhs.argtypes = [pp, C.POINTER(OrcMacro), d, d]
        _lib.orc_coarse.argtypes = [pp, C.POINTER(OrcMacro), C.POINTER(OrcMacro)]
        _lib.orc_lsq_fit.argtypes = [C.c_int, d, d, C.c_double, C.c_double, d, d]
        _lib.orc_lsq_fit.restype = C.c_int
        _lib.orc_extrapolate.argtypes = [C.c_double] * 4
        _lib.orc_extrapolate.restype = C.c_double
        _lib.orc_rate_generator.argtypes = [C.c_int, d, d]
        _lib.orc_rate_generator.restype = None
        _lib.orc_expm.argtypes = [C.c_int, d, d, d, d]
        _lib.orc_expm.restype = None
        _lib.orc_rate_fit.argtypes = [C.c_int, C.c_int, d, C.c_double, d]
        _lib.orc_rate_fit.restype = C.c_int
        _lib.orc_rate_propagate.argtypes = [C.c_int, d, C.c_double, d, C.c_int, d]
        _lib.orc_rate_propagate.restype = None
        _lib.orc_parareal_scalar.argtypes = [C.c_int, C.c_int] + [C.c_double] * 5 + [d, d]
        _lib.orc_parareal.argtypes = [pp, d, d, C.POINTER(OrcMacro), d, C.POINTER(OrcResult)]
        _lib.orc_parareal.restype = C.c_int
        _lib.orc_fine_serial.argtypes = [pp, d, C.POINTER(OrcStats), d]
        _lib.orc_adjoint.argtypes = [pp, d, d, d, d, d]
        _lib.orc_adjoint.restype = C.c_int
        _lib.orc_adjoint_loss.argtypes = [pp, d, d, d, d, d]
        _lib.orc_adjoint_loss.restype = C.c_int
    return _lib


def _dp(a: np.ndarray | None):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def problem(p) -> OrcProblem:
    """Build the oracle's own problem record from a workloads.Problem."""
    max_iter = p.max_iter if p.max_iter > 0 else p.N
    return OrcProblem(
        p.c3, p.c1, p.kappa, p.c0, p.B, p.BE, p.B0, p.m0, p.s0, p.T, p.N, p.dt, p.P,
        p.coarse_h, p.n_regions, p.threshold, p.variant, p.seed, p.problem_tag, p.tol, max_iter,
        p.coarse_model, p.threshold2, p.threshold3, p.family, p.K, p.g, p.q2,
    )


def philox(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform(word: int) -> float:
    return lib().orc_uniform(int(word) & 0xFFFFFFFF)


def normal(p, tag: int, j: int, n: int, particle: int) -> float:
    pr = problem(p)
    return lib().orc_normal(C.byref(pr), tag, j, n, particle)


def initial(p) -> np.ndarray:
    pr = problem(p)
    u = np.empty(p.P, np.float64)
    lib().orc_initial(C.byref(pr), _dp(u))
    return u


def wrap(x: float) -> float:
    """The plane rotator's shift of x modulo 2 pi into [-pi, pi]."""
    return lib().orc_wrap(float(x))


def fine_steps(p) -> int:
    return lib().orc_fine_steps(C.byref(problem(p)))


def fine_h(p) -> float:
    return lib().orc_fine_h(C.byref(problem(p)))


def fine(p, n: int, u_in: np.ndarray, return_means: bool = False):
    pr = problem(p)
    u_in = np.ascontiguousarray(u_in, dtype=np.float64)
    out = np.empty(p.P, np.float64)
    means = np.empty(fine_steps(p) + 1, np.float64) if return_means else None
    lib().orc_fine(C.byref(pr), n, _dp(u_in), _dp(out), _dp(means))
    return (out, means) if return_means else out


def stats_dict(st: OrcStats) -> dict:
    return {
        "count": list(st.count), "mean": list(st.mean), "var": list(st.var),
        "min": list(st.min), "max": list(st.max), "gmean": st.gmean, "gvar": st.gvar,
    }


def restrict(p, u: np.ndarray) -> dict:
    pr = problem(p)
    u = np.ascontiguousarray(u, dtype=np.float64)
    st = OrcStats()
    lib().orc_restrict(C.byref(pr), _dp(u), C.byref(st))
    return stats_dict(st)


def _stats_struct(p, u):
    pr = problem(p)
    st = OrcStats()
    lib().orc_restrict(C.byref(pr), _dp(u), C.byref(st))
    return st


def match(p, n: int, mu, sigma, do_region, u: np.ndarray) -> np.ndarray:
    pr = problem(p)
    u = np.ascontiguousarray(u, dtype=np.float64)
    st = _stats_struct(p, u)
    mu_a = np.ascontiguousarray(mu, dtype=np.float64)
    sg_a = np.ascontiguousarray(sigma, dtype=np.float64)
    do = (C.c_int * MAX_REGIONS)(*[int(x) for x in do_region])
    out = np.empty_like(u)
    lib().orc_match(C.byref(pr), n, _dp(mu_a), _dp(sg_a), do, C.byref(st), _dp(u), _dp(out))
    return out


def macro(frac, mean, var) -> OrcMacro:
    pad = lambda v: list(v) + [0.0] * (MAX_REGIONS - len(v))
    return OrcMacro((C.c_double * MAX_REGIONS)(*pad(frac)), (C.c_double * MAX_REGIONS)(*pad(mean)),
                    (C.c_double * MAX_REGIONS)(*pad(var)))


def mixture(p, frac, mean, var):
    pr = problem(p)
    m, v = C.c_double(), C.c_double()
    r = macro(frac, mean, var)
    lib().orc_mixture(C.byref(pr), C.byref(r), C.byref(m), C.byref(v))
    return m.value, v.value


def coarse_rhs(p, frac, mean, var):
    pr = problem(p)
    r = macro(frac, mean, var)
    dm = np.zeros(MAX_REGIONS)
    dv = np.zeros(MAX_REGIONS)
    lib().orc_coarse_rhs(C.byref(pr), C.byref(r), _dp(dm), _dp(dv))
    return dm, dv


def coarse(p, frac, mean, var):
    pr = problem(p)
    r = macro(frac, mean, var)
    out = OrcMacro()
    lib().orc_coarse(C.byref(pr), C.byref(r), C.byref(out))
    return list(out.frac), list(out.mean), list(out.var)


def coarse_steps(p) -> int:
    return lib().orc_coarse_steps(C.byref(problem(p)))


def lsq_fit(t, y, p0: float, dT: float):
    t = np.ascontiguousarray(t, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    a, b = C.c_double(), C.c_double()
    rc = lib().orc_lsq_fit(len(t), _dp(t), _dp(y), p0, dT, C.byref(a), C.byref(b))
    return rc, a.value, b.value


def extrapolate(p_k: float, alpha: float, beta: float, dt_ahead: float) -> float:
    return lib().orc_extrapolate(p_k, alpha, beta, dt_ahead)


def rate_generator(I: int, omega) -> np.ndarray:
    """A of dP/dt = A P from the rates omega[i (I-1) + (j < i ? j : j-1)] (D_i -> D_j)."""
    om = np.ascontiguousarray(omega, dtype=np.float64)
    A = np.zeros(I * I)
    lib().orc_rate_generator(I, _dp(om), _dp(A))
    return A.reshape(I, I)


def expm(X, dX=None):
    """The oracle's matrix exponential (and its derivative in direction dX)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[0]
    E = np.zeros(n * n)
    dE = np.zeros(n * n)
    dXa = None if dX is None else np.ascontiguousarray(dX, dtype=np.float64)
    lib().orc_expm(n, _dp(X), _dp(dXa), _dp(E), _dp(dE) if dX is not None else None)
    return (E.reshape(n, n), dE.reshape(n, n)) if dX is not None else E.reshape(n, n)


def rate_fit(fr, dT: float):
    """Fit the rates to fractions fr [(k+1), I]; returns (rc, omega)."""
    fr = np.ascontiguousarray(fr, dtype=np.float64)
    k, I = fr.shape[0] - 1, fr.shape[1]
    om = np.zeros(max(I * (I - 1), 1))
    rc = lib().orc_rate_fit(I, k, _dp(fr), dT, _dp(om))
    return rc, om[: I * (I - 1)]


def rate_propagate(I: int, omega, dT: float, p_in, m: int) -> np.ndarray:
    om = np.ascontiguousarray(omega, dtype=np.float64)
    pi = np.ascontiguousarray(p_in, dtype=np.float64)
    out = np.zeros(I)
    lib().orc_rate_propagate(I, _dp(om), dT, _dp(pi), m, _dp(out))
    return out


def parareal_scalar(N, K, u0, Fm, Fa, Gm, Ga, noise=None) -> np.ndarray:
    out = np.zeros((K + 1) * (N + 1))
    nz = None if noise is None else np.ascontiguousarray(noise, dtype=np.float64).reshape(-1)
    lib().orc_parareal_scalar(N, K, u0, Fm, Fa, Gm, Ga, _dp(nz), _dp(out))
    return out.reshape(K + 1, N + 1)


def parareal(p, u0: np.ndarray | None = None, want_parts: bool = False) -> dict:
    """Full MC-moments Parareal.  Returns the per-sweep global moments
    hist[k][n] = (M, V), the final macro states, the result record and
    (optionally) the final particle iterates u^K_n."""
    pr = problem(p)
    N = p.N
    K = pr.max_iter
    hist = np.full((K + 1, N + 1, 2), np.nan)
    mac = (OrcMacro * (N + 1))()
    parts = np.empty((N + 1) * p.P) if want_parts else None
    res = OrcResult()
    u0a = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    rc = lib().orc_parareal(C.byref(pr), _dp(u0a), _dp(hist.reshape(-1)), mac, _dp(parts), C.byref(res))
    if rc != 0:
        raise ValueError(f"orc_parareal returned {rc}")
    out = {
        "hist": hist[: res.sweeps + 1],
        "frac": np.array([list(m.frac) for m in mac]),
        "mean": np.array([list(m.mean) for m in mac]),
        "var": np.array([list(m.var) for m in mac]),
        "sweeps": res.sweeps, "converged": bool(res.converged), "last_change": res.last_change,
        "accepted": res.accepted_total, "rejected": res.rejected_total,
    }
    if want_parts:
        out["parts"] = parts.reshape(N + 1, p.P)
    return out


def fine_serial(p, u0: np.ndarray | None = None, want_parts: bool = False) -> dict:
    pr = problem(p)
    N = p.N
    sts = (OrcStats * (N + 1))()
    parts = np.empty((N + 1) * p.P) if want_parts else None
    u0a = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    lib().orc_fine_serial(C.byref(pr), _dp(u0a), sts, _dp(parts))
    out = {
        "stats": [stats_dict(s) for s in sts],
        "gmean": np.array([s.gmean for s in sts]),
        "gvar": np.array([s.gvar for s in sts]),
    }
    if want_parts:
        out["parts"] = parts.reshape(N + 1, p.P)
    return out


N_THETA = 7  # (c3, c1, kappa, c0, B0, B, BE)


def adjoint(p, gm, gv, u0: np.ndarray | None = None):
    """Gradient of sum_n gm[n] M_n + gv[n] V_n (n = 1..N) w.r.t.
    (c3, c1, kappa, c0, B0, B, BE), and the moments (M_n, V_n), n = 0..N."""
    pr = problem(p)
    gma = np.ascontiguousarray(gm, dtype=np.float64)
    gva = np.ascontiguousarray(gv, dtype=np.float64)
    grad = np.zeros(N_THETA)
    mom = np.zeros(2 * (p.N + 1))
    u0a = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    rc = lib().orc_adjoint(C.byref(pr), _dp(u0a), _dp(gma), _dp(gva), _dp(grad), _dp(mom))
    if rc != 0:
        raise ValueError(f"orc_adjoint returned {rc}")
    return grad, mom.reshape(p.N + 1, 2)


def adjoint_loss(p, m_tgt, v_tgt, u0: np.ndarray | None = None):
    """L = sum_n (M_n - m*_n)^2 + (V_n - v*_n)^2 and dL/d(c3, c1, kappa, c0, B0, B, BE)."""
    pr = problem(p)
    mt = np.ascontiguousarray(m_tgt, dtype=np.float64)
    vt = np.ascontiguousarray(v_tgt, dtype=np.float64)
    grad = np.zeros(N_THETA)
    L = C.c_double()
    u0a = None if u0 is None else np.ascontiguousarray(u0, dtype=np.float64)
    rc = lib().orc_adjoint_loss(C.byref(pr), _dp(u0a), _dp(mt), _dp(vt), _dp(grad), C.byref(L))
    if rc != 0:
        raise ValueError(f"orc_adjoint_loss returned {rc}")
    return L.value, grad
