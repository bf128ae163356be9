"""Thin Python binding of libmmp.so (C-ABI in include/mmp.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory (the workspace and any
ensembles) and the stream.  There is no fallback: if libmmp.so is missing
or cannot load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads

Problem = workloads.Problem  # the problem record every call takes

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmmp.so")

MMP_OK = 0
MMP_FP64, MMP_MIXED = 0, 1
MMP_UNIMODAL, MMP_MULTIMODAL, MMP_LEARNING = 0, 1, 2
MOMENT_STRIDE = 16   # MMP_MOMENT_STRIDE
STAT_STRIDE = 32     # MMP_STAT_STRIDE
MAX_REGIONS = 4      # MMP_MAX_REGIONS


def moment_region(i: int) -> int:
    """Offset of region i's (fraction, mean, variance) in a moment row."""
    return 3 * i if i < 2 else 3 * i + 2


def stat_region(i: int) -> int:
    """Offset of region i's (count, mean, variance, min, max) in a restriction record."""
    return 5 * i if i < 2 else 5 * i + 6
N_THETA = 7         # MMP_N_THETA: (c3, c1, kappa, c0, B0, B, BE)

ERRORS = {
    -1: "MMP_ERR_INVALID_ARG", -2: "MMP_ERR_WORKSPACE", -3: "MMP_ERR_UNSUPPORTED",
    -4: "MMP_ERR_CUDA", -5: "MMP_ERR_NUMERIC", -6: "MMP_ERR_TIMEOUT", -7: "MMP_ERR_STATE",
}

EXPORTED = [
    "mmp_strerror", "mmp_version", "mmp_last_cuda_error", "mmp_workspace_size", "mmp_create",
    "mmp_destroy", "mmp_set_initial", "mmp_lift", "mmp_iterate", "mmp_run", "mmp_status",
    "mmp_get_moments", "mmp_get_particles", "mmp_fine_serial", "mmp_fine", "mmp_philox",
    "mmp_normals", "mmp_get_plan", "mmp_set_timing", "mmp_timing", "mmp_fine_static",
    "mmp_set_params", "mmp_adjoint_workspace_size", "mmp_adjoint_forward", "mmp_adjoint_backward", "mmp_adjoint",
    "mmp_batch_info", "mmp_autotune_workspace_size", "mmp_autotune", "mmp_set_tuning", "mmp_set_batch_nq",
    "mmp_state_size", "mmp_get_state", "mmp_set_state", "mmp_probe_wait",
    "mmp_sweep_fine", "mmp_sweep_coarse", "mmp_get_records", "mmp_set_records", "mmp_get_output", "mmp_set_output",
    "mmp_sweep_info", "mmp_probe_fma", "mmp_probe_step",
]


class MMPError(RuntimeError):
    """A negative MMP_* return code (.code) with the call that returned it."""
    def __init__(self, code: int, where: str):
        name = ERRORS.get(code, str(code))
        msg = _lib.mmp_strerror(code).decode() if _lib is not None else name
        extra = ""
        if code == -4 and _lib is not None:
            extra = f" (cuda error {_lib.mmp_last_cuda_error()})"
        super().__init__(f"{where}: {name}: {msg}{extra}")
        self.code = code


class ProblemDesc(C.Structure):
    """ctypes mirror of mmp_problem_desc (field order and types as in include/mmp.h)."""
    _fields_ = [
        ("c3", C.c_double), ("c1", C.c_double), ("kappa", C.c_double), ("c0", C.c_double),
        ("B", C.c_double), ("BE", C.c_double), ("B0", C.c_double),
        ("m0", C.c_double), ("s0", C.c_double),
        ("T", C.c_double), ("N", C.c_int), ("dt", C.c_double), ("P", C.c_longlong),
        ("coarse_h", C.c_double), ("n_regions", C.c_int), ("threshold", C.c_double),
        ("variant", C.c_int), ("precision", C.c_int), ("seed", C.c_ulonglong),
        ("problem_tag", C.c_uint), ("tol", C.c_double), ("max_iter", C.c_int), ("coarse_model", C.c_int),
        ("threshold2", C.c_double), ("threshold3", C.c_double),
        ("family", C.c_int), ("K", C.c_double), ("g", C.c_double),
    ]


_lib = None


def load():
    """Load libmmp.so (building nothing); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libmmp.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.POINTER(C.c_double)
    pd = C.POINTER(ProblemDesc)
    sig = {
        "mmp_strerror": ([i], C.c_char_p),
        "mmp_version": ([], i),
        "mmp_last_cuda_error": ([], i),
        "mmp_workspace_size": ([pd, i, C.POINTER(C.c_size_t)], i),
        "mmp_create": ([C.POINTER(vp), pd, i, vp, C.c_size_t, vp], i),
        "mmp_destroy": ([vp], i),
        "mmp_set_initial": ([vp, i, vp, i], i),
        "mmp_lift": ([vp], i),
        "mmp_iterate": ([vp, i, C.POINTER(i)], i),
        "mmp_run": ([vp, C.POINTER(i)], i),
        "mmp_status": ([vp, i, C.POINTER(i), C.POINTER(i), d, C.POINTER(i)], i),
        "mmp_get_moments": ([vp, i, d], i),
        "mmp_get_particles": ([vp, i, i, vp, i], i),
        "mmp_fine_serial": ([vp, i, i, d, vp], i),
        "mmp_fine": ([vp, i, i, vp, vp, d], i),
        "mmp_philox": ([vp, C.POINTER(C.c_uint), vp, ll, vp], i),
        "mmp_normals": ([pd, i, C.c_uint, C.c_uint, ll, vp, vp], i),
        "mmp_get_plan": ([vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i)], i),
        "mmp_set_timing": ([vp, i], i),
        "mmp_timing": ([vp, i, d, C.POINTER(ll), d, C.POINTER(ll)], i),
        "mmp_fine_static": ([pd, i, vp, vp, vp, vp], i),
        "mmp_set_params": ([vp, i, d, i], i),
        "mmp_adjoint_workspace_size": ([vp, i, i, C.POINTER(C.c_size_t)], i),
        "mmp_adjoint_forward": ([vp, i, i, vp, C.c_size_t, d], i),
        "mmp_adjoint_backward": ([vp, i, d, d, vp, C.c_size_t, d], i),
        "mmp_adjoint": ([vp, i, d, d, i, vp, C.c_size_t, d, d], i),
        "mmp_batch_info": ([vp, C.POINTER(i), C.POINTER(i)], i),
        "mmp_autotune_workspace_size": ([pd, C.POINTER(C.c_size_t)], i),
        "mmp_autotune": ([pd, C.POINTER(i), i, i, vp, C.c_size_t, vp, C.POINTER(i), d], i),
        "mmp_set_tuning": ([i, ll, ll, i], i),
        "mmp_set_batch_nq": ([i, i], i),
        "mmp_state_size": ([vp, C.POINTER(C.c_size_t)], i),
        "mmp_get_state": ([vp, vp], i),
        "mmp_set_state": ([vp, vp], i),
        "mmp_probe_wait": ([i, i, C.c_double, vp, C.c_size_t, vp, C.POINTER(C.c_uint)], i),
        "mmp_sweep_fine": ([vp, i, i, i], i),
        "mmp_sweep_coarse": ([vp, i, C.POINTER(i)], i),
        "mmp_get_records": ([vp, i, i, i, d], i),
        "mmp_set_records": ([vp, i, i, i, d], i),
        "mmp_get_output": ([vp, i, i, vp, i], i),
        "mmp_set_output": ([vp, i, i, vp, i], i),
        "mmp_sweep_info": ([vp, i, d], i),
        "mmp_probe_fma": ([i, vp, C.c_size_t, vp, d], i),
        "mmp_probe_step": ([i, vp, C.c_size_t, vp, d], i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != MMP_OK:
        raise MMPError(rc, where)


def desc(p: workloads.Problem) -> ProblemDesc:
    """The C descriptor of a problem record; refuses the terms the kernels do not run."""
    if p.q2 != 0.0:
        # the library's kernels do not carry the second-moment coupling
        raise MMPError(-3, "desc")
    prec = MMP_MIXED if p.precision == "mixed" else MMP_FP64
    return ProblemDesc(p.c3, p.c1, p.kappa, p.c0, p.B, p.BE, p.B0, p.m0, p.s0, p.T, p.N, p.dt, p.P,
                       p.coarse_h, p.n_regions, p.threshold, p.variant, prec, p.seed, p.problem_tag,
                       p.tol, p.max_iter, p.coarse_model, p.threshold2, p.threshold3, p.family, p.K, p.g)


def _descs(problems) -> C.Array:
    arr = (ProblemDesc * len(problems))()
    for k, p in enumerate(problems):
        arr[k] = desc(p)
    return arr


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return int(getattr(stream, "cuda_stream", stream))


# ---- one Python function per C entry point --------------------------------

def mmp_strerror(code: int) -> str:
    """Name of a return code."""
    return load().mmp_strerror(code).decode()


def mmp_version() -> int:
    """C-ABI version of the loaded library (MMP_VERSION)."""
    return load().mmp_version()


def mmp_workspace_size(problems) -> int:
    """Bytes of device workspace a context over these problems needs."""
    arr = _descs(problems)
    n = C.c_size_t()
    _check(load().mmp_workspace_size(arr, len(problems), C.byref(n)), "mmp_workspace_size")
    return n.value


def mmp_create(problems, workspace_ptr: int, workspace_bytes: int, stream=None) -> C.c_void_p:
    """A context over caller-owned device workspace (256-byte aligned); draws the initial ensembles."""
    arr = _descs(problems)
    ctx = C.c_void_p()
    _check(load().mmp_create(C.byref(ctx), arr, len(problems), C.c_void_p(workspace_ptr), workspace_bytes,
                             C.c_void_p(_stream_handle(stream))), "mmp_create")
    return ctx


def mmp_destroy(ctx) -> None:
    """Frees the context (a host object); the workspace stays the caller's."""
    _check(load().mmp_destroy(ctx), "mmp_destroy")


def mmp_set_initial(ctx, prob: int, u0_ptr: int, from_host: bool) -> None:
    """Replaces problem prob's initial ensemble by P values at u0_ptr (host or device)."""
    _check(load().mmp_set_initial(ctx, prob, C.c_void_p(u0_ptr), int(from_host)), "mmp_set_initial")


def mmp_lift(ctx) -> None:
    """Iteration k = 0: restriction of u0, sequential coarse sweep, lifting records."""
    _check(load().mmp_lift(ctx), "mmp_lift")


def mmp_iterate(ctx, n_iter: int) -> bool:
    """Up to n_iter fine + coarse sweeps (Eq. mM_parareal_other_k_NEW); True when every problem stopped."""
    done = C.c_int()
    _check(load().mmp_iterate(ctx, n_iter, C.byref(done)), "mmp_iterate")
    return bool(done.value)


def mmp_run(ctx) -> int:
    """Lift, then sweep until every problem stops; returns the largest sweep count."""
    k = C.c_int()
    _check(load().mmp_run(ctx, C.byref(k)), "mmp_run")
    return k.value


def mmp_status(ctx, prob: int) -> dict:
    """Sweeps done, converged, last change and device error code of problem prob."""
    s, c, e = C.c_int(), C.c_int(), C.c_int()
    ch = C.c_double()
    _check(load().mmp_status(ctx, prob, C.byref(s), C.byref(c), C.byref(ch), C.byref(e)), "mmp_status")
    return {"sweeps": s.value, "converged": bool(c.value), "last_change": ch.value, "dev_err": e.value}


def mmp_get_moments(ctx, prob: int, N: int) -> np.ndarray:
    """Macro states rho_n, n = 0..N, as an [(N+1), MOMENT_STRIDE] array."""
    out = np.empty((N + 1) * MOMENT_STRIDE, np.float64)
    _check(load().mmp_get_moments(ctx, prob, out.ctypes.data_as(C.POINTER(C.c_double))), "mmp_get_moments")
    return out.reshape(N + 1, MOMENT_STRIDE)


def mmp_get_particles(ctx, prob: int, n: int, dst_ptr: int, to_host: bool) -> None:
    """Slice-end particles u_n (n = 0..N) of problem prob, copied to dst_ptr."""
    _check(load().mmp_get_particles(ctx, prob, n, C.c_void_p(dst_ptr), int(to_host)), "mmp_get_particles")


def mmp_fine_serial(ctx, prob: int, n_end: int, parts_ptr: int | None = None) -> np.ndarray:
    """Restriction records of the serial fine run u_0..u_{n_end} ([(n_end+1), STAT_STRIDE])."""
    out = np.empty((n_end + 1) * STAT_STRIDE, np.float64)
    _check(load().mmp_fine_serial(ctx, prob, n_end, out.ctypes.data_as(C.POINTER(C.c_double)),
                                  C.c_void_p(parts_ptr or 0)), "mmp_fine_serial")
    return out.reshape(n_end + 1, STAT_STRIDE)


def mmp_fine(ctx, prob: int, n: int, u_in_ptr: int, u_out_ptr: int) -> np.ndarray:
    """One fine propagation F_n of the ensemble at u_in_ptr into u_out_ptr; its restriction record."""
    out = np.empty(STAT_STRIDE, np.float64)
    _check(load().mmp_fine(ctx, prob, n, C.c_void_p(u_in_ptr), C.c_void_p(u_out_ptr),
                           out.ctypes.data_as(C.POINTER(C.c_double))), "mmp_fine")
    return out


def mmp_get_plan(ctx, prob: int) -> dict:
    """Launch shape of problem prob's fine kernel (quads per thread, CTAs per slice, ...)."""
    a, b, c, e = C.c_int(), C.c_int(), C.c_int(), C.c_int()
    _check(load().mmp_get_plan(ctx, prob, C.byref(a), C.byref(b), C.byref(c), C.byref(e)), "mmp_get_plan")
    return {"quads_per_thread": a.value, "ctas_per_slice": b.value, "max_concurrent_slices": c.value,
            "particles_in_shared": bool(e.value)}


def mmp_set_timing(ctx, on: bool) -> None:
    """Switches CUDA-event timing of every fine launch on or off."""
    _check(load().mmp_set_timing(ctx, int(on)), "mmp_set_timing")


def mmp_timing(ctx, reset: bool = False) -> dict:
    """Fine-kernel milliseconds, launches and particle-steps, other launches (since the last reset)."""
    ms, steps = C.c_double(), C.c_double()
    fl, ol = C.c_longlong(), C.c_longlong()
    _check(load().mmp_timing(ctx, int(reset), C.byref(ms), C.byref(fl), C.byref(steps), C.byref(ol)),
           "mmp_timing")
    return {"fine_ms": ms.value, "fine_launches": fl.value, "fine_particle_steps": steps.value,
            "other_launches": ol.value}


def mmp_batch_info(ctx) -> dict:
    """Whether the context batches its problems and replays its sweeps from a CUDA graph."""
    b, g = C.c_int(), C.c_int()
    _check(load().mmp_batch_info(ctx, C.byref(b), C.byref(g)), "mmp_batch_info")
    return {"batched": bool(b.value), "graph": bool(g.value)}


def mmp_autotune(p: workloads.Problem, candidates=None, probe_steps: int = 0, stream=None) -> dict:
    """Time one fine launch per candidate quads-per-thread count (see the
    C header); returns the fastest count and the rate of each candidate."""
    import torch

    dsc = desc(p)
    nb = C.c_size_t()
    _check(load().mmp_autotune_workspace_size(C.byref(dsc), C.byref(nb)), "mmp_autotune_workspace_size")
    ws = torch.empty(max(1, nb.value), dtype=torch.uint8, device="cuda")
    prec = dsc.precision
    cands = list(candidates) if candidates is not None else list(range(1, (32 if prec == MMP_MIXED else 16) + 1))
    carr = (C.c_int * len(cands))(*cands)
    rates = np.zeros(len(cands))
    best = C.c_int()
    _check(load().mmp_autotune(C.byref(dsc), carr, len(cands), int(probe_steps), C.c_void_p(ws.data_ptr()),
                               nb.value, C.c_void_p(_stream_handle(stream)), C.byref(best),
                               rates.ctypes.data_as(C.POINTER(C.c_double))), "mmp_autotune")
    del ws
    return {"best_nq": best.value, "rates": dict(zip(cands, rates.tolist()))}


def mmp_set_tuning(precision: str, p_lo: int, p_hi: int, quads_per_thread: int) -> None:
    """Registers quads per thread for problems of a precision with p_lo <= P <= p_hi."""
    prec = MMP_MIXED if precision == "mixed" else MMP_FP64
    _check(load().mmp_set_tuning(prec, int(p_lo), int(p_hi), int(quads_per_thread)), "mmp_set_tuning")


def mmp_set_batch_nq(precision: str, quads_per_thread: int) -> None:
    """Cap on quads per thread of batched contexts of a precision created afterwards."""
    prec = MMP_MIXED if precision == "mixed" else MMP_FP64
    _check(load().mmp_set_batch_nq(prec, int(quads_per_thread)), "mmp_set_batch_nq")


def mmp_get_state(ctx) -> bytes:
    """The context's checkpoint (see the C header) as bytes."""
    n = C.c_size_t()
    _check(load().mmp_state_size(ctx, C.byref(n)), "mmp_state_size")
    buf = (C.c_char * n.value)()
    _check(load().mmp_get_state(ctx, buf), "mmp_get_state")
    return bytes(buf)


def mmp_set_state(ctx, blob: bytes) -> None:
    """Restores a checkpoint taken by mmp_get_state into a context over the same problems."""
    buf = C.create_string_buffer(blob, len(blob))
    _check(load().mmp_set_state(ctx, buf), "mmp_set_state")


def mmp_sweep_fine(ctx, prob: int, n_lo: int, n_hi: int) -> None:
    """Fine phase of the next sweep over slices [n_lo, n_hi) (asynchronous)."""
    _check(load().mmp_sweep_fine(ctx, prob, n_lo, n_hi), "mmp_sweep_fine")


def mmp_sweep_coarse(ctx, prob: int) -> bool:
    """Driver phase of the pending sweep over all slices; True when the problem stopped."""
    done = C.c_int()
    _check(load().mmp_sweep_coarse(ctx, prob, C.byref(done)), "mmp_sweep_coarse")
    return bool(done.value)


def mmp_get_records(ctx, prob: int, n_lo: int, n_hi: int) -> np.ndarray:
    """Restriction records of slices [n_lo, n_hi), [n_hi - n_lo, STAT_STRIDE]."""
    out = np.zeros((max(n_hi - n_lo, 0), STAT_STRIDE))
    _check(load().mmp_get_records(ctx, prob, n_lo, n_hi, out.ctypes.data_as(C.POINTER(C.c_double))),
           "mmp_get_records")
    return out


def mmp_set_records(ctx, prob: int, n_lo: int, n_hi: int, rows) -> None:
    """Write restriction records of slices [n_lo, n_hi)."""
    arr = np.ascontiguousarray(rows, dtype=np.float64)
    _check(load().mmp_set_records(ctx, prob, n_lo, n_hi, arr.ctypes.data_as(C.POINTER(C.c_double))),
           "mmp_set_records")


def mmp_get_output(ctx, prob: int, n: int, dst_ptr: int, to_host: bool) -> None:
    """Copy the latest fine output of slice n to dst."""
    _check(load().mmp_get_output(ctx, prob, n, dst_ptr, 1 if to_host else 0), "mmp_get_output")


def mmp_set_output(ctx, prob: int, n: int, src_ptr: int, from_host: bool) -> None:
    """Replace the latest fine output of slice n by src."""
    _check(load().mmp_set_output(ctx, prob, n, src_ptr, 1 if from_host else 0), "mmp_set_output")


def mmp_sweep_info(ctx, prob: int) -> dict:
    """Counters of the device-side iteration (acceptance, fit use, last change)."""
    out = np.zeros(6)
    _check(load().mmp_sweep_info(ctx, prob, out.ctypes.data_as(C.POINTER(C.c_double))), "mmp_sweep_info")
    return {"accepted": int(out[0]), "rejected": int(out[1]), "fit_used": bool(out[2]),
            "fit_alpha": float(out[3]), "fit_beta": float(out[4]), "change": float(out[5])}


def mmp_probe_fma(precision: str, stream=None) -> float:
    """FMA throughput of the device in TFLOP/s, FP64 ("fp64") or FP32 ("mixed")."""
    import torch

    sink = torch.empty(64, dtype=torch.uint8, device="cuda")
    tf = C.c_double()
    prec = MMP_MIXED if precision == "mixed" else MMP_FP64
    _check(load().mmp_probe_fma(prec, sink.data_ptr(), sink.numel(), _stream_handle(stream), C.byref(tf)),
           "mmp_probe_fma")
    return tf.value


def mmp_probe_step(form: int, stream=None) -> float:
    """Particle-steps/s of the fine step's arithmetic without the cross-CTA
    exchange: form 0 with the particles in registers, form 1 in shared
    memory with a CTA barrier every step (the fine kernel's layout)."""
    import torch

    sink = torch.empty(64, dtype=torch.uint8, device="cuda")
    r = C.c_double()
    _check(load().mmp_probe_step(int(form), sink.data_ptr(), sink.numel(), _stream_handle(stream), C.byref(r)),
           "mmp_probe_step")
    return r.value


def mmp_probe_wait(channel: int, G: int, limit_ms: float, ws_ptr: int, ws_bytes: int, stream=None):
    """Self-test of the bounded group wait: (return code, status word); the
    code is MMP_ERR_TIMEOUT (-6) when the wait ran out as it must for G >= 2."""
    st = C.c_uint()
    rc = load().mmp_probe_wait(channel, G, float(limit_ms), ws_ptr, ws_bytes, _stream_handle(stream), C.byref(st))
    return rc, st.value


def mmp_fine_static(p: workloads.Problem, n: int, u_in_ptr: int, u_out_ptr: int, stats_ptr: int | None,
                    stream=None) -> None:
    """One fine propagation with no device allocation (scratch from the
    library's static array); asynchronous on `stream`."""
    dsc = desc(p)
    _check(load().mmp_fine_static(C.byref(dsc), n, C.c_void_p(u_in_ptr), C.c_void_p(u_out_ptr),
                                  C.c_void_p(stats_ptr or 0), C.c_void_p(_stream_handle(stream))),
           "mmp_fine_static")


def mmp_set_params(ctx, prob: int, theta) -> None:
    """theta = (c3, c1, kappa, c0, B0) or (c3, c1, kappa, c0, B0, B, BE)."""
    t = np.ascontiguousarray(theta, dtype=np.float64).ravel()
    _check(load().mmp_set_params(ctx, prob, t.ctypes.data_as(C.POINTER(C.c_double)), t.size), "mmp_set_params")


def mmp_adjoint_workspace_size(ctx, prob: int, ckpt_every: int) -> int:
    """Bytes of adjoint workspace for a checkpoint every ckpt_every fine steps."""
    n = C.c_size_t()
    _check(load().mmp_adjoint_workspace_size(ctx, prob, ckpt_every, C.byref(n)), "mmp_adjoint_workspace_size")
    return n.value


def mmp_adjoint_forward(ctx, prob: int, ckpt_every: int, ws_ptr: int, ws_bytes: int, N: int) -> np.ndarray:
    """Recording serial fine run; slice-end (M_n, V_n), n = 0..N, as an [(N+1), 2] array."""
    mom = np.empty(2 * (N + 1), np.float64)
    _check(load().mmp_adjoint_forward(ctx, prob, ckpt_every, C.c_void_p(ws_ptr), ws_bytes,
                                      mom.ctypes.data_as(C.POINTER(C.c_double))), "mmp_adjoint_forward")
    return mom.reshape(N + 1, 2)


def mmp_adjoint_backward(ctx, prob: int, gm, gv, ws_ptr: int, ws_bytes: int) -> np.ndarray:
    """Gradient of sum gm M_n + gv V_n in (c3, c1, kappa, c0, B0, B, BE) after a forward run."""
    gma = np.ascontiguousarray(gm, dtype=np.float64)
    gva = np.ascontiguousarray(gv, dtype=np.float64)
    grad = np.empty(N_THETA, np.float64)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(load().mmp_adjoint_backward(ctx, prob, dp(gma), dp(gva), C.c_void_p(ws_ptr), ws_bytes, dp(grad)),
           "mmp_adjoint_backward")
    return grad


def mmp_adjoint(ctx, prob: int, m_tgt, v_tgt, ckpt_every: int, ws_ptr: int, ws_bytes: int):
    """Loss sum (M_n - m*)^2 + (V_n - v*)^2 of the serial fine run and its
    gradient in (c3, c1, kappa, c0, B0, B, BE), in one call."""
    mt = np.ascontiguousarray(m_tgt, dtype=np.float64)
    vt = np.ascontiguousarray(v_tgt, dtype=np.float64)
    grad = np.empty(N_THETA, np.float64)
    loss = C.c_double()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(load().mmp_adjoint(ctx, prob, dp(mt), dp(vt), ckpt_every, C.c_void_p(ws_ptr), ws_bytes, dp(grad),
                              C.byref(loss)), "mmp_adjoint")
    return loss.value, grad


def mmp_philox(ctr_ptr: int, key, out_ptr: int, n: int, stream=None) -> None:
    """Philox-4x32-10 of n counters at ctr_ptr under key into out_ptr (device, 16-byte aligned)."""
    k = (C.c_uint * 2)(int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF)
    _check(load().mmp_philox(C.c_void_p(ctr_ptr), k, C.c_void_p(out_ptr), n,
                             C.c_void_p(_stream_handle(stream))), "mmp_philox")


def mmp_normals(p: workloads.Problem, tag: int, j: int, n: int, count: int, out_ptr: int, stream=None) -> None:
    """The normals the fine propagator draws for (tag, step j, slice n), count of them, into out_ptr."""
    dsc = desc(p)
    _check(load().mmp_normals(C.byref(dsc), tag, j, n, count, C.c_void_p(out_ptr),
                              C.c_void_p(_stream_handle(stream))), "mmp_normals")


# ---- convenience wrapper ---------------------------------------------------

class Solver:
    """Owns a torch workspace and a context for a list of problems."""

    def __init__(self, problems, stream=None):
        import torch

        self.problems = list(problems) if isinstance(problems, (list, tuple)) else [problems]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        nbytes = mmp_workspace_size(self.problems)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
        self.ctx = mmp_create(self.problems, self.workspace.data_ptr(), nbytes, self.stream)

    def dtype(self, prob: int = 0):
        import torch
        return torch.float32 if self.problems[prob].precision == "mixed" else torch.float64

    def run(self) -> int:
        return mmp_run(self.ctx)

    def lift(self) -> None:
        mmp_lift(self.ctx)

    def iterate(self, n: int = 1) -> bool:
        return mmp_iterate(self.ctx, n)

    def moments(self, prob: int = 0) -> np.ndarray:
        return mmp_get_moments(self.ctx, prob, self.problems[prob].N)

    def plan(self, prob: int = 0) -> dict:
        return mmp_get_plan(self.ctx, prob)

    def status(self, prob: int = 0) -> dict:
        return mmp_status(self.ctx, prob)

    def particles(self, n: int, prob: int = 0):
        import torch
        out = torch.empty(self.problems[prob].P + 4, dtype=self.dtype(prob), device="cuda")
        mmp_get_particles(self.ctx, prob, n, out.data_ptr(), False)
        torch.cuda.current_stream().synchronize()
        return out[: self.problems[prob].P]

    def serial(self, prob: int = 0, n_end: int | None = None, want_last: bool = False):
        """Serial reference through slice end n_end (default N): restriction
        records of u_0..u_{n_end}, and u_{n_end} itself if want_last."""
        import torch
        n_end = self.problems[prob].N if n_end is None else n_end
        last = None
        if want_last:
            last = torch.empty(self.problems[prob].P + 4, dtype=self.dtype(prob), device="cuda")
        st = mmp_fine_serial(self.ctx, prob, n_end, last.data_ptr() if last is not None else None)
        return (st, last[: self.problems[prob].P]) if want_last else st

    def set_initial(self, u0, prob: int = 0) -> None:
        import torch
        if isinstance(u0, torch.Tensor) and u0.is_cuda:
            mmp_set_initial(self.ctx, prob, u0.data_ptr(), False)
        else:
            arr = np.ascontiguousarray(u0, dtype=np.float32 if self.problems[prob].precision == "mixed" else np.float64)
            mmp_set_initial(self.ctx, prob, arr.ctypes.data, True)

    def state(self) -> bytes:
        """Checkpoint of the run (workspace contents and iteration state)."""
        return mmp_get_state(self.ctx)

    def restore(self, blob: bytes) -> None:
        """Resume from a checkpoint of a Solver with the same problems."""
        mmp_set_state(self.ctx, blob)

    def close(self) -> None:
        if self.ctx is not None:
            mmp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run(problems, stream=None) -> list[dict]:
    """Solve one problem or a list of problems (batched in one context when
    they share a precision and kernel form) to convergence; per problem its
    status (sweeps, converged, last_change, dev_err) and its moments
    [(N+1), MOMENT_STRIDE] (per-region fraction, mean, variance; global
    mean and variance)."""
    s = Solver(problems, stream)
    try:
        s.run()
        return [dict(s.status(i), moments=s.moments(i)) for i in range(len(s.problems))]
    finally:
        s.close()


# ---- adjoint as a torch.autograd.Function -----------------------------------

THETA_NAMES = ("c3", "c1", "kappa", "c0", "B0", "B", "BE")


class Adjoint:
    """Caller-owned adjoint workspace for one problem of a Solver."""

    def __init__(self, solver: Solver, prob: int = 0, ckpt_every: int = 64):
        import torch

        self.solver, self.prob, self.ckpt_every = solver, prob, ckpt_every
        self.nbytes = mmp_adjoint_workspace_size(solver.ctx, prob, ckpt_every)
        self.ws = torch.empty(max(self.nbytes, 256), dtype=torch.uint8, device="cuda")

    def forward(self, theta) -> np.ndarray:
        mmp_set_params(self.solver.ctx, self.prob, theta)
        return mmp_adjoint_forward(self.solver.ctx, self.prob, self.ckpt_every, self.ws.data_ptr(), self.nbytes,
                                   self.solver.problems[self.prob].N)

    def backward(self, gm, gv) -> np.ndarray:
        return mmp_adjoint_backward(self.solver.ctx, self.prob, gm, gv, self.ws.data_ptr(), self.nbytes)

    def loss_and_grad(self, theta, m_tgt, v_tgt):
        """Loss against moment targets and its gradient at theta, one call."""
        mmp_set_params(self.solver.ctx, self.prob, theta)
        return mmp_adjoint(self.solver.ctx, self.prob, m_tgt, v_tgt, self.ckpt_every, self.ws.data_ptr(),
                           self.nbytes)


def _autograd_function():
    import torch

    class FineMoments(torch.autograd.Function):
        """theta = (c3, c1, kappa, c0, B0[, B, BE]) -> slice-end moments
        [(N+1), 2] (mean, population variance) of the serial fine run; the
        backward is the library's adjoint kernel (gradient in as many
        coefficients as theta holds)."""

        @staticmethod
        def forward(ctx, theta, adj):
            mom = adj.forward(theta.detach().cpu().double().numpy())
            ctx.adj = adj
            ctx.n_theta = theta.numel()
            ctx.dtype = theta.dtype
            return torch.from_numpy(mom).to(theta.dtype)

        @staticmethod
        def backward(ctx, g):
            g = g.detach().cpu().double().numpy()
            grad = ctx.adj.backward(g[1:, 0], g[1:, 1])
            return torch.from_numpy(grad[: ctx.n_theta]).to(ctx.dtype), None

    return FineMoments


_fine_moments_cls = None


def __getattr__(name: str):
    # mmp.FineMoments is built on first access, so that importing the
    # binding does not import torch
    global _fine_moments_cls
    if name == "FineMoments":
        if _fine_moments_cls is None:
            _fine_moments_cls = _autograd_function()
        return _fine_moments_cls
    raise AttributeError(name)


def fine_moments(theta, adj: Adjoint):
    """Differentiable slice-end moments of the serial fine run
    (FineMoments.apply(theta, adj))."""
    return __getattr__("FineMoments").apply(theta, adj)


def double_well_theta(kappa, sigma, a, b):
    """theta of dX = (-V'(X) + kappa (E[X] - X)) dt + sigma dW, V = a x^4 - b x^2,
    built with torch operations so that gradients flow to (kappa, sigma, a, b)."""
    import torch

    zero = torch.zeros((), dtype=torch.float64)
    return torch.stack([4 * a, 2 * b - kappa, kappa, zero, sigma])
