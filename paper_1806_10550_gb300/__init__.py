"""GB300 Newton--ADI thin-film solver: Python binding of ``libtfadi.so``.

Argument marshalling only: every step of the time integration runs in the
CUDA kernels of ``csrc/`` behind the C ABI of ``include/tf.h``.  Grids are
``torch.float64`` CUDA tensors of shape ``(ny, nx)`` (row-major, x
contiguous); PyTorch supplies device memory and the stream.  There is no
CPU fallback: without the built library or a CUDA device every call raises.

Functions carry the names of the C ABI: ``tf_params_default``, ``tf_init``,
``tf_destroy``, ``tf_residual``, ``tf_newton_iteration``,
``tf_newton_adi_step``, ``tf_advance``, ``tf_ensemble_advance``, ``tf_strerror``,
``tf_adjoint_step`` (the reverse of the fixed-iteration step), the tape of a
checkpointed trajectory ``tf_tape_create``, ``tf_tape_forward``,
``tf_tape_backward``, ``tf_tape_info``, ``tf_tape_timing``,
``tf_tape_destroy``, and for the
radial Fourier analysis ``tf_spectrum_params_default``,
``tf_spectrum_plan_create``, ``tf_spectrum_run``, ``tf_spectrum_plan_info``,
``tf_spectrum_timing``, ``tf_spectrum_plan_destroy``.
"""
from __future__ import annotations

import ctypes as C
import os

from ._build import LIB as _LIB_PATH
from ._build import build as _build_lib

TF_OK = 0
TF_ERR_ARG = -1
TF_ERR_CUDA = -2
TF_ERR_NOMEM = -3
TF_STEP_CONVERGED = 0
TF_STEP_NOT_CONVERGED = 1
TF_STEP_NONPOSITIVE = 2
TF_STEP_ZERO_PIVOT = 3
TF_ADV_DONE = 0
TF_ADV_MAX_ATTEMPTS = 1
TF_ADV_DT_MIN = 2
TF_ADV_RUPTURE = 3
TF_MODEL_POWERLAW = 0
TF_MODEL_LINEAR = 1
TF_MODEL_NLC = 2
TF_MODEL_POLYMER = 3
TF_FP64 = 0
TF_FP32_BULK = 1
TF_SOLVER_TWISTED = 0
TF_SOLVER_PARTITIONED = 1
TF_SOLVER_AUTO = 2


class TfParams(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("ds", C.c_double), ("model", C.c_int),
        ("cap_C", C.c_double), ("b", C.c_double), ("n", C.c_int), ("m", C.c_int),
        ("kappa", C.c_double), ("contact_angle", C.c_double), ("c0", C.c_double),
        ("c1", C.c_double), ("theta", C.c_double), ("newton_tol", C.c_double),
        ("newton_max_iter", C.c_int), ("newton_fixed_iter", C.c_int),
        ("dt_min", C.c_double), ("dt_max", C.c_double), ("dt_shrink", C.c_double),
        ("dt_grow", C.c_double), ("grow_after", C.c_int), ("rupture_h", C.c_double),
        ("precision", C.c_int),
        ("nlc_K", C.c_double), ("nlc_N", C.c_double), ("nlc_beta", C.c_double),
        ("nlc_w", C.c_double),
        ("pol_C", C.c_double), ("pol_A_SiOx", C.c_double), ("pol_A_Si", C.c_double),
        ("pol_d", C.c_double), ("line_solver", C.c_int),
    ]


class TfNorms(C.Structure):
    _fields_ = [("gnorm", C.c_double), ("mass", C.c_double), ("hmin", C.c_double)]


class TfStepInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("iterations", C.c_int), ("err", C.c_double),
                ("gnorm", C.c_double), ("mass", C.c_double), ("hmin", C.c_double)]


class TfStepRecord(C.Structure):
    _fields_ = [("t", C.c_double), ("dt", C.c_double), ("accepted", C.c_int),
                ("iterations", C.c_int), ("status", C.c_int), ("err", C.c_double),
                ("gnorm", C.c_double), ("mass", C.c_double), ("hmin", C.c_double)]


class TfAdvanceInfo(C.Structure):
    _fields_ = [("status", C.c_int), ("attempts", C.c_int), ("accepted", C.c_int),
                ("newton_iterations", C.c_int), ("t", C.c_double), ("dt", C.c_double)]


class TfTiming(C.Structure):
    _fields_ = [("enabled", C.c_int), ("launches", C.c_int), ("explicit_launches", C.c_int),
                ("rhs_launches", C.c_int), ("x_launches", C.c_int), ("y_launches", C.c_int),
                ("explicit_ms", C.c_double), ("rhs_ms", C.c_double), ("x_ms", C.c_double),
                ("y_ms", C.c_double)]


_lib = None


class TfSpectrumParams(C.Structure):
    _fields_ = [("H0", C.c_double), ("q_cut", C.c_double), ("sigma", C.c_double),
                ("points_per_interval", C.c_int), ("n_eval", C.c_int)]


class TfSpectrumInfo(C.Structure):
    _fields_ = [("n_p", C.c_int), ("n_q", C.c_int), ("n_radii", C.c_int), ("n_intervals", C.c_int),
                ("n_eval", C.c_int), ("n_peaks", C.c_int), ("q_dominant", C.c_double),
                ("value_dominant", C.c_double)]


class TfSpectrumOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in (
        "amplitude", "smoothed", "radial_q", "radial_value", "node_q", "node_value",
        "curve_q", "curve_value", "peak_q", "peak_value")] + [("peak_cap", C.c_int)]


def library(build_if_missing: bool = True):
    """Load ``libtfadi.so`` (building it with nvcc when it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {_LIB_PATH}")
        _build_lib()
    L = C.CDLL(_LIB_PATH)
    vp, dp = C.c_void_p, C.c_double
    L.tf_params_default.argtypes = [C.POINTER(TfParams)]
    L.tf_params_default.restype = None
    L.tf_init.argtypes = [C.POINTER(TfParams), vp, C.POINTER(vp)]
    L.tf_destroy.argtypes = [vp]
    L.tf_destroy.restype = None
    L.tf_strerror.argtypes = [C.c_int]
    L.tf_strerror.restype = C.c_char_p
    L.tf_kappa.argtypes = [vp]
    L.tf_kappa.restype = dp
    L.tf_residual.argtypes = [vp, vp, vp, dp, vp, C.POINTER(TfNorms)]
    L.tf_newton_iteration.argtypes = [vp, vp, vp, dp, vp, vp, vp, C.POINTER(TfStepInfo)]
    L.tf_newton_adi_step.argtypes = [vp, vp, vp, dp, C.POINTER(TfStepInfo)]
    L.tf_advance.argtypes = [vp, vp, dp, dp, dp, C.c_int, vp, vp, C.POINTER(TfStepRecord),
                             C.POINTER(TfAdvanceInfo), C.POINTER(C.c_int)]
    L.tf_ensemble_advance.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(dp),
                                      C.POINTER(dp), C.POINTER(dp), C.POINTER(C.c_int),
                                      C.POINTER(TfAdvanceInfo), C.POINTER(C.c_int), C.c_int]
    L.tf_tune_line_solver.argtypes = [C.POINTER(TfParams), vp, vp, dp, C.c_int, C.c_int,
                                      C.POINTER(C.c_int), C.POINTER(dp)]
    L.tf_tuned_line_solver.argtypes = [C.POINTER(TfParams)]
    L.tf_tuned_line_solver.restype = C.c_int
    L.tf_line_solver.argtypes = [vp]
    L.tf_line_solver.restype = C.c_int
    L.tf_probe_fma.argtypes = [C.c_int, vp, C.POINTER(dp)]
    L.tf_timing_enable.argtypes = [vp, C.c_int]
    L.tf_timing_get.argtypes = [vp, C.POINTER(TfTiming)]
    L.tf_adjoint_step.argtypes = [vp, vp, dp, C.c_int, vp, vp, vp, C.POINTER(dp), C.POINTER(dp)]
    L.tf_adjoint_timing.argtypes = [C.POINTER(dp), C.c_int]
    L.tf_tape_create.argtypes = [vp, C.c_int, C.c_int, dp, C.c_int, C.POINTER(vp)]
    L.tf_tape_destroy.argtypes = [vp]
    L.tf_tape_destroy.restype = None
    L.tf_tape_info.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_size_t),
                               C.POINTER(C.c_int)]
    L.tf_tape_forward.argtypes = [vp, vp, vp]
    L.tf_tape_backward.argtypes = [vp, vp, vp, C.POINTER(dp), C.POINTER(dp)]
    L.tf_tape_timing.argtypes = [vp, C.POINTER(dp), C.c_int]
    L.tf_spectrum_params_default.argtypes = [C.POINTER(TfSpectrumParams)]
    L.tf_spectrum_params_default.restype = None
    L.tf_spectrum_plan_create.argtypes = [C.c_int, C.c_int, dp, C.POINTER(TfSpectrumParams), vp,
                                          C.POINTER(vp)]
    L.tf_spectrum_plan_destroy.argtypes = [vp]
    L.tf_spectrum_plan_destroy.restype = None
    L.tf_spectrum_plan_info.argtypes = [vp, C.POINTER(TfSpectrumInfo)]
    L.tf_spectrum_run.argtypes = [vp, vp, C.POINTER(TfSpectrumOut), C.POINTER(TfSpectrumInfo)]
    L.tf_spectrum_timing.argtypes = [vp, C.POINTER(dp), C.c_int]
    for f in ("tf_init", "tf_residual", "tf_newton_iteration", "tf_newton_adi_step", "tf_advance",
              "tf_ensemble_advance", "tf_timing_enable", "tf_timing_get", "tf_adjoint_step",
              "tf_adjoint_timing", "tf_tape_create", "tf_tape_info", "tf_tape_forward",
              "tf_tape_backward", "tf_tape_timing",
              "tf_spectrum_plan_create",
              "tf_spectrum_plan_info", "tf_spectrum_run", "tf_spectrum_timing", "tf_tune_line_solver", "tf_probe_fma"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def tf_strerror(code: int) -> str:
    return library().tf_strerror(code).decode()


def _check(code: int, what: str):
    if code < 0:
        raise RuntimeError(f"{what}: {tf_strerror(code)} ({code})")
    return code


def tf_params_default(**overrides) -> TfParams:
    p = TfParams()
    library().tf_params_default(C.byref(p))
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError(k)
        setattr(p, k, v)
    return p


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("a CUDA device is required: this library has no CPU path")
    return torch


class Context:
    """Owns one ``tf_ctx`` (workspace on the device, bound to a stream)."""

    def __init__(self, params: TfParams, stream=None):
        torch = _torch()
        self.params = params
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(library().tf_init(C.byref(params), C.c_void_p(stream.cuda_stream), C.byref(h)),
               "tf_init")
        self.handle = h
        self.shape = (params.ny, params.nx)

    @property
    def kappa(self) -> float:
        return library().tf_kappa(self.handle)

    @property
    def line_solver(self) -> int:
        """The line solver this context uses (TF_SOLVER_TWISTED or _PARTITIONED)."""
        return library().tf_line_solver(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            library().tf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ptr(self, t, name, writable=False):
        """Device pointer of a float64 CUDA grid of this context's shape."""
        torch = _torch()
        if t is None:
            return None
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError(f"{name} must be a torch.float64 CUDA tensor")
        if tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {self.shape}")
        return C.c_void_p(t.data_ptr())


def tf_init(params: TfParams, stream=None) -> Context:
    return Context(params, stream)


def tf_destroy(ctx: Context):
    ctx.close()


def tf_residual(ctx: Context, h_k, h_old, dt: float, G=None) -> dict:
    n = TfNorms()
    _check(library().tf_residual(ctx.handle, ctx.ptr(h_k, "h_k"), ctx.ptr(h_old, "h_old"),
                                 float(dt), ctx.ptr(G, "G"), C.byref(n)), "tf_residual")
    return dict(gnorm=n.gnorm, mass=n.mass, hmin=n.hmin)


def _info(i: TfStepInfo) -> dict:
    return dict(status=i.status, iterations=i.iterations, err=i.err, gnorm=i.gnorm,
                mass=i.mass, hmin=i.hmin)


def tf_newton_iteration(ctx: Context, h_k, h_old, dt: float, h_next, w=None, v=None) -> dict:
    i = TfStepInfo()
    _check(library().tf_newton_iteration(ctx.handle, ctx.ptr(h_k, "h_k"), ctx.ptr(h_old, "h_old"),
                                         float(dt), ctx.ptr(w, "w"), ctx.ptr(v, "v"),
                                         ctx.ptr(h_next, "h_next"), C.byref(i)),
           "tf_newton_iteration")
    return _info(i)


def tf_newton_adi_step(ctx: Context, h_old, h_new, dt: float) -> dict:
    i = TfStepInfo()
    _check(library().tf_newton_adi_step(ctx.handle, ctx.ptr(h_old, "h_old"),
                                        ctx.ptr(h_new, "h_new"), float(dt), C.byref(i)),
           "tf_newton_adi_step")
    return _info(i)


def tf_advance(ctx: Context, h, t0: float, t_end: float, dt0: float, max_attempts: int,
               dt_replay=None, iter_replay=None, records: bool = True, streak: int = 0):
    """Advance ``h`` in place; returns (info dict, list of per-attempt records).

    ``streak`` is the controller's count of consecutive accepted steps at the
    start; the info dict's ``streak`` is its value at the end, so passing a
    call's ``t``, ``dt`` and ``streak`` to the next continues the same run."""
    import numpy as np
    recs = (TfStepRecord * max(1, max_attempts))() if records else None
    dtr = itr = None
    if dt_replay is not None:
        dtr_a = np.ascontiguousarray(dt_replay, dtype=np.float64)
        if dtr_a.shape[0] < max_attempts:
            raise ValueError("dt_replay shorter than max_attempts")
        dtr = C.c_void_p(dtr_a.ctypes.data)
    if iter_replay is not None:
        itr_a = np.ascontiguousarray(iter_replay, dtype=np.int32)
        if itr_a.shape[0] < max_attempts:
            raise ValueError("iter_replay shorter than max_attempts")
        itr = C.c_void_p(itr_a.ctypes.data)
    info = TfAdvanceInfo()
    st = C.c_int(int(streak))
    _check(library().tf_advance(ctx.handle, ctx.ptr(h, "h"), float(t0), float(t_end), float(dt0),
                                int(max_attempts), dtr, itr, recs, C.byref(info), C.byref(st)),
           "tf_advance")
    out = []
    if records:
        for r in recs[: info.attempts]:
            out.append(dict(t=r.t, dt=r.dt, accepted=bool(r.accepted), iterations=r.iterations,
                            status=r.status, err=r.err, gnorm=r.gnorm, mass=r.mass, hmin=r.hmin))
    return dict(status=info.status, attempts=info.attempts, accepted=info.accepted,
                newton_iterations=info.newton_iterations, t=info.t, dt=info.dt,
                streak=st.value), out


def tf_tune_line_solver(params: TfParams, h, dt: float, iters: int = 3, copies: int = 1,
                        stream=None) -> dict:
    """Time the line solvers that apply to ``params`` on ``copies`` films
    iterating at once from the CUDA film ``h`` and keep the faster for
    contexts created with ``TF_SOLVER_AUTO``; returns dict(best=solver,
    ms=[twisted, partitioned]) (ms per film iteration, -1 where a solver
    does not apply)."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    if tuple(h.shape) != (params.ny, params.nx) or h.dtype != torch.float64 or not h.is_cuda:
        raise ValueError("h must be a CUDA float64 tensor of the params' shape")
    best = C.c_int()
    ms = (C.c_double * 2)()
    _check(library().tf_tune_line_solver(C.byref(params), C.c_void_p(stream.cuda_stream),
                                         C.c_void_p(h.contiguous().data_ptr()), float(dt), int(iters),
                                         int(copies), C.byref(best), ms), "tf_tune_line_solver")
    return dict(best=best.value, ms=[ms[0], ms[1]])


def tf_probe_fma(precision: int, stream=None) -> float:
    """Measured FMA throughput of the current GPU in TFLOP/s (2 flops per
    FMA), FP64 (TF_FP64) or FP32 (TF_FP32_BULK)."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    out = C.c_double()
    _check(library().tf_probe_fma(int(precision), C.c_void_p(stream.cuda_stream), C.byref(out)),
           "tf_probe_fma")
    return out.value


def tf_tuned_line_solver(params: TfParams) -> int:
    """The tuned solver for ``params``' key, or -1."""
    return library().tf_tuned_line_solver(C.byref(params))


TF_ENSEMBLE_AUTO = 0
TF_ENSEMBLE_HOST = 1


def tf_ensemble_advance(ctxs, hs, t0, t_end, dt0, max_attempts, streak=0, engine=TF_ENSEMBLE_AUTO):
    """Advance independent films together (``tf_advance`` on each, their
    work interleaved on the contexts' streams).  ``ctxs``: contexts, one per
    film, each best on its own stream; ``hs``: their grids (advanced in
    place); ``t0``, ``t_end``, ``dt0``, ``max_attempts``, ``streak``: one
    value or one per film; ``engine``: TF_ENSEMBLE_AUTO (each film's run as
    one CUDA graph with its controller on the device, where the context
    allows it) or TF_ENSEMBLE_HOST.  Returns one info dict per film (with its
    ``streak`` at the end)."""
    n = len(ctxs)
    if len(hs) != n:
        raise ValueError("one grid per context")

    def arr(v, ctype):
        vals = list(v) if hasattr(v, "__len__") else [v] * n
        if len(vals) != n:
            raise ValueError("one value per film")
        return (ctype * max(1, n))(*vals)

    ctx_a = (C.c_void_p * max(1, n))(*[c.handle.value for c in ctxs])
    h_a = (C.c_void_p * max(1, n))(*[c.ptr(h, "h").value for c, h in zip(ctxs, hs)])
    infos = (TfAdvanceInfo * max(1, n))()
    st = arr(streak, C.c_int)
    _check(library().tf_ensemble_advance(n, ctx_a, h_a, arr(t0, C.c_double), arr(t_end, C.c_double),
                                         arr(dt0, C.c_double), arr(max_attempts, C.c_int), infos, st,
                                         int(engine)),
           "tf_ensemble_advance")
    return [dict(status=i.status, attempts=i.attempts, accepted=i.accepted,
                 newton_iterations=i.newton_iterations, t=i.t, dt=i.dt, streak=st[k])
            for k, i in enumerate(infos[:n])]


def tf_adjoint_step(ctx: Context, h_old, dt: float, K: int, g, g_h=None, h_new=None) -> dict:
    """Reverse of the K-iteration time step from ``h_old``: returns dict with
    ``g_h`` (the cotangent of h_old, a CUDA tensor), ``g_kappa``, ``g_theta``
    and ``h_new`` (u^K) when given or requested."""
    torch = _torch()
    if g_h is None:
        g_h = torch.empty_like(g)
    gk, gt = C.c_double(), C.c_double()
    _check(library().tf_adjoint_step(ctx.handle, ctx.ptr(h_old, "h_old"), float(dt), int(K),
                                     ctx.ptr(g, "g"), ctx.ptr(h_new, "h_new"), ctx.ptr(g_h, "g_h"),
                                     C.byref(gk), C.byref(gt)), "tf_adjoint_step")
    return dict(g_h=g_h, g_kappa=gk.value, g_theta=gt.value, h_new=h_new)


def unrolled_step(h, ctx: Context, dt: float, K: int):
    """u^K of the time step with exactly K Newton iterations from ``h``, as a
    differentiable torch operation: the forward runs K tf_newton_iteration
    calls, the backward tf_adjoint_step (which recomputes the forward, so
    only h is kept between the two).  ``ctx``: an FP64 context."""
    torch = _torch()

    class _UnrolledStep(torch.autograd.Function):
        @staticmethod
        def forward(actx, x):
            u = x.detach().contiguous()
            cur = u
            w, v = torch.empty_like(u), torch.empty_like(u)
            for _ in range(int(K)):
                nxt = torch.empty_like(u)
                tf_newton_iteration(ctx, cur, u, dt, nxt, w=w, v=v)
                cur = nxt
            actx.save_for_backward(u)
            return cur

        @staticmethod
        def backward(actx, g):
            (u,) = actx.saved_tensors
            return tf_adjoint_step(ctx, u, dt, int(K), g.contiguous())["g_h"]

    return _UnrolledStep.apply(h)


ADJOINT_GROUPS = ("forward", "band", "solve_t", "line_x", "line_y", "D", "kappa")


def tf_adjoint_timing() -> dict:
    """Kernel time (ms) of the last tf_adjoint_step by group."""
    ms = (C.c_double * len(ADJOINT_GROUPS))()
    _check(library().tf_adjoint_timing(ms, len(ADJOINT_GROUPS)), "tf_adjoint_timing")
    return dict(zip(ADJOINT_GROUPS, list(ms)))


TAPE_GROUPS = ("tape_forward", "recompute") + ADJOINT_GROUPS


class Tape:
    """Owns one ``tf_tape``: ``nsteps`` fixed steps of ``K`` iterations at
    ``dt`` with a checkpoint every ``every`` steps (0: ceil(sqrt(nsteps))).
    Keeps its context alive."""

    def __init__(self, ctx: Context, nsteps: int, K: int, dt: float, every: int = 0):
        h = C.c_void_p()
        _check(library().tf_tape_create(ctx.handle, int(nsteps), int(K), float(dt), int(every),
                                        C.byref(h)), "tf_tape_create")
        self.handle, self.ctx = h, ctx
        self.nsteps, self.K, self.dt = int(nsteps), int(K), float(dt)

    def close(self):
        if getattr(self, "handle", None):
            library().tf_tape_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tf_tape_create(ctx: Context, nsteps: int, K: int, dt: float, every: int = 0) -> Tape:
    return Tape(ctx, nsteps, K, dt, every)


def tf_tape_destroy(tape: Tape):
    tape.close()


def tf_tape_info(tape: Tape) -> dict:
    e, n, f = C.c_int(), C.c_int(), C.c_int()
    b = C.c_size_t()
    _check(library().tf_tape_info(tape.handle, C.byref(e), C.byref(n), C.byref(b), C.byref(f)),
           "tf_tape_info")
    return dict(every=e.value, checkpoints=n.value, bytes=b.value, forward_done=bool(f.value))


def tf_tape_forward(tape: Tape, h0, hT=None):
    """u^N of the tape's trajectory from ``h0`` (returns ``hT``)."""
    torch = _torch()
    if hT is None:
        hT = torch.empty_like(h0)
    r = library().tf_tape_forward(tape.handle, tape.ctx.ptr(h0, "h0"), tape.ctx.ptr(hT, "hT"))
    if r > 0:
        raise RuntimeError(f"tf_tape_forward: step failure {r} (the trajectory left the model's domain)")
    _check(r, "tf_tape_forward")
    return hT


def tf_tape_backward(tape: Tape, g, g_h0=None) -> dict:
    """Reverse of the last forward for the cotangent ``g`` of u^N: dict with
    ``g_h0`` (CUDA tensor), ``g_kappa`` and ``g_theta``."""
    torch = _torch()
    if g_h0 is None:
        g_h0 = torch.empty_like(g)
    gk, gt = C.c_double(), C.c_double()
    _check(library().tf_tape_backward(tape.handle, tape.ctx.ptr(g, "g"), tape.ctx.ptr(g_h0, "g_h0"),
                                      C.byref(gk), C.byref(gt)), "tf_tape_backward")
    return dict(g_h0=g_h0, g_kappa=gk.value, g_theta=gt.value)


def tf_tape_timing(tape: Tape) -> dict:
    """Kernel time (ms) of the tape's last forward and backward by group."""
    ms = (C.c_double * len(TAPE_GROUPS))()
    _check(library().tf_tape_timing(tape.handle, ms, len(TAPE_GROUPS)), "tf_tape_timing")
    return dict(zip(TAPE_GROUPS, list(ms)))


def trajectory(h0, theta, params: TfParams, dt: float, K: int, nsteps: int, every: int = 0):
    """u^N after ``nsteps`` fixed steps of ``K`` iterations from ``h0``, as a
    differentiable function of the film ``h0`` and of the contact angle
    ``theta`` (radians, a float64 tensor; kappa = (1 - cos theta)/(b M) of the
    power law).  ``params``: an FP64 power-law parameter set (its kappa and
    contact angle are replaced).  The forward keeps ceil(N/every)
    checkpoints; the backward recomputes one segment at a time and chains the
    steps' adjoints (tf_tape_backward)."""
    torch = _torch()

    class _Trajectory(torch.autograd.Function):
        @staticmethod
        def forward(actx, x, th):
            p = TfParams.from_buffer_copy(params)
            p.kappa = 0.0
            p.contact_angle = float(th)
            ctx = Context(p)
            tape = Tape(ctx, nsteps, K, dt, every)
            actx.tape = tape
            actx.theta_like = th
            return tf_tape_forward(tape, x.detach().contiguous())

        @staticmethod
        def backward(actx, g):
            r = tf_tape_backward(actx.tape, g.contiguous())
            th = actx.theta_like
            return r["g_h0"], torch.tensor(r["g_theta"], dtype=th.dtype, device=th.device)

    return _Trajectory.apply(h0, theta)


def tf_timing_enable(ctx: Context, on: bool = True):
    _check(library().tf_timing_enable(ctx.handle, int(bool(on))), "tf_timing_enable")


def tf_timing_get(ctx: Context) -> dict:
    t = TfTiming()
    _check(library().tf_timing_get(ctx.handle, C.byref(t)), "tf_timing_get")
    return {k: getattr(t, k) for k, _ in TfTiming._fields_}


def tf_spectrum_params_default(**overrides) -> TfSpectrumParams:
    sp = TfSpectrumParams()
    library().tf_spectrum_params_default(C.byref(sp))
    for k, v in overrides.items():
        if not hasattr(sp, k):
            raise AttributeError(k)
        setattr(sp, k, v)
    return sp


def _info_dict(i: TfSpectrumInfo) -> dict:
    return {k: getattr(i, k) for k, _ in TfSpectrumInfo._fields_}


class SpectrumPlan:
    """Owns one ``tf_spectrum_plan``: the radial Fourier analysis of
    ``(ny, nx)`` float64 CUDA grids with spacing ``ds``."""

    def __init__(self, nx: int, ny: int, ds: float, params: TfSpectrumParams, stream=None):
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.shape = (ny, nx)
        self.params = params
        h = C.c_void_p()
        _check(library().tf_spectrum_plan_create(int(nx), int(ny), float(ds), C.byref(params),
                                                 C.c_void_p(stream.cuda_stream), C.byref(h)),
               "tf_spectrum_plan_create")
        self.handle = h

    def info(self) -> dict:
        i = TfSpectrumInfo()
        _check(library().tf_spectrum_plan_info(self.handle, C.byref(i)), "tf_spectrum_plan_info")
        return _info_dict(i)

    def close(self):
        if getattr(self, "handle", None):
            library().tf_spectrum_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tf_spectrum_plan_create(nx: int, ny: int, ds: float, params: TfSpectrumParams,
                            stream=None) -> SpectrumPlan:
    return SpectrumPlan(nx, ny, ds, params, stream)


def tf_spectrum_plan_destroy(plan: SpectrumPlan):
    plan.close()


def tf_spectrum_plan_info(plan: SpectrumPlan) -> dict:
    return plan.info()


def tf_spectrum_run(plan: SpectrumPlan, h, outputs: bool = True, peak_cap: int = 64) -> dict:
    """Analyse ``h``; returns the info fields and, with ``outputs``, every
    stage as NumPy arrays (amplitude and smoothed [n_q, n_p], radial_q/_value,
    node_q/_value, curve_q/_value, peaks [(q, value)], highest first)."""
    import numpy as np
    torch = _torch()
    if not isinstance(h, torch.Tensor) or h.dtype != torch.float64 or not h.is_cuda:
        raise TypeError("h must be a torch.float64 CUDA tensor")
    if tuple(h.shape) != plan.shape or not h.is_contiguous():
        raise ValueError(f"h must be contiguous with shape {plan.shape}")
    i = TfSpectrumInfo()
    if not outputs:
        _check(library().tf_spectrum_run(plan.handle, C.c_void_p(h.data_ptr()), None, C.byref(i)),
               "tf_spectrum_run")
        return _info_dict(i)
    pi = plan.info()
    arrs = dict(amplitude=np.empty((pi["n_q"], pi["n_p"])), smoothed=np.empty((pi["n_q"], pi["n_p"])),
                radial_q=np.empty(pi["n_radii"]), radial_value=np.empty(pi["n_radii"]),
                node_q=np.empty(pi["n_intervals"] + 1), node_value=np.empty(pi["n_intervals"] + 1),
                curve_q=np.empty(pi["n_eval"]), curve_value=np.empty(pi["n_eval"]),
                peak_q=np.empty(max(1, peak_cap)), peak_value=np.empty(max(1, peak_cap)))
    o = TfSpectrumOut(**{k: a.ctypes.data for k, a in arrs.items()}, peak_cap=int(peak_cap))
    _check(library().tf_spectrum_run(plan.handle, C.c_void_p(h.data_ptr()), C.byref(o), C.byref(i)),
           "tf_spectrum_run")
    r = _info_dict(i)
    npk = min(i.n_peaks, peak_cap)
    pq, pv = arrs.pop("peak_q"), arrs.pop("peak_value")
    r.update(arrs)
    r["peaks"] = list(zip(pq[:npk].tolist(), pv[:npk].tolist()))
    return r


def tf_spectrum_timing(plan: SpectrumPlan) -> list:
    """Kernel durations (ms) of the last run: row DCTs, column DCTs,
    smoothing along p and q, radial means, and the fit with sampling and
    maxima (five kernels)."""
    ms = (C.c_double * 6)()
    _check(library().tf_spectrum_timing(plan.handle, ms, 6), "tf_spectrum_timing")
    return list(ms)


def params_for_workload(w: dict, precision: int = TF_FP64, **overrides) -> TfParams:
    """tf_params of a workload description (see tests/golden/workloads.json)."""
    p = tf_params_default(
        nx=int(w["N"]), ny=int(w["N"]), ds=float(w["ds"]), cap_C=float(w["cap_C"]),
        b=float(w["b"]), n=int(w["n"]), m=int(w["m"]), kappa=float(w["kappa"]),
        contact_angle=float(w["theta_c"]), theta=float(w["theta"]),
        newton_tol=float(w["tol"]), newton_max_iter=int(w["max_iter"]),
        dt_min=float(w["dt_min"]), dt_max=float(w["dt_max"]), dt_shrink=float(w["dt_shrink"]),
        dt_grow=float(w["dt_grow"]), grow_after=int(w["grow_after"]),
        rupture_h=float(w["rupture_h"]), model=int(w.get("model", TF_MODEL_POWERLAW)),
        precision=precision)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


__all__ = [n for n in dir() if n.startswith(("tf_", "TF_", "Tf"))] + [
    "Context", "SpectrumPlan", "library", "params_for_workload", "unrolled_step"]
