"""GB300 Newton--ADI thin-film solver: Python binding of ``libtfadi.so``.

Argument marshalling only: every step of the time integration runs in the
CUDA kernels of ``csrc/`` behind the C ABI of ``include/tf.h``.  Grids are
``torch.float64`` CUDA tensors of shape ``(ny, nx)`` (row-major, x
contiguous); PyTorch supplies device memory and the stream.  There is no
CPU fallback: without the built library or a CUDA device every call raises.

Functions carry the names of the C ABI: ``tf_params_default``, ``tf_init``,
``tf_destroy``, ``tf_residual``, ``tf_newton_iteration``,
``tf_newton_adi_step``, ``tf_advance``, ``tf_ensemble_advance``, ``tf_strerror``.
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
        ("pol_d", C.c_double),
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
                             C.POINTER(TfAdvanceInfo)]
    L.tf_ensemble_advance.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp), C.POINTER(dp),
                                      C.POINTER(dp), C.POINTER(dp), C.POINTER(C.c_int),
                                      C.POINTER(TfAdvanceInfo)]
    L.tf_timing_enable.argtypes = [vp, C.c_int]
    L.tf_timing_get.argtypes = [vp, C.POINTER(TfTiming)]
    for f in ("tf_init", "tf_residual", "tf_newton_iteration", "tf_newton_adi_step", "tf_advance",
              "tf_ensemble_advance", "tf_timing_enable", "tf_timing_get"):
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
               dt_replay=None, iter_replay=None, records: bool = True):
    """Advance ``h`` in place; returns (info dict, list of per-attempt records)."""
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
    _check(library().tf_advance(ctx.handle, ctx.ptr(h, "h"), float(t0), float(t_end), float(dt0),
                                int(max_attempts), dtr, itr, recs, C.byref(info)), "tf_advance")
    out = []
    if records:
        for r in recs[: info.attempts]:
            out.append(dict(t=r.t, dt=r.dt, accepted=bool(r.accepted), iterations=r.iterations,
                            status=r.status, err=r.err, gnorm=r.gnorm, mass=r.mass, hmin=r.hmin))
    return dict(status=info.status, attempts=info.attempts, accepted=info.accepted,
                newton_iterations=info.newton_iterations, t=info.t, dt=info.dt), out


def tf_ensemble_advance(ctxs, hs, t0, t_end, dt0, max_attempts):
    """Advance independent films together (``tf_advance`` on each, their
    work interleaved on the contexts' streams).  ``ctxs``: contexts, one per
    film, each best on its own stream; ``hs``: their grids (advanced in
    place); ``t0``, ``t_end``, ``dt0``, ``max_attempts``: one value or one per
    film.  Returns one info dict per film."""
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
    _check(library().tf_ensemble_advance(n, ctx_a, h_a, arr(t0, C.c_double), arr(t_end, C.c_double),
                                         arr(dt0, C.c_double), arr(max_attempts, C.c_int), infos),
           "tf_ensemble_advance")
    return [dict(status=i.status, attempts=i.attempts, accepted=i.accepted,
                 newton_iterations=i.newton_iterations, t=i.t, dt=i.dt) for i in infos[:n]]


def tf_timing_enable(ctx: Context, on: bool = True):
    _check(library().tf_timing_enable(ctx.handle, int(bool(on))), "tf_timing_enable")


def tf_timing_get(ctx: Context) -> dict:
    t = TfTiming()
    _check(library().tf_timing_get(ctx.handle, C.byref(t)), "tf_timing_get")
    return {k: getattr(t, k) for k, _ in TfTiming._fields_}


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
    "Context", "library", "params_for_workload"]
