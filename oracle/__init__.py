"""FP64 CPU oracle of the Newton--ADI thin-film time step (test infrastructure).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The CUDA library
and its Python binding never import, link or call it.

The arithmetic lives in ``tf_oracle.c`` (plain C, IEEE double, no FMA
contraction).  This module compiles it on first use with ``gcc`` and wraps it
with ``ctypes`` over NumPy float64 arrays in row-major ``[ny, nx]`` layout.
The radial Fourier analysis of films (App. Radial Fourier Transform) is
``oracle.radial_fourier`` (NumPy/SciPy, FP64); the discrete adjoint of the
unrolled time step is ``oracle.adjoint`` (complex steps through a NumPy
restatement of the forward map).

Paper: Lam, Cummings & Kondic, "Computing dynamics of thin films via large
scale GPU-based simulations" -- Sec. Numerical Method (flux form, eq.
GovEqnCell2; trapezoidal rule, eq. TrapRule; Newton and ADI, eqs.
NewtonIterativeForm and JacobianSystem1-3; adaptive time stepping, Fig.
FlowChartTime and eq. NewtonError; boundary conditions, eq.
BoundaryConditions).
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tf_oracle.c")
_HDR = os.path.join(_HERE, "tf_oracle.h")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

MODEL_POWERLAW = 0
MODEL_LINEAR = 1
MODEL_NLC = 2
MODEL_POLYMER = 3


class _Model(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("ds", C.c_double), ("model", C.c_int),
        ("cap_C", C.c_double), ("b", C.c_double), ("kappa", C.c_double),
        ("n", C.c_int), ("m", C.c_int), ("c0", C.c_double), ("c1", C.c_double),
        ("theta", C.c_double),
        ("nlc_K", C.c_double), ("nlc_N", C.c_double), ("nlc_beta", C.c_double),
        ("nlc_w", C.c_double),
        ("pol_C", C.c_double), ("pol_A1", C.c_double), ("pol_A2", C.c_double),
        ("pol_d", C.c_double),
    ]


class _Control(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("max_iter", C.c_int), ("fixed_iter", C.c_int),
        ("dt_min", C.c_double), ("dt_max", C.c_double), ("dt_shrink", C.c_double),
        ("dt_grow", C.c_double), ("grow_after", C.c_int), ("rupture_h", C.c_double),
    ]


class _StepInfo(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("iterations", C.c_int), ("err", C.c_double),
        ("gnorm", C.c_double), ("mass", C.c_double), ("hmin", C.c_double),
    ]


class _Record(C.Structure):
    _fields_ = [
        ("t", C.c_double), ("dt", C.c_double), ("accepted", C.c_int),
        ("iterations", C.c_int), ("status", C.c_int), ("err", C.c_double),
        ("gnorm", C.c_double), ("mass", C.c_double), ("hmin", C.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile ``tf_oracle.c`` into ``oracle/_build/liboracle.so``.

    FMA contraction is off so that every product and sum rounds separately,
    as the C source is written.  OpenMP (over independent lines and rows) is
    used when the compiler supports it; it changes no result.
    """
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        raise RuntimeError("oracle build needs gcc")
    base = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    try:
        subprocess.run(base[:-1] + ["-fopenmp", "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        L.or_kappa_from_contact_angle.restype = C.c_double
        L.or_kappa_from_contact_angle.argtypes = [C.c_double, C.c_double, C.c_int, C.c_int]
        L.or_dpi.restype = C.c_double
        L.or_dpi.argtypes = [C.POINTER(_Model), C.c_double]
        L.or_pi.argtypes = [C.POINTER(_Model), C.c_double, dp, dp, dp]
        L.or_mobility.argtypes = [C.POINTER(_Model), C.c_double, dp, dp, dp, dp]
        L.or_lsa.argtypes = [C.POINTER(_Model), C.c_double, dp, dp]
        L.or_laplacian.argtypes = [C.POINTER(_Model), dp, dp]
        L.or_operator_D.argtypes = [C.POINTER(_Model), dp, dp]
        L.or_explicit_part.argtypes = [C.POINTER(_Model), dp, C.c_double, dp]
        L.or_residual.argtypes = [C.POINTER(_Model), dp, dp, C.c_double, dp]
        L.or_jx_row.argtypes = [C.POINTER(_Model), dp, C.c_double, C.c_int, dp]
        L.or_jy_col.argtypes = [C.POINTER(_Model), dp, C.c_double, C.c_int, dp]
        L.or_penta_solve.restype = C.c_int
        L.or_penta_solve.argtypes = [C.c_int, dp, dp, dp]
        L.or_newton_iteration.restype = C.c_int
        L.or_newton_iteration.argtypes = [C.POINTER(_Model), dp, dp, C.c_double,
                                          dp, dp, dp, dp, dp, dp]
        L.or_step.restype = C.c_int
        L.or_step.argtypes = [C.POINTER(_Model), C.POINTER(_Control), dp, C.c_double,
                              dp, C.POINTER(_StepInfo)]
        L.or_advance.restype = C.c_int
        L.or_advance.argtypes = [C.POINTER(_Model), C.POINTER(_Control), dp, C.c_double,
                                 C.c_double, C.c_double, C.c_int, dp,
                                 C.POINTER(C.c_int), C.POINTER(_Record), dp, dp,
                                 C.POINTER(C.c_int)]
        L.or_num_threads.restype = C.c_int
        L.or_set_num_threads.restype = None
        L.or_set_num_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


@dataclass
class Model:
    """The PDE and its discretisation (names follow the paper)."""
    nx: int
    ny: int
    ds: float
    model: int = MODEL_POWERLAW
    cap_C: float = 1.0
    b: float = 0.1
    kappa: float = 0.0
    n: int = 3
    m: int = 2
    c0: float = 1.0
    c1: float = 1.0
    theta: float = 0.5
    # NLC model, eq. NLC_paras (K, N, beta, w; with cap_C = 0.0857, b = 0.01)
    nlc_K: float = 36.0
    nlc_N: float = 1.67
    nlc_beta: float = 1.0
    nlc_w: float = 0.05
    # polymer model, eq. Polymer_scales (C, A_SiOx, A_Si, d; with cap_C = 0.00581)
    pol_C: float = 1.181
    pol_A1: float = 41.25
    pol_A2: float = -243.75
    pol_d: float = 191.0

    def c(self) -> _Model:
        return _Model(self.nx, self.ny, self.ds, self.model, self.cap_C, self.b,
                      self.kappa, self.n, self.m, self.c0, self.c1, self.theta,
                      self.nlc_K, self.nlc_N, self.nlc_beta, self.nlc_w,
                      self.pol_C, self.pol_A1, self.pol_A2, self.pol_d)


@dataclass
class Control:
    """Newton and time-step control (Fig. FlowChartTime, eq. NewtonError)."""
    tol: float = 1e-10
    max_iter: int = 10
    fixed_iter: int = 0
    dt_min: float = 1e-9
    dt_max: float = 1e30
    dt_shrink: float = 0.5
    dt_grow: float = 1.25
    grow_after: int = 5
    rupture_h: float = 0.0

    def c(self) -> _Control:
        return _Control(self.tol, self.max_iter, self.fixed_iter, self.dt_min,
                        self.dt_max, self.dt_shrink, self.dt_grow, self.grow_after,
                        self.rupture_h)


def kappa_from_contact_angle(theta_c: float, b: float, n: int, m: int) -> float:
    return lib().or_kappa_from_contact_angle(theta_c, b, n, m)


def mobility(M: Model, h: float):
    f0, f1, d0, d1 = (C.c_double() for _ in range(4))
    lib().or_mobility(C.byref(M.c()), h, C.byref(f0), C.byref(f1), C.byref(d0),
                      C.byref(d1))
    return f0.value, f1.value, d0.value, d1.value


def dpi(M: Model, h: float) -> float:
    return lib().or_dpi(C.byref(M.c()), h)


def pi_derivs(M: Model, h: float):
    """(Pi, Pi', Pi'') of the model's disjoining pressure at height h."""
    p, d1, d2 = C.c_double(), C.c_double(), C.c_double()
    lib().or_pi(C.byref(M.c()), h, C.byref(p), C.byref(d1), C.byref(d2))
    return p.value, d1.value, d2.value


def lsa(M: Model, h0: float):
    """(q_m, sigma_m) of a flat film of height h0."""
    qm, sm = C.c_double(), C.c_double()
    lib().or_lsa(C.byref(M.c()), h0, C.byref(qm), C.byref(sm))
    return qm.value, sm.value


def _grid(M: Model, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    assert u.shape == (M.ny, M.nx), (u.shape, (M.ny, M.nx))
    return u


def laplacian(M: Model, u):
    u = _grid(M, u)
    out = np.empty_like(u)
    lib().or_laplacian(C.byref(M.c()), _p(u), _p(out))
    return out


def operator_D(M: Model, u):
    u = _grid(M, u)
    out = np.empty_like(u)
    lib().or_operator_D(C.byref(M.c()), _p(u), _p(out))
    return out


def explicit_part(M: Model, un, dt: float):
    un = _grid(M, un)
    out = np.empty_like(un)
    lib().or_explicit_part(C.byref(M.c()), _p(un), dt, _p(out))
    return out


def residual(M: Model, uk, bn, dt: float):
    uk, bn = _grid(M, uk), _grid(M, bn)
    out = np.empty_like(uk)
    lib().or_residual(C.byref(M.c()), _p(uk), _p(bn), dt, _p(out))
    return out


def jx_row(M: Model, uk, dt: float, j: int):
    uk = _grid(M, uk)
    band = np.empty((M.nx, 5))
    lib().or_jx_row(C.byref(M.c()), _p(uk), dt, j, _p(band))
    return band


def jy_col(M: Model, uk, dt: float, i: int):
    uk = _grid(M, uk)
    band = np.empty((M.ny, 5))
    lib().or_jy_col(C.byref(M.c()), _p(uk), dt, i, _p(band))
    return band


def band_to_dense(band: np.ndarray) -> np.ndarray:
    n = band.shape[0]
    A = np.zeros((n, n))
    for r in range(n):
        for c in range(5):
            col = r + c - 2
            if 0 <= col < n:
                A[r, col] = band[r, c]
    return A


def penta_solve(band, rhs):
    band = np.ascontiguousarray(band, dtype=np.float64)
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    n = rhs.shape[0]
    x = np.zeros(n)
    s = lib().or_penta_solve(n, _p(band), _p(rhs), _p(x))
    return x, s


def newton_iteration(M: Model, uk, bn, dt: float):
    """One iteration: returns dict with G, w, v, unew, err, gnorm, status."""
    uk, bn = _grid(M, uk), _grid(M, bn)
    G, w, v, unew = (np.empty_like(uk) for _ in range(4))
    err, gn = C.c_double(), C.c_double()
    s = lib().or_newton_iteration(C.byref(M.c()), _p(uk), _p(bn), dt, _p(G), _p(w),
                                  _p(v), _p(unew), C.byref(err), C.byref(gn))
    return dict(G=G, w=w, v=v, unew=unew, err=err.value, gnorm=gn.value, status=s)


def step(M: Model, ctl: Control, un, dt: float):
    un = _grid(M, un)
    out = np.empty_like(un)
    info = _StepInfo()
    s = lib().or_step(C.byref(M.c()), C.byref(ctl.c()), _p(un), dt, _p(out),
                      C.byref(info))
    return out, dict(status=s, iterations=info.iterations, err=info.err,
                     gnorm=info.gnorm, mass=info.mass, hmin=info.hmin)


@dataclass
class AdvanceResult:
    h: np.ndarray
    t: float
    dt: float
    status: int
    records: list = field(default_factory=list)

    def accepted(self):
        return [r for r in self.records if r["accepted"]]


def advance(M: Model, ctl: Control, h0, t0: float, t_end: float, dt0: float,
            max_attempts: int, dt_replay=None, iter_replay=None) -> AdvanceResult:
    """Adaptive time stepping of Fig. FlowChartTime; replay of accepted steps
    when ``dt_replay`` (and optionally ``iter_replay``) is given."""
    h = np.array(_grid(M, h0), dtype=np.float64, copy=True)
    recs = (_Record * max(1, max_attempts))()
    t, dt, st = C.c_double(), C.c_double(), C.c_int()
    dtr = None
    itr = None
    if dt_replay is not None:
        dtr_a = np.ascontiguousarray(dt_replay, dtype=np.float64)
        assert dtr_a.shape[0] >= max_attempts
        dtr = _p(dtr_a)
    if iter_replay is not None:
        itr_a = np.ascontiguousarray(iter_replay, dtype=np.int32)
        assert itr_a.shape[0] >= max_attempts
        itr = itr_a.ctypes.data_as(C.POINTER(C.c_int))
    n = lib().or_advance(C.byref(M.c()), C.byref(ctl.c()), _p(h), t0, t_end, dt0,
                         max_attempts, dtr, itr, recs, C.byref(t), C.byref(dt),
                         C.byref(st))
    records = [dict(t=r.t, dt=r.dt, accepted=bool(r.accepted), iterations=r.iterations,
                    status=r.status, err=r.err, gnorm=r.gnorm, mass=r.mass, hmin=r.hmin)
               for r in recs[:n]]
    return AdvanceResult(h=h, t=t.value, dt=dt.value, status=st.value, records=records)


def num_threads() -> int:
    return lib().or_num_threads()


def set_num_threads(n: int) -> None:
    """Threads of the following oracle calls; the results do not depend on
    it (each line is one thread's work, with the same arithmetic)."""
    lib().or_set_num_threads(int(n))
