"""The allocation-free residual against the context-based one.

tf_residual_noalloc is for callers that may not allocate device memory
(a host framework owning every allocation, a latency-bounded loop, a plugin
with buffers but no context).  It must give what tf_residual gives, call
after call, while sharing one fixed scratch array: two calls in a row with
different grids, sizes and precision modes are each compared with
tf_residual at the residual-parity tolerances (1e-13 FP64, 1e-12
FP32-bulk, relative to the residual's largest value when that exceeds
1).  Grids above its fixed capacity must be refused.  This file is
collected last and must pass alone or after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

KAPPA = 1.2061475842818314


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    L = tf.library()
    L.tf_residual_noalloc.argtypes = [C.POINTER(tf.TfParams), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_double, C.c_void_p, C.POINTER(tf.TfNorms)]
    L.tf_residual_noalloc.restype = C.c_int
    return T


def _pair(torch, nx, ny, mode, seed):
    h_old = S.spinodal_film(nx, ny, 1.0, 0.05, seed=seed)
    h_k = h_old + 0.01 * S.spinodal_film(nx, ny, 0.0, 1.0, seed=seed + 1)
    return (torch.from_numpy(h_k).cuda(), torch.from_numpy(h_old).cuda())


def test_noalloc_residual_matches_context_residual_twice(torch):
    L = tf.library()
    cases = [(300, 257, tf.TF_FP64, 3.0, 11), (1024, 2048, tf.TF_FP32_BULK, 7.0, 12)]
    for nx, ny, mode, dt, seed in cases:  # two calls in a row on the shared scratch
        p = tf.tf_params_default(nx=nx, ny=ny, ds=1.3, kappa=KAPPA, precision=mode)
        h_k, h_old = _pair(torch, nx, ny, mode, seed)
        G_ref = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
        ctx = tf.Context(p)
        ref = tf.tf_residual(ctx, h_k, h_old, dt, G_ref)
        ctx.close()
        G = torch.full((ny, nx), np.nan, dtype=torch.float64, device="cuda")
        n = tf.TfNorms()
        stream = torch.cuda.current_stream().cuda_stream
        rc = L.tf_residual_noalloc(C.byref(p), C.c_void_p(stream), C.c_void_p(h_k.data_ptr()),
                                   C.c_void_p(h_old.data_ptr()), dt, C.c_void_p(G.data_ptr()),
                                   C.byref(n))
        assert rc == tf.TF_OK
        # FP64: round-off of the same stencil; FP32-bulk: the two entry points
        # form b^n with different double-float kernels, each accurate to about
        # 2^-46 of the terms it adds, so the bound scales with the residual
        # (|G| reaches 3 on these films)
        scale = max(1.0, float(G_ref.abs().max()))
        tol = (1e-13 if mode == tf.TF_FP64 else 1e-12) * scale
        assert float((G - G_ref).abs().max()) <= tol
        assert abs(n.gnorm - ref["gnorm"]) <= tol
        assert n.mass == ref["mass"] and n.hmin == ref["hmin"]


def test_noalloc_refuses_grids_above_capacity(torch):
    L = tf.library()
    p = tf.tf_params_default(nx=2048, ny=1025, ds=1.0, kappa=KAPPA)  # 2^21 + 2048 cells
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    rc = L.tf_residual_noalloc(C.byref(p), None, C.c_void_p(x.data_ptr()),
                               C.c_void_p(x.data_ptr()), 1.0, C.c_void_p(x.data_ptr()), None)
    assert rc == tf.TF_ERR_ARG
