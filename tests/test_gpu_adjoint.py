"""GPU parity of the discrete adjoint of the fixed-iteration Newton--ADI step
(tf_adjoint_step) against the oracle (complex-step Jacobian, transposed).

Tolerances: the GPU's reverse sweep and the oracle's full Jacobian differ by
rounding only (both exact derivatives of maps that agree to ~1e-15), so the
cotangents agree to 1e-10 of their largest entry.  At the 1024^2 adjoint
workload the adjoint is checked against central finite differences of the
GPU's own forward step on 32 random directions: <g, (Phi(u+hd) - Phi(u-hd))/2h>
against <g_h, d>, to 1e-6 relative (h = 1e-6 |u|: truncation O(h^2) and
rounding O(1e-16/h)).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import oracle.adjoint as AD
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    tf.library()
    return T


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def setup(nx, ny, model=O.MODEL_POWERLAW):
    kappa = O.kappa_from_contact_angle(math.radians(20.0), 0.1, 3, 2)
    qm, sm = O.lsa(O.Model(nx=1, ny=1, ds=1.0, kappa=kappa), 1.0)
    ds = 2 * math.pi / qm / 6
    kw = dict(model=model, c0=0.6, c1=0.25) if model == O.MODEL_LINEAR else {}
    M = O.Model(nx=nx, ny=ny, ds=ds, kappa=kappa, **kw)
    p = tf.tf_params_default(nx=nx, ny=ny, ds=ds, precision=tf.TF_FP64,
                             model=tf.TF_MODEL_LINEAR if model == O.MODEL_LINEAR else tf.TF_MODEL_POWERLAW,
                             c0=0.6, c1=0.25)
    dt = (2.0 / sm) / 400 if model == O.MODEL_POWERLAW else 0.05
    return M, p, dt


@pytest.mark.parametrize("nx,ny,K", [(7, 5, 3), (10, 9, 3), (12, 6, 1), (6, 11, 2), (1, 8, 3), (8, 1, 3), (13, 12, 3)])
@pytest.mark.parametrize("model", [O.MODEL_POWERLAW, O.MODEL_LINEAR])
def test_adjoint_matches_oracle(torch, nx, ny, K, model):
    M, p, dt = setup(nx, ny, model)
    u = S.spinodal_film(nx, ny, 1.0, 0.05, seed=nx * 7 + ny)
    g = np.random.default_rng(nx + 100 * ny).standard_normal((ny, nx))
    ref_h = AD.step_fixed(M, u, dt, K)
    ref_g, ref_k = AD.vjp(M, u, dt, K, g)
    ctx = tf.Context(p)
    h_new = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    r = tf.tf_adjoint_step(ctx, dev(torch, u), dt, K, dev(torch, g), h_new=h_new)
    assert np.max(np.abs(h_new.cpu().numpy() - ref_h)) <= 1e-13
    gh = r["g_h"].cpu().numpy()
    assert np.max(np.abs(gh - ref_g)) <= 1e-10 * np.max(np.abs(ref_g))
    if model == O.MODEL_POWERLAW:
        assert abs(r["g_kappa"] - ref_k) <= 1e-9 * abs(ref_k)
        assert abs(r["g_theta"] - ref_k * AD.dkappa_dtheta(math.radians(20.0), 0.1, 3, 2)) <= 1e-9 * abs(r["g_theta"])
    else:
        assert r["g_kappa"] == 0.0


def test_adjoint_rejects_unsupported_contexts(torch):
    for kw in (dict(precision=tf.TF_FP32_BULK), dict(model=tf.TF_MODEL_NLC, cap_C=0.0857, b=0.01)):
        p = tf.tf_params_default(nx=8, ny=8, ds=1.0, **kw)
        ctx = tf.Context(p)
        z = torch.ones((8, 8), dtype=torch.float64, device="cuda")
        with pytest.raises(RuntimeError):
            tf.tf_adjoint_step(ctx, z, 1e-3, 3, z.clone())
    ctx = tf.Context(tf.tf_params_default(nx=8, ny=8, ds=1.0))
    z = torch.ones((8, 8), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        tf.tf_adjoint_step(ctx, z, 1e-3, 0, z.clone())


def test_adjoint_workload_against_central_differences(torch):
    # the 1024^2 adjoint workload: 16 lambda_m square, dt = 0.01, three Newton
    # iterations
    W = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))
    w = W["adjoint1k"]
    N, K, dt = w["N"], w["fixed_iter"], w["dt_fixed"]
    p = tf.params_for_workload(w, tf.TF_FP64)
    ctx = tf.Context(p)
    u = dev(torch, S.spinodal_film(N, N, w["h0"], w["eps"], w["seed"]))
    rng = np.random.default_rng(5)
    g = dev(torch, rng.standard_normal((N, N)))
    r = tf.tf_adjoint_step(ctx, u, dt, K, g)
    gh = r["g_h"]
    fw = tf.Context(tf.params_for_workload(w, tf.TF_FP64, newton_fixed_iter=K))
    out_p, out_m = torch.empty_like(u), torch.empty_like(u)
    worst = 0.0
    for _ in range(32):
        d = dev(torch, rng.standard_normal((N, N)))
        h = 1e-6
        tf.tf_newton_adi_step(fw, u + h * d, out_p, dt)
        tf.tf_newton_adi_step(fw, u - h * d, out_m, dt)
        fd = float(torch.sum(g * (out_p - out_m))) / (2 * h)
        ad = float(torch.sum(gh * d))
        worst = max(worst, abs(fd - ad) / abs(ad))
    assert worst <= 1e-6, worst
    # kappa: central difference in kappa through the forward step (h = 1e-4
    # kappa: the kappa derivative is small, so a smaller h drowns in rounding)
    hk = 1e-4 * ctx.kappa
    ctx_p = tf.Context(tf.params_for_workload(w, tf.TF_FP64, newton_fixed_iter=K, kappa=ctx.kappa + hk))
    ctx_m = tf.Context(tf.params_for_workload(w, tf.TF_FP64, newton_fixed_iter=K, kappa=ctx.kappa - hk))
    tf.tf_newton_adi_step(ctx_p, u, out_p, dt)
    tf.tf_newton_adi_step(ctx_m, u, out_m, dt)
    fdk = float(torch.sum(g * (out_p - out_m))) / (2 * hk)
    assert abs(fdk - r["g_kappa"]) <= 1e-6 * abs(r["g_kappa"])


def test_unrolled_step_is_differentiable_in_torch(torch):
    # torch.autograd.gradcheck: the backward (tf_adjoint_step) against the
    # forward's finite differences, every input direction of a small film
    M, p, dt = setup(6, 5)
    ctx = tf.Context(p)
    h = dev(torch, S.spinodal_film(6, 5, 1.0, 0.05, seed=12)).requires_grad_(True)
    assert torch.autograd.gradcheck(lambda x: tf.unrolled_step(x, ctx, dt, 3), (h,), eps=1e-6, atol=1e-8,
                                     rtol=1e-6)
    out = tf.unrolled_step(h, ctx, dt, 3)
    assert np.max(np.abs(out.detach().cpu().numpy() - AD.step_fixed(M, h.detach().cpu().numpy(), dt, 3))) <= 1e-13
