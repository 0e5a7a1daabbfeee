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


# --------------------------------------------------------------------------
# Trajectories of fixed steps with checkpoints (tf_tape_*)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nx,ny,K,nsteps,every", [(7, 5, 3, 5, 0), (7, 5, 3, 5, 2), (10, 9, 2, 4, 1),
                                                   (6, 11, 1, 3, 3), (8, 1, 3, 6, 4)])
def test_tape_matches_oracle_trajectory(torch, nx, ny, K, nsteps, every):
    M, p, dt = setup(nx, ny)
    u = S.spinodal_film(nx, ny, 1.0, 0.05, seed=3 * nx + ny)
    g = np.random.default_rng(nx * ny).standard_normal((ny, nx))
    hs = AD.trajectory(M, u, dt, K, nsteps)
    ref_g, ref_k = AD.trajectory_vjp(M, u, dt, K, nsteps, g)
    ctx = tf.Context(p)
    tape = tf.tf_tape_create(ctx, nsteps, K, dt, every)
    info = tf.tf_tape_info(tape)
    e = every or math.ceil(math.sqrt(nsteps))
    assert info["every"] == e and info["checkpoints"] == math.ceil(nsteps / e)
    assert not info["forward_done"]
    hT = tf.tf_tape_forward(tape, dev(torch, u))
    assert tf.tf_tape_info(tape)["forward_done"]
    assert np.max(np.abs(hT.cpu().numpy() - hs[-1])) <= 1e-13
    r = tf.tf_tape_backward(tape, dev(torch, g))
    assert np.max(np.abs(r["g_h0"].cpu().numpy() - ref_g)) <= 1e-10 * np.max(np.abs(ref_g))
    assert abs(r["g_kappa"] - ref_k) <= 1e-9 * abs(ref_k)


def test_tape_result_does_not_depend_on_the_interval(torch):
    # every segment recomputes the forward's own bits, so any checkpoint
    # interval gives the same result bit for bit; the forward is the same as
    # repeated fixed-iteration steps
    nx, ny, K, nsteps, dt = 96, 64, 3, 10, 0.02
    p = tf.tf_params_default(nx=nx, ny=ny, ds=1.5, precision=tf.TF_FP64)
    ctx = tf.Context(p)
    u = dev(torch, S.spinodal_film(nx, ny, 1.0, 0.02, seed=77))
    g = dev(torch, np.random.default_rng(78).standard_normal((ny, nx)))
    fw = tf.Context(tf.tf_params_default(nx=nx, ny=ny, ds=1.5, precision=tf.TF_FP64, newton_fixed_iter=K))
    cur = u.clone()
    for _ in range(nsteps):
        nxt = torch.empty_like(cur)
        tf.tf_newton_adi_step(fw, cur, nxt, dt)
        cur = nxt
    res = []
    for every in (1, 2, 3, 4, 10, 0):
        tape = tf.tf_tape_create(ctx, nsteps, K, dt, every)
        hT = tf.tf_tape_forward(tape, u)
        assert torch.equal(hT, cur)
        r = tf.tf_tape_backward(tape, g)
        r2 = tf.tf_tape_backward(tape, g)  # repeatable
        assert torch.equal(r["g_h0"], r2["g_h0"]) and r["g_kappa"] == r2["g_kappa"]
        res.append(r)
        t = tf.tf_tape_timing(tape)
        assert t["tape_forward"] > 0 and t["recompute"] > 0 and t["solve_t"] > 0
        assert t["forward"] == 0.0  # the reverse takes the iterates of the recomputed segments
    for r in res[1:]:
        assert torch.equal(r["g_h0"], res[0]["g_h0"])
        assert r["g_kappa"] == res[0]["g_kappa"]


def test_tape_arguments(torch):
    p = tf.tf_params_default(nx=16, ny=8, ds=1.0, precision=tf.TF_FP64)
    ctx = tf.Context(p)
    for bad in (dict(nsteps=0), dict(K=0), dict(K=65), dict(dt=0.0), dict(every=-1), dict(every=6)):
        kw = dict(nsteps=5, K=3, dt=0.01, every=0)
        kw.update(bad)
        with pytest.raises(RuntimeError):
            tf.tf_tape_create(ctx, **kw)
    with pytest.raises(RuntimeError):
        tf.tf_tape_create(tf.Context(tf.tf_params_default(nx=16, ny=8, ds=1.0, precision=tf.TF_FP32_BULK)),
                          5, 3, 0.01)
    tape = tf.tf_tape_create(ctx, 5, 3, 0.01)
    z = torch.ones((8, 16), dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):  # no forward yet
        tf.tf_tape_backward(tape, z)
    # a film that leaves the model's domain: reported, and the tape stays unusable
    neg = -z
    with pytest.raises(RuntimeError):
        tf.tf_tape_forward(tape, neg)
    assert not tf.tf_tape_info(tape)["forward_done"]
    with pytest.raises(RuntimeError):
        tf.tf_tape_backward(tape, z)


def test_trajectory_is_differentiable_in_torch(torch):
    # torch.autograd.gradcheck over the film and the contact angle
    nx, ny = 6, 5
    M, p, dt = setup(nx, ny)
    h = dev(torch, S.spinodal_film(nx, ny, 1.0, 0.05, seed=21)).requires_grad_(True)
    th = torch.tensor(math.radians(20.0), dtype=torch.float64, device="cuda", requires_grad=True)
    f = lambda x, t: tf.trajectory(x, t, p, dt, 2, 4, every=2)  # noqa: E731
    assert torch.autograd.gradcheck(f, (h, th), eps=1e-6, atol=1e-8, rtol=1e-6)
    out = f(h, th)
    assert np.max(np.abs(out.detach().cpu().numpy() - AD.trajectory(M, h.detach().cpu().numpy(), dt, 2, 4)[-1])) \
        <= 1e-13


def _loss_difference(a_p, a_m, t):
    # |a+ - t|^2 - |a- - t|^2 written as sum (a+ - a-)(a+ + a- - 2t): no
    # cancellation between two large sums
    return float(((a_p - a_m) * (a_p + a_m - 2.0 * t)).sum())


def test_adjoint_trajectory_workload_against_central_differences(torch):
    """The adjoint workload: 1024^2 on 16 lambda_m, 400 steps of 3 Newton
    iterations at dt = 0.01, loss |h(T) - h_target|^2 with h_target the same
    trajectory from another seed's film; gradients of the loss with respect
    to the initial film (32 random directions) and the contact angle against
    central differences of the GPU forward, to 1e-6 relative."""
    W = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))
    w = W["adjoint1k"]
    N, K, dt, ns = w["N"], w["fixed_iter"], w["dt_fixed"], w["steps"]
    p = tf.params_for_workload(w, tf.TF_FP64)
    th0 = w["theta_c"]

    def run(h0, th):
        q = tf.TfParams.from_buffer_copy(p)
        q.kappa, q.contact_angle = 0.0, th
        tape = tf.tf_tape_create(tf.Context(q), ns, K, dt)
        return tape, tf.tf_tape_forward(tape, h0)

    u = dev(torch, S.spinodal_film(N, N, w["h0"], w["eps"], w["seed"]))
    _, target = run(dev(torch, S.spinodal_film(N, N, w["h0"], w["eps"], w["target_seed"])), th0)
    tape, hT = run(u, th0)
    assert tf.tf_tape_info(tape)["every"] == 20
    r = tf.tf_tape_backward(tape, 2.0 * (hT - target))
    gh = r["g_h0"]
    rng = np.random.default_rng(5)
    worst = 0.0
    for _ in range(32):
        d = dev(torch, rng.standard_normal((N, N)))
        h = 1e-6
        _, ap = run(u + h * d, th0)
        _, am = run(u - h * d, th0)
        fd = _loss_difference(ap, am, target) / (2 * h)
        ad = float(torch.sum(gh * d))
        worst = max(worst, abs(fd - ad) / abs(ad))
    assert worst <= 1e-6, worst
    ht = 1e-4
    _, ap = run(u, th0 + ht)
    _, am = run(u, th0 - ht)
    fdt = _loss_difference(ap, am, target) / (2 * ht)
    assert abs(fdt - r["g_theta"]) <= 1e-6 * abs(r["g_theta"]), (fdt, r["g_theta"])
