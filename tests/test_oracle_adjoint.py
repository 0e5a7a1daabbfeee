"""Pins of the adjoint oracle (the unrolled Newton--ADI step, Sec. Numerical
Method, differentiated by complex steps).

- the complex-capable NumPy forward map equals the C oracle on real inputs:
  D, the line bands of J_x and J_y, one Newton iteration, and the whole
  step with a fixed number of iterations;
- directional derivatives (columns of the Jacobian, and the kappa column)
  equal central finite differences of the C oracle's step on random
  directions to the finite-difference error;
- the linear model: the step is linear in u^n, so the Jacobian times u^n
  reproduces the step itself;
- d kappa / d theta_c against a finite difference of the C oracle's kappa.
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.adjoint as AD
from paper_1806_10550_gb300 import synthetic as S


def model(nx, ny, **kw):
    kappa = O.kappa_from_contact_angle(math.radians(20.0), 0.1, 3, 2)
    qm, sm = O.lsa(O.Model(nx=1, ny=1, ds=1.0, kappa=kappa), 1.0)
    ds = 2 * math.pi / qm / 6
    M = O.Model(nx=nx, ny=ny, ds=ds, kappa=kappa, **kw)
    return M, sm


def c_step(M, un, dt, K):
    out, info = O.step(M, O.Control(fixed_iter=K), un, dt)
    return out


@pytest.mark.parametrize("nx,ny", [(7, 5), (10, 9), (1, 8)])
def test_numpy_forward_matches_c_oracle(nx, ny):
    M, sm = model(nx, ny)
    dt = 0.05 / sm
    u = S.spinodal_film(nx, ny, 1.0, 0.05, seed=nx + ny)
    assert np.max(np.abs(AD.operator_D(M, u) - O.operator_D(M, u))) < 1e-13 * np.max(np.abs(O.operator_D(M, u)))
    L = AD.laplacian(M, u)
    for j in range(ny):
        ref = O.band_to_dense(O.jx_row(M, u, dt, j))
        assert np.max(np.abs(AD.line_matrix(M, u[j, :], L[j, :], dt) - ref)) < 1e-13
    for i in range(nx):
        ref = O.band_to_dense(O.jy_col(M, u, dt, i))
        assert np.max(np.abs(AD.line_matrix(M, u[:, i], L[:, i], dt) - ref)) < 1e-13
    bn = O.explicit_part(M, u, dt)
    r = O.newton_iteration(M, u, bn, dt)
    w, v, un = AD.newton_iteration(M, u, bn, dt)
    assert np.max(np.abs(w - r["w"])) < 1e-12 * np.max(np.abs(r["w"]))
    assert np.max(np.abs(un - r["unew"])) < 1e-14
    assert np.max(np.abs(AD.step_fixed(M, u, dt, 3) - c_step(M, u, dt, 3))) < 1e-14


@pytest.mark.parametrize("model_id", [O.MODEL_POWERLAW, O.MODEL_LINEAR])
def test_directional_derivatives_match_central_differences(model_id):
    nx, ny, K = 6, 5, 3
    kw = dict(model=model_id, c0=0.7, c1=0.3) if model_id == O.MODEL_LINEAR else {}
    M, sm = model(nx, ny, **kw)
    dt = (2.0 / sm) / 400 if model_id == O.MODEL_POWERLAW else 0.05
    u = S.spinodal_film(nx, ny, 1.0, 0.05, seed=3)
    J, Jk = AD.jacobian(M, u, dt, K)
    rng = np.random.default_rng(1)
    for _ in range(8):
        d = rng.standard_normal(u.shape)
        h = 1e-6
        fd = (c_step(M, u + h * d, dt, K) - c_step(M, u - h * d, dt, K)) / (2 * h)
        jd = (J @ d.ravel()).reshape(u.shape)
        assert np.max(np.abs(jd - fd)) < 1e-7 * max(1.0, np.max(np.abs(fd)))
    if model_id == O.MODEL_POWERLAW:
        hk = 1e-6 * M.kappa
        Mp = O.Model(**{**M.__dict__, "kappa": M.kappa + hk})
        Mm = O.Model(**{**M.__dict__, "kappa": M.kappa - hk})
        fdk = (c_step(Mp, u, dt, K) - c_step(Mm, u, dt, K)) / (2 * hk)
        assert np.max(np.abs(Jk - fdk.ravel())) < 1e-6 * max(1e-12, np.max(np.abs(fdk)))


def test_vjp_is_transpose_of_the_jacobian():
    M, sm = model(5, 4)
    dt = (2.0 / sm) / 400
    u = S.spinodal_film(5, 4, 1.0, 0.05, seed=8)
    g = np.random.default_rng(2).standard_normal(u.shape)
    J, Jk = AD.jacobian(M, u, dt, 3)
    gu, gk = AD.vjp(M, u, dt, 3, g)
    d = np.random.default_rng(3).standard_normal(u.shape)
    assert abs(np.sum(gu * d) - g.ravel() @ (J @ d.ravel())) < 1e-12 * np.sum(np.abs(g))
    assert abs(gk - g.ravel() @ Jk) < 1e-12 * abs(gk) + 1e-300


def test_linear_model_step_is_linear():
    M, _ = model(6, 4, model=O.MODEL_LINEAR, c0=0.5, c1=0.2)
    u = S.spinodal_film(6, 4, 1.0, 0.05, seed=4)
    J, _ = AD.jacobian(M, u, 0.1, 3)
    assert np.max(np.abs((J @ u.ravel()).reshape(u.shape) - c_step(M, u, 0.1, 3))) < 1e-13


def test_dkappa_dtheta():
    th, h = math.radians(23.0), 1e-6
    fd = (O.kappa_from_contact_angle(th + h, 0.1, 3, 2) - O.kappa_from_contact_angle(th - h, 0.1, 3, 2)) / (2 * h)
    assert abs(AD.dkappa_dtheta(th, 0.1, 3, 2) - fd) < 1e-8 * abs(fd)


def test_trajectory_vjp_is_the_chain_rule():
    """The chained steps' adjoints equal the transposed complex-step Jacobian
    of the whole trajectory (one complex step through all N steps), and the
    trajectory's last state equals the C oracle run step by step."""
    M, sm = model(5, 4)
    dt, K, N = (2.0 / sm) / 400, 2, 4
    u = S.spinodal_film(5, 4, 1.0, 0.05, seed=12)
    g = np.random.default_rng(13).standard_normal(u.shape)
    hs = AD.trajectory(M, u, dt, K, N)
    c = u
    for _ in range(N):
        c = c_step(M, c, dt, K)
    assert np.max(np.abs(hs[-1] - c)) < 1e-13
    J, Jk = AD.trajectory_jacobian(M, u, dt, K, N)
    gu, gk = AD.trajectory_vjp(M, u, dt, K, N, g)
    assert np.max(np.abs(gu.ravel() - J.T @ g.ravel())) < 1e-11 * np.max(np.abs(gu))
    assert abs(gk - Jk @ g.ravel()) < 1e-11 * abs(gk)
