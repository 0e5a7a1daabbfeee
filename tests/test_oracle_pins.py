"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms (the discrete single-mode amplification, the linear model's matrix
form, the dispersion relation), invariants (mass, flatness, mirror symmetry,
dimensional reduction), library routines (LAPACK dense solves) and finite
differences of the residual.  A dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1806_10550_gb300 import synthetic as S

TH20 = math.radians(20.0)
KAPPA = 1.2061475842818314  # (1 - cos 20 deg) / (0.1 * 1/2), checked below


def pl_model(nx, ny, ds, **kw):
    return O.Model(nx=nx, ny=ny, ds=ds, kappa=KAPPA, **kw)


def lin_model(nx, ny, ds, c0=1.0, c1=1.0, **kw):
    return O.Model(nx=nx, ny=ny, ds=ds, model=O.MODEL_LINEAR, c0=c0, c1=c1, **kw)


def neumann_second_difference(n, ds):
    """1-D second difference with even reflection: rows [1,-2,1]/ds^2, the
    missing neighbour at a wall replaced by the cell itself."""
    L = np.zeros((n, n))
    for i in range(n):
        if i > 0:
            L[i, i - 1] += 1.0
            L[i, i] -= 1.0
        if i < n - 1:
            L[i, i + 1] += 1.0
            L[i, i] -= 1.0
    return L / (ds * ds)


def pi_powerlaw(h, b=0.1, n=3, m=2, kappa=KAPPA):
    return kappa * ((b / h) ** n - (b / h) ** m)


def dpi_numeric(h, **kw):
    # Central difference of the printed disjoining pressure (independent of
    # the oracle's analytic derivative).
    e = 1e-5 * h
    return (pi_powerlaw(h + e, **kw) - pi_powerlaw(h - e, **kw)) / (2 * e)


# --------------------------------------------------------------------------
# Parameters and linear stability
# --------------------------------------------------------------------------

def test_kappa_and_lsa_values():
    k = O.kappa_from_contact_angle(TH20, 0.1, 3, 2)
    assert abs(k - (1 - math.cos(TH20)) / (0.1 * 0.5)) < 1e-15
    assert abs(k - KAPPA) < 1e-15
    M = pl_model(4, 4, 1.0)
    assert abs(O.dpi(M, 1.0) - dpi_numeric(1.0)) < 1e-9
    qm, sm = O.lsa(M, 1.0)
    f1 = dpi_numeric(1.0)  # h0^3 Pi'(h0) at h0 = 1
    assert abs(qm - math.sqrt(f1 / 2)) < 1e-8
    assert abs(sm - f1 * f1 / 4) < 1e-10


def test_lsa_linear_model_printed_values():
    # Fig. dispersion_curves (a): linear model q_m = 1/sqrt(2), omega_m = 1/4.
    qm, sm = O.lsa(lin_model(4, 4, 1.0), 1.0)
    assert abs(qm - 1 / math.sqrt(2)) < 1e-15
    assert abs(sm - 0.25) < 1e-15


def test_mobility_derivatives_match_finite_differences():
    M = pl_model(4, 4, 1.0)
    for h in (0.15, 0.4, 1.0, 2.5):
        f0, f1, d0, d1 = O.mobility(M, h)
        e = 1e-6 * h
        fp = O.mobility(M, h + e)
        fm = O.mobility(M, h - e)
        assert abs(f0 - h ** 3) < 1e-15 * max(1, h ** 3)
        scale = h ** 2 * KAPPA * max(2 * (0.1 / h) ** 2, 3 * (0.1 / h) ** 3)
        assert abs(f1 - h ** 3 * dpi_numeric(h)) < 1e-7 * scale
        assert abs(d0 - (fp[0] - fm[0]) / (2 * e)) < 1e-7 * abs(d0)
        assert abs(d1 - (fp[1] - fm[1]) / (2 * e)) < 1e-6 * scale / h


# --------------------------------------------------------------------------
# Invariants
# --------------------------------------------------------------------------

def test_flat_film_stays_flat():
    M = pl_model(13, 9, 1.7)
    u = np.full((9, 13), 0.83)
    assert np.all(O.operator_D(M, u) == 0.0)
    out, info = O.step(M, O.Control(), u, 5.0)
    assert info["status"] == 0 and info["iterations"] == 1
    assert np.all(out == u)


@pytest.mark.parametrize("model", ["pl", "lin"])
def test_mass_conserved_after_every_iterate(model):
    nx, ny = 23, 17
    M = pl_model(nx, ny, 1.3) if model == "pl" else lin_model(nx, ny, 1.3, c1=0.7)
    u0 = S.spinodal_film(nx, ny, 1.0, 0.05, seed=7)
    dt = 2.0
    bn = O.explicit_part(M, u0, dt)
    m0 = u0.sum()
    assert abs(bn.sum() - m0) < 1e-13 * m0
    D = O.operator_D(M, u0)
    assert abs(D.sum()) < 1e-14 * np.abs(D).sum()
    uk = u0
    for _ in range(4):
        r = O.newton_iteration(M, uk, bn, dt)
        assert r["status"] == 0
        assert abs(r["unew"].sum() - m0) < 2e-14 * m0
        # The columns of J_x, J_y sum to zero: sum(w) = sum(-G), sum(v) = sum(w).
        assert abs(r["w"].sum() + r["G"].sum()) < 1e-13 * np.abs(r["G"]).sum() + 1e-17
        uk = r["unew"]


def test_mirror_symmetry():
    nx, ny = 19, 11
    M = pl_model(nx, ny, 2.1)
    u = S.spinodal_film(nx, ny, 1.0, 0.05, seed=3)
    a, ia = O.step(M, O.Control(), u, 3.0)
    b, ib = O.step(M, O.Control(), u[:, ::-1].copy(), 3.0)
    assert ia["iterations"] == ib["iterations"]
    assert np.max(np.abs(a[:, ::-1] - b)) < 1e-14
    c, ic = O.step(M, O.Control(), u[::-1, :].copy(), 3.0)
    assert np.max(np.abs(a[::-1, :] - c)) < 1e-14


def test_y_uniform_film_reduces_to_one_dimension():
    nx, ny = 21, 8
    phi = S.spinodal_film(nx, 1, 1.0, 0.05, seed=11)
    u2 = np.repeat(phi, ny, axis=0)
    M2, M1 = pl_model(nx, ny, 1.9), pl_model(nx, 1, 1.9)
    dt = 4.0
    r2 = O.newton_iteration(M2, u2, O.explicit_part(M2, u2, dt), dt)
    r1 = O.newton_iteration(M1, phi, O.explicit_part(M1, phi, dt), dt)
    for j in range(ny):
        assert np.max(np.abs(r2["unew"][j] - r1["unew"][0])) < 1e-15
    # x-uniform film against a single column
    u2t = np.ascontiguousarray(u2.T)
    Mt, Mc = pl_model(ny, nx, 1.9), pl_model(1, nx, 1.9)
    rt = O.newton_iteration(Mt, u2t, O.explicit_part(Mt, u2t, dt), dt)
    col = np.ascontiguousarray(phi.T)
    rc = O.newton_iteration(Mc, col, O.explicit_part(Mc, col, dt), dt)
    for i in range(ny):
        assert np.max(np.abs(rt["unew"][:, i] - rc["unew"][:, 0])) < 1e-15


# --------------------------------------------------------------------------
# Operators against independent constructions
# --------------------------------------------------------------------------

def test_linear_model_operator_is_c0_L2_plus_c1_L():
    nx, ny, ds, c0, c1 = 9, 7, 0.8, 1.3, 0.6
    M = lin_model(nx, ny, ds, c0=c0, c1=c1)
    Lx = neumann_second_difference(nx, ds)
    Ly = neumann_second_difference(ny, ds)
    L = np.kron(np.eye(ny), Lx) + np.kron(Ly, np.eye(nx))
    u = S.spinodal_film(nx, ny, 1.0, 0.3, seed=5)
    ref = (c0 * L @ (L @ u.ravel()) + c1 * L @ u.ravel()).reshape(ny, nx)
    assert np.max(np.abs(O.operator_D(M, u) - ref)) < 1e-12 * np.max(np.abs(ref))
    lap = O.laplacian(M, u)
    assert np.max(np.abs(lap.ravel() - L @ u.ravel())) < 1e-12 * np.max(np.abs(lap))


def test_linear_model_line_bands_closed_form():
    nx, ny, ds, c0, c1, th, dt = 10, 6, 0.9, 1.1, 0.4, 0.5, 0.7
    M = lin_model(nx, ny, ds, c0=c0, c1=c1, theta=th)
    u = S.spinodal_film(nx, ny, 1.0, 0.3, seed=8)
    Lx = neumann_second_difference(nx, ds)
    Ly = neumann_second_difference(ny, ds)
    for j in (0, 3, ny - 1):
        Ax = O.band_to_dense(O.jx_row(M, u, dt, j))
        ref = np.eye(nx) + th * dt * (c0 * Lx @ Lx + c1 * Lx)
        assert np.max(np.abs(Ax - ref)) < 1e-12 * np.max(np.abs(ref))
    for i in (0, 4, nx - 1):
        Ay = O.band_to_dense(O.jy_col(M, u, dt, i))
        ref = np.eye(ny) + th * dt * (c0 * Ly @ Ly + c1 * Ly)
        assert np.max(np.abs(Ay - ref)) < 1e-12 * np.max(np.abs(ref))


def _fd_jacobian(M, u, h=1e-6):
    n = u.size
    J = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = h
        J[:, k] = (O.operator_D(M, (u.ravel() + e).reshape(u.shape)).ravel()
                   - O.operator_D(M, (u.ravel() - e).reshape(u.shape)).ravel()) / (2 * h)
    return J


def test_jacobian_band_equals_fd_jacobian_in_one_dimension():
    # With a single row (or column) there is no mixed term, so the line band
    # is exactly I + theta dt dD/du.
    nx, ds, dt, th = 14, 0.6, 0.37, 0.5
    M = pl_model(nx, 1, ds, theta=th)
    u = S.spinodal_film(nx, 1, 0.7, 0.2, seed=9)
    Jfd = _fd_jacobian(M, u)
    A = O.band_to_dense(O.jx_row(M, u, dt, 0))
    ref = np.eye(nx) + th * dt * Jfd
    assert np.max(np.abs(A - ref)) < 1e-6 * np.max(np.abs(ref - np.eye(nx)))
    Mc = pl_model(1, nx, ds, theta=th)
    uc = np.ascontiguousarray(u.T)
    Jc = _fd_jacobian(Mc, uc)
    Ac = O.band_to_dense(O.jy_col(Mc, uc, dt, 0))
    refc = np.eye(nx) + th * dt * Jc
    assert np.max(np.abs(Ac - refc)) < 1e-6 * np.max(np.abs(refc - np.eye(nx)))


# --------------------------------------------------------------------------
# Pentadiagonal solver against LAPACK
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 17, 64])
def test_penta_solve_matches_dense_lu(n):
    rng = np.random.default_rng(n)
    band = rng.uniform(-1, 1, (n, 5))
    band[:, 2] = 5.0 + rng.uniform(0, 1, n)
    rhs = rng.uniform(-1, 1, n)
    x, s = O.penta_solve(band, rhs)
    assert s == 0
    ref = np.linalg.solve(O.band_to_dense(band), rhs)
    assert np.max(np.abs(x - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


def test_penta_solve_on_real_jacobian_bands():
    nx, ny = 40, 6
    M = pl_model(nx, ny, 0.5)
    u = S.spinodal_film(nx, ny, 1.0, 0.1, seed=2)
    rng = np.random.default_rng(0)
    for dt in (1e-3, 1.0, 100.0):
        band = O.jx_row(M, u, dt, 2)
        rhs = rng.uniform(-1, 1, nx)
        x, s = O.penta_solve(band, rhs)
        ref = np.linalg.solve(O.band_to_dense(band), rhs)
        assert s == 0
        assert np.max(np.abs(x - ref)) < 1e-11 * np.max(np.abs(ref))


def test_penta_zero_pivot_reported():
    band = np.zeros((3, 5))
    band[:, 2] = [0.0, 1.0, 1.0]
    x, s = O.penta_solve(band, np.ones(3))
    assert s == 3


# --------------------------------------------------------------------------
# The converged step against closed forms and a dense Newton solve
# --------------------------------------------------------------------------

def discrete_k2(p, n, ds):
    k = math.pi * p / (n * ds)
    return 4.0 / (ds * ds) * math.sin(k * ds / 2) ** 2


def amplification(lam, dt, th=0.5):
    return (1 - (1 - th) * dt * lam) / (1 + th * dt * lam)


@pytest.mark.parametrize("px,py", [(3, 0), (0, 2), (2, 3)])
def test_linear_model_single_mode_amplification(px, py):
    nx, ny, ds, c0, c1, dt, eps = 24, 20, 0.7, 1.0, 1.0, 0.3, 0.2
    M = lin_model(nx, ny, ds, c0=c0, c1=c1)
    u = S.mode_film(nx, ny, ds, 1.0, eps, px, py)
    k2 = discrete_k2(px, nx, ds) + discrete_k2(py, ny, ds)
    g = amplification(c0 * k2 * k2 - c1 * k2, dt)
    out, info = O.step(M, O.Control(tol=1e-14, max_iter=200), u, dt)
    assert info["status"] == 0
    ref = 1.0 + g * (u - 1.0)
    assert np.max(np.abs(out - ref)) < 1e-13


@pytest.mark.parametrize("eps", [1e-5, 1e-6])
def test_thin_film_small_mode_matches_linear_theory(eps):
    # Linearised about h0, the scheme acts on a mode like the linear model
    # with c0 = f0(h0), c1 = f1(h0): amplification g up to O(eps).
    nx, ny, h0, dt = 32, 24, 1.0, 400.0
    ds = 62.054056935531534 / 8
    M = pl_model(nx, ny, ds)
    px, py = 5, 2
    u = S.mode_film(nx, ny, ds, h0, eps, px, py)
    f0 = h0 ** 3
    f1 = h0 ** 3 * dpi_numeric(h0)
    k2 = discrete_k2(px, nx, ds) + discrete_k2(py, ny, ds)
    g = amplification(f0 * k2 * k2 - f1 * k2, dt)
    out, info = O.step(M, O.Control(tol=1e-13, max_iter=100), u, dt)
    assert info["status"] == 0
    pert = (u - h0) / (h0 * eps)
    got = (out - h0) / (h0 * eps)
    err = np.max(np.abs(got - g * pert))
    assert err < 200 * eps + 1e-7, (err, g)


def test_growth_rate_converges_to_continuum_dispersion():
    # sigma(k) = h0^3 k^2 (Pi'(h0) - k^2): a 1-D film, fine grid, small dt.
    h0 = 1.0
    lam = 62.054056935531534
    nx, ds = 256, lam / 64
    M = pl_model(nx, 1, ds)
    f1 = dpi_numeric(h0)
    for p in (4, 6, 8):  # k below, at and above k_m = 2 pi / lam
        k = math.pi * p / (nx * ds)
        sigma = h0 ** 3 * k * k * (f1 - k * k)
        dt = 0.005 / abs(sigma)
        u = S.mode_film(nx, 1, ds, h0, 1e-7, p, 0)
        out, info = O.step(M, O.Control(tol=1e-14, max_iter=50), u, dt)
        assert info["status"] == 0
        rate = math.log((out[0, 0] - h0) / (u[0, 0] - h0)) / dt
        assert abs(rate - sigma) < 2e-3 * abs(sigma), (p, rate, sigma)


def test_fixed_point_matches_dense_full_newton():
    nx, ny, dt = 6, 5, 3.0
    M = pl_model(nx, ny, 1.1)
    un = S.spinodal_film(nx, ny, 1.0, 0.08, seed=21)
    out, info = O.step(M, O.Control(tol=1e-15, max_iter=400), un, dt)
    bn = O.explicit_part(M, un, dt)
    # Full Newton with a finite-difference Jacobian and dense LAPACK solves.
    u = un.copy()
    for _ in range(30):
        G = O.residual(M, u, bn, dt).ravel()
        J = np.eye(u.size) + M.theta * dt * _fd_jacobian(M, u)
        u = u - np.linalg.solve(J, G).reshape(u.shape)
    assert np.max(np.abs(O.residual(M, u, bn, dt))) < 1e-14
    assert np.max(np.abs(out - u)) < 1e-12


# --------------------------------------------------------------------------
# Convergence orders (Sec. Convergence protocol)
# --------------------------------------------------------------------------

def test_temporal_order_two():
    n, ds, T = 16, 4.0, 2000.0
    M = pl_model(n, n, ds)
    u0 = S.mode_film(n, n, ds, 1.0, 0.1, 2, 1)
    ctl = O.Control(tol=1e-14, max_iter=100)
    sols = []
    for k in range(5):
        nsteps = 4 * 2 ** k
        u = u0.copy()
        for _ in range(nsteps):
            u, info = O.step(M, ctl, u, T / nsteps)
            assert info["status"] == 0
        sols.append(u)
    e = [np.sqrt(np.mean((s - sols[-1]) ** 2)) for s in sols[:-1]]
    orders = [math.log2(e[i] / e[i + 1]) for i in range(len(e) - 1)]
    assert 1.8 < orders[-2] < 2.4, orders


def test_spatial_order_two():
    # Tripled grids keep the coarse cell centres (I_k = 3^k I_0).
    L, T = 48.0, 400.0
    sols = []
    for N in (12, 36, 108):
        ds = L / N
        M = pl_model(N, N, ds)
        u = S.mode_film(N, N, ds, 1.0, 0.1, 1, 1)
        for _ in range(4):
            u, info = O.step(M, O.Control(tol=1e-14, max_iter=100), u, T / 4)
            assert info["status"] == 0
        sols.append(u)
    def coarse(u, f):
        return u[f // 2::f, f // 2::f]
    e0 = np.sqrt(np.mean((sols[0] - coarse(sols[2], 9)) ** 2))
    e1 = np.sqrt(np.mean((sols[1] - coarse(sols[2], 3)) ** 2))
    # With the finest grid as reference, e0/e1 = (9^p - 1)/(3^p - 1)... for p = 2: 10.
    assert 7.0 < e0 / e1 < 14.0, (e0, e1)


# --------------------------------------------------------------------------
# Adaptive time stepping (Fig. FlowChartTime)
# --------------------------------------------------------------------------

def test_controller_shrinks_grows_and_replays():
    n, ds = 16, 3.0
    M = pl_model(n, n, ds)
    u0 = S.spinodal_film(n, n, 1.0, 0.01, seed=4)
    ctl = O.Control(tol=1e-10, max_iter=10, dt_max=50.0, grow_after=2)
    res = O.advance(M, ctl, u0, 0.0, 400.0, 1000.0, 400)
    assert res.status == 0 and res.t == 400.0
    recs = res.records
    assert not recs[0]["accepted"]  # dt0 = 1000 (clipped to 400) is too large
    assert recs[0]["dt"] == 400.0
    for a, b in zip(recs, recs[1:]):
        if not a["accepted"]:
            assert b["dt"] == pytest.approx(a["dt"] * 0.5)
    assert all(r["dt"] <= 1000.0 for r in recs)
    acc = res.accepted()
    assert abs(acc[-1]["t"] + acc[-1]["dt"] - 400.0) < 1e-9
    # replay the accepted sequence (step sizes and iteration counts)
    dts = np.array([r["dt"] for r in acc])
    its = np.array([r["iterations"] for r in acc], dtype=np.int32)
    rep = O.advance(M, ctl, u0, 0.0, 1e30, 1.0, len(acc), dt_replay=dts, iter_replay=its)
    assert np.array_equal(rep.h, res.h)
    assert abs(u0.sum() - res.h.sum()) < 1e-12 * u0.sum()


def test_controller_fails_below_dt_min():
    n = 8
    M = pl_model(n, n, 1.0)
    u0 = S.spinodal_film(n, n, 1.0, 0.3, seed=4)
    ctl = O.Control(tol=1e-16, max_iter=2, dt_min=1e-3)
    res = O.advance(M, ctl, u0, 0.0, 10.0, 1.0, 100)
    assert res.status == 2
    assert not any(r["accepted"] for r in res.records)


def test_nonpositive_height_rejected():
    n = 8
    M = pl_model(n, n, 1.0)
    u0 = np.full((n, n), 1.0)
    u0[3, 4] = 0.0
    out, info = O.step(M, O.Control(), u0, 1.0)
    assert info["status"] in (2, 3)  # non-finite height or pivot: rejected


def test_newton_error_is_max_relative_update():
    # eq. NewtonError: max |v / u_k| over the grid, on a film far from h = 1.
    nx, ny, dt = 12, 10, 2.0
    M = pl_model(nx, ny, 0.4)
    uk = S.spinodal_film(nx, ny, 0.25, 0.05, seed=31)
    r = O.newton_iteration(M, uk, O.explicit_part(M, uk, dt), dt)
    v = r["unew"] - uk
    assert r["err"] == pytest.approx(np.max(np.abs(v) / uk), rel=1e-12)
    assert r["err"] > 3.0 * np.max(np.abs(v))


def test_results_do_not_depend_on_the_thread_count():
    """Every line is one thread's work with the same arithmetic, so one
    thread and all cores give bit-identical steps (the single-thread and
    all-core oracle timings compute the same thing)."""
    M = pl_model(96, 80, 0.05)
    h0 = S.spinodal_film(96, 80, 1.0, 0.01, 7)
    ctl = O.Control(tol=1e-10, max_iter=10)
    n0 = O.num_threads()
    try:
        O.set_num_threads(1)
        assert O.num_threads() == 1
        h1, i1 = O.step(M, ctl, h0, 1e-3)
    finally:
        O.set_num_threads(n0)
    assert O.num_threads() == n0
    hn, i_n = O.step(M, ctl, h0, 1e-3)
    assert i1["iterations"] == i_n["iterations"]
    assert np.array_equal(h1, hn)
