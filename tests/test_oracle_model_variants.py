"""Pins of the oracle's NLC and polymer disjoining pressures (Sec. Thin Film
Models, eqs. DisjPressNLC, mh_model, NLC_paras, DisjPressPolymer,
Polymer_scales).

Independent of the oracle's own formulas:
- the paper's printed linear-stability values (Fig. dispersion_curves (b),
  (c)) and the printed zero of Pi_NLC (Sec. Nematic Liquid Crystals);
- finite differences of Pi and of the mobilities against the analytic
  derivatives;
- the invariants of the whole time step (mass after every iterate, mirror
  symmetry, the 1-D band against a finite-difference Jacobian) and the
  small-amplitude linear theory, for both models.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so

import oracle as O
from paper_1806_10550_gb300 import synthetic as S

H0_NLC, H0_POL = 0.5, 3.9  # Sec. Validation: initial thickness per model


def nlc(nx, ny, ds, **kw):
    return O.Model(nx=nx, ny=ny, ds=ds, model=O.MODEL_NLC, cap_C=0.0857, b=0.01, **kw)


def pol(nx, ny, ds, **kw):
    return O.Model(nx=nx, ny=ny, ds=ds, model=O.MODEL_POLYMER, cap_C=0.00581, **kw)


def test_nlc_printed_lsa_values():
    # Fig. dispersion_curves (b): q_m ~ 1.482, omega_m ~ 0.05169 at H0 = 0.5
    qm, wm = O.lsa(nlc(4, 4, 1.0), H0_NLC)
    assert abs(qm - 1.482) < 5e-4
    assert abs(wm - 0.05169) < 5e-6


def test_polymer_printed_growth_rate():
    # Fig. dispersion_curves (c): omega_m ~ 2.040 at H0 = 3.9.  For any Pi the
    # LSA relations give q_m^4 = omega_m / f0(H0), and the printed parameters
    # give f0(H0) = C H0^3 = 0.3446; the printed omega_m then fixes
    # q_m = 1.5598, so the printed q_m (1.600) is read as a misprint.
    qm, wm = O.lsa(pol(4, 4, 1.0), H0_POL)
    assert abs(wm - 2.040) < 5e-4
    f0 = 0.00581 * H0_POL ** 3
    assert abs(qm - (2.040 / f0) ** 0.25) < 1e-4


def test_nlc_pi_zero_thickness():
    # Sec. Nematic Liquid Crystals: Pi_NLC vanishes at H0 ~ 0.2624
    M = nlc(4, 4, 1.0)
    root = so.brentq(lambda h: O.pi_derivs(M, h)[0], 0.1, 0.4, xtol=1e-14)
    assert abs(root - 0.2624) < 5e-5


@pytest.mark.parametrize("which,hs", [
    ("nlc", (0.012, 0.02, 0.05, 0.1, 0.2624, 0.5, 1.0, 2.0)),
    ("pol", (1.0, 2.0, 3.9, 8.0, 50.0, 300.0)),
])
def test_pi_derivatives_match_finite_differences(which, hs):
    M = nlc(4, 4, 1.0) if which == "nlc" else pol(4, 4, 1.0)
    for h in hs:
        p, d1, d2 = O.pi_derivs(M, h)
        e = 1e-5 * h
        pp, d1p, _ = O.pi_derivs(M, h + e)
        pm, d1m, _ = O.pi_derivs(M, h - e)
        fd1 = (pp - pm) / (2 * e)
        fd2 = (d1p - d1m) / (2 * e)
        assert abs(d1 - fd1) <= 1e-7 * max(abs(d1), abs(p) / h, 1e-300), (h, d1, fd1)
        assert abs(d2 - fd2) <= 1e-7 * max(abs(d2), abs(d1) / h, 1e-300), (h, d2, fd2)


@pytest.mark.parametrize("which", ["nlc", "pol"])
def test_mobility_is_c_h3_and_h3_dpi_with_derivatives(which):
    M = nlc(4, 4, 1.0) if which == "nlc" else pol(4, 4, 1.0)
    for h in ((0.05, 0.3, 0.5, 1.2) if which == "nlc" else (2.0, 3.9, 6.0)):
        f0, f1, d0, d1 = O.mobility(M, h)
        _, dpi, _ = O.pi_derivs(M, h)
        assert abs(f0 - M.cap_C * h ** 3) < 1e-15 * f0
        assert abs(f1 - h ** 3 * dpi) < 1e-14 * abs(f1)
        e = 1e-6 * h
        fp, fm = O.mobility(M, h + e), O.mobility(M, h - e)
        assert abs(d0 - (fp[0] - fm[0]) / (2 * e)) < 1e-7 * abs(d0)
        assert abs(d1 - (fp[1] - fm[1]) / (2 * e)) < 1e-6 * max(abs(d1), abs(f1) / h)


def _case(which):
    if which == "nlc":
        lam = 2 * math.pi / O.lsa(nlc(4, 4, 1.0), H0_NLC)[0]
        return nlc, H0_NLC, lam, 0.05
    lam = 2 * math.pi / O.lsa(pol(4, 4, 1.0), H0_POL)[0]
    return pol, H0_POL, lam, 0.05


@pytest.mark.parametrize("which", ["nlc", "pol"])
def test_mass_conserved_after_every_iterate(which):
    mk, h0, lam, eps = _case(which)
    nx, ny = 23, 17
    M = mk(nx, ny, lam / 6)
    wm = O.lsa(M, h0)[1]
    u0 = S.spinodal_film(nx, ny, h0, eps, seed=7)
    dt = 0.2 / wm
    bn = O.explicit_part(M, u0, dt)
    m0 = u0.sum()
    assert abs(bn.sum() - m0) < 1e-13 * m0
    uk = u0
    for _ in range(4):
        r = O.newton_iteration(M, uk, bn, dt)
        assert r["status"] == 0
        assert abs(r["unew"].sum() - m0) < 2e-14 * m0
        assert abs(r["w"].sum() + r["G"].sum()) < 1e-13 * np.abs(r["G"]).sum() + 1e-17
        uk = r["unew"]


@pytest.mark.parametrize("which", ["nlc", "pol"])
def test_mirror_symmetry(which):
    mk, h0, lam, eps = _case(which)
    nx, ny = 19, 11
    M = mk(nx, ny, lam / 5)
    dt = 0.005 / O.lsa(M, h0)[1]  # the coarse grid (5 cells per wavelength) is stiff
    u = S.spinodal_film(nx, ny, h0, eps, seed=3)
    a, ia = O.step(M, O.Control(), u, dt)
    assert ia["status"] == 0
    b, ib = O.step(M, O.Control(), u[:, ::-1].copy(), dt)
    assert ia["iterations"] == ib["iterations"]
    assert np.max(np.abs(a[:, ::-1] - b)) < 1e-14 * h0
    c, _ = O.step(M, O.Control(), u[::-1, :].copy(), dt)
    assert np.max(np.abs(a[::-1, :] - c)) < 1e-14 * h0


def _fd_jacobian(M, u):
    n = u.size
    J = np.zeros((n, n))
    base = u.ravel()
    for k in range(n):
        e = 1e-6 * max(1.0, abs(base[k]))
        up, um = base.copy(), base.copy()
        up[k] += e
        um[k] -= e
        J[:, k] = (O.operator_D(M, up.reshape(u.shape)) - O.operator_D(M, um.reshape(u.shape))).ravel() / (2 * e)
    return J


@pytest.mark.parametrize("which", ["nlc", "pol"])
def test_jacobian_band_equals_fd_jacobian_in_one_dimension(which):
    mk, h0, lam, eps = _case(which)
    nx = 14
    M = mk(nx, 1, lam / 6)
    dt = 0.1 / O.lsa(M, h0)[1]
    u = S.spinodal_film(nx, 1, h0, 0.2, seed=9)
    A = O.band_to_dense(O.jx_row(M, u, dt, 0))
    ref = np.eye(nx) + 0.5 * dt * _fd_jacobian(M, u)
    assert np.max(np.abs(A - ref)) < 1e-6 * np.max(np.abs(ref - np.eye(nx)))


def _discrete_k2(p, n, ds):
    k = math.pi * p / (n * ds)
    return (4 / ds ** 2) * math.sin(k * ds / 2) ** 2


@pytest.mark.parametrize("which", ["nlc", "pol"])
def test_small_mode_matches_linear_theory(which):
    # About a flat film h0 the scheme acts on a single cosine mode like the
    # linear model with c0 = f0(h0), c1 = f1(h0) (Sec. Linear Stability
    # Analysis), up to O(eps).
    mk, h0, lam, _ = _case(which)
    nx, ny, eps = 32, 24, 1e-6
    ds = lam / 8
    M = mk(nx, ny, ds)
    f0, f1, _, _ = O.mobility(M, h0)
    px, py = 5, 2
    k2 = _discrete_k2(px, nx, ds) + _discrete_k2(py, ny, ds)
    lam_k = f0 * k2 * k2 - f1 * k2
    dt = 0.2 / O.lsa(M, h0)[1]
    g = (1 - 0.5 * dt * lam_k) / (1 + 0.5 * dt * lam_k)
    u = S.mode_film(nx, ny, ds, h0, eps, px, py)
    out, info = O.step(M, O.Control(tol=1e-13, max_iter=100), u, dt)
    assert info["status"] == 0
    pert = (u - h0) / (h0 * eps)
    got = (out - h0) / (h0 * eps)
    assert np.max(np.abs(got - g * pert)) < 200 * eps + 1e-7
