"""Pins of the oracle's two-dimensional line bands and of the disjoining
pressures where the earlier pins are blind.

1. The x-line band (I + theta dt J_x) of a genuinely two-dimensional film,
   entry by entry, against central finite differences of the x-face flux
   divergence in which the transverse part of the Laplacian is held at u_k.
   That frozen part is exactly the neglected mixed term J_xy of eq.
   DirectionSplit, so these differences are J_x as the direction split
   defines it (the y-line band likewise with x and y exchanged).  On a 1-D
   film, or a film uniform across the lines, the along-line and the full
   Laplacian coincide; here they do not, so a band whose
   coefficient-derivative terms used the along-line Laplacian instead of the
   full one fails.  The flux divergence written here is tied to the oracle's
   own D: the x- and y-face parts at u_k must add up to operator_D.
2. Pi_POL against -dpsi/dh of the printed potential psi_POL (eq.
   DisjPressPolymer) at heights where its substrate term (A_SiOx -
   A_Si)/(12 pi (h + d)^2) is not negligible.
3. Pi_NLC at h = 2b and h = 2b + w, where the switch g(h) of eq. mh_model
   takes the values 1/2 and (1 + tanh 1)/2 exactly: a closed form that
   fixes the switch's centre and width.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1806_10550_gb300 import synthetic as S

KAPPA = 1.2061475842818314  # power law, contact angle 20 degrees, b = 0.1


def lap_along_x(u, ds):
    """Second difference along rows, walls by even reflection (a missing
    neighbour is the cell itself and adds nothing)."""
    L = np.zeros_like(u)
    L[:, :-1] += u[:, 1:] - u[:, :-1]
    L[:, 1:] += u[:, :-1] - u[:, 1:]
    return L / ds ** 2


def lap_along_y(u, ds):
    return lap_along_x(u.T, ds).T


def mobility_grid(M, u):
    f0 = np.empty_like(u)
    f1 = np.empty_like(u)
    for idx, h in np.ndenumerate(u):
        f0[idx], f1[idx], _, _ = O.mobility(M, float(h))
    return f0, f1


def x_face_divergence(M, u, L):
    """sum over the two x-faces of each cell of +-F/ds with
    F = fbar0 (L_q - L_p)/ds + fbar1 (u_q - u_p)/ds, fbar the mean of the two
    cell values (Sec. Flux Discretization), no flux through the walls."""
    ds = M.ds
    f0, f1 = mobility_grid(M, u)
    F = (0.5 * (f0[:, :-1] + f0[:, 1:]) * (L[:, 1:] - L[:, :-1]) / ds
         + 0.5 * (f1[:, :-1] + f1[:, 1:]) * (u[:, 1:] - u[:, :-1]) / ds)
    D = np.zeros_like(u)
    D[:, :-1] += F / ds
    D[:, 1:] -= F / ds
    return D


def y_face_divergence(M, u, L):
    Mt = O.Model(**{**M.__dict__, "nx": M.ny, "ny": M.nx})
    return x_face_divergence(Mt, u.T, L.T).T


def fd_x_band(M, uk, dt, j, rel=1e-6):
    """Dense (I + theta dt dDx/du) of row j by central differences, with the
    y part of the Laplacian frozen at u_k."""
    nx = M.nx
    Lyy = lap_along_y(uk, M.ds)
    A = np.eye(nx)
    for i in range(nx):
        e = rel * abs(uk[j, i])
        up = uk.copy()
        um = uk.copy()
        up[j, i] += e
        um[j, i] -= e
        Dp = x_face_divergence(M, up, lap_along_x(up, M.ds) + Lyy)[j]
        Dm = x_face_divergence(M, um, lap_along_x(um, M.ds) + Lyy)[j]
        A[:, i] += M.theta * dt * (Dp - Dm) / (2 * e)
    return A


def transpose_model(M):
    return O.Model(**{**M.__dict__, "nx": M.ny, "ny": M.nx})


MODELS = {
    "powerlaw": dict(make=lambda nx, ny: O.Model(nx=nx, ny=ny, ds=1.0, kappa=KAPPA),
                     h0=1.0, amp=0.2, dt=0.5),
    "nlc": dict(make=lambda nx, ny: O.Model(nx=nx, ny=ny, ds=0.25, model=O.MODEL_NLC,
                                             cap_C=0.0857, b=0.01),
                h0=0.5, amp=0.2, dt=0.05),
    "polymer": dict(make=lambda nx, ny: O.Model(nx=nx, ny=ny, ds=0.5, model=O.MODEL_POLYMER,
                                                 cap_C=0.00581),
                    h0=3.9, amp=0.2, dt=2.0),
}


@pytest.mark.parametrize("shape", [(8, 8), (9, 7)])
@pytest.mark.parametrize("model", sorted(MODELS))
def test_face_divergences_add_up_to_operator_D(model, shape):
    cfg = MODELS[model]
    nx, ny = shape
    M = cfg["make"](nx, ny)
    u = S.spinodal_film(nx, ny, cfg["h0"], cfg["amp"], seed=31 + nx)
    L = O.laplacian(M, u)
    assert np.max(np.abs(lap_along_x(u, M.ds) + lap_along_y(u, M.ds) - L)) <= 1e-13 * np.max(np.abs(L))
    D = x_face_divergence(M, u, L) + y_face_divergence(M, u, L)
    ref = O.operator_D(M, u)
    assert np.max(np.abs(D - ref)) <= 1e-12 * np.max(np.abs(ref))


@pytest.mark.parametrize("shape", [(8, 8), (9, 7)])
@pytest.mark.parametrize("model", sorted(MODELS))
def test_x_band_equals_fd_of_x_faces_with_transverse_laplacian_frozen(model, shape):
    cfg = MODELS[model]
    nx, ny = shape
    M = cfg["make"](nx, ny)
    u = S.spinodal_film(nx, ny, cfg["h0"], cfg["amp"], seed=41 + ny)
    dt = cfg["dt"]
    # the transverse Laplacian really varies across the faces
    Lyy = lap_along_y(u, M.ds)
    assert np.max(np.abs(np.diff(Lyy, axis=1))) > 0.1 * np.max(np.abs(lap_along_x(u, M.ds)))
    for j in range(ny):
        A = O.band_to_dense(O.jx_row(M, u, dt, j))
        ref = fd_x_band(M, u, dt, j)
        scale = np.max(np.abs(ref - np.eye(nx)))
        assert np.max(np.abs(A - ref)) <= 1e-7 * scale, (j, np.max(np.abs(A - ref)), scale)


@pytest.mark.parametrize("shape", [(8, 8), (9, 7)])
@pytest.mark.parametrize("model", sorted(MODELS))
def test_y_band_equals_fd_of_y_faces_with_transverse_laplacian_frozen(model, shape):
    cfg = MODELS[model]
    nx, ny = shape
    M = cfg["make"](nx, ny)
    u = S.spinodal_film(nx, ny, cfg["h0"], cfg["amp"], seed=51 + nx)
    dt = cfg["dt"]
    Mt = transpose_model(M)
    ut = np.ascontiguousarray(u.T)
    for i in range(nx):
        A = O.band_to_dense(O.jy_col(M, u, dt, i))
        ref = fd_x_band(Mt, ut, dt, i)  # column i of u is row i of u^T
        scale = np.max(np.abs(ref - np.eye(ny)))
        assert np.max(np.abs(A - ref)) <= 1e-7 * scale, (i, np.max(np.abs(A - ref)), scale)


# --------------------------------------------------------------------------
# disjoining pressures
# --------------------------------------------------------------------------

def psi_polymer(h, C=1.181, A1=41.25, A2=-243.75, d=191.0):
    """The printed potential of eq. DisjPressPolymer."""
    return C / h ** 8 - A1 / (12 * math.pi * h ** 2) + (A1 - A2) / (12 * math.pi * (h + d) ** 2)


@pytest.mark.parametrize("h", [20.0, 100.0, 300.0])
def test_polymer_pi_is_minus_dpsi_dh(h):
    M = O.Model(nx=4, ny=4, ds=1.0, model=O.MODEL_POLYMER, cap_C=0.00581)
    # fourth-order central difference of the printed potential
    e = 1e-3 * h
    dpsi = (-psi_polymer(h + 2 * e) + 8 * psi_polymer(h + e) - 8 * psi_polymer(h - e)
            + psi_polymer(h - 2 * e)) / (12 * e)
    pi = O.pi_derivs(M, h)[0]
    # the substrate term is far above the tolerance at these heights (0.6% of
    # Pi at h = 20, 28% at 100, more than Pi itself at 300)
    sub = 2 * (41.25 + 243.75) / (12 * math.pi * (h + 191.0) ** 3)
    assert sub > 5e-3 * abs(pi)
    assert abs(pi - (-dpsi)) <= 1e-9 * abs(pi), (h, pi, -dpsi)


@pytest.mark.parametrize("x,g", [(0.0, 0.5), (1.0, 0.5 * (1.0 + math.tanh(1.0)))])
def test_nlc_pi_at_the_switch_centre_and_one_width_above(x, g):
    # eq. mh_model at h = 2b + x w: g = [1 + tanh(x)]/2, so
    # Pi = K[r^3 - r^2] + (N/2) (g h/(h^2 + beta^2))^2 with r = b/h.
    b, w, K, N, beta = 0.01, 0.05, 36.0, 1.67, 1.0
    M = O.Model(nx=4, ny=4, ds=1.0, model=O.MODEL_NLC, cap_C=0.0857, b=b)
    h = 2 * b + x * w
    r = b / h
    ref = K * (r ** 3 - r ** 2) + 0.5 * N * (g * h / (h * h + beta * beta)) ** 2
    pi = O.pi_derivs(M, h)[0]
    assert abs(pi - ref) <= 1e-13 * abs(ref), (pi, ref)
