"""Oracle of the discrete adjoint of the unrolled Newton--ADI time step --
TEST INFRASTRUCTURE ONLY (the import rule of ``oracle/`` applies).

The map differentiated is the time step with a fixed number K of Newton
iterations and a fixed dt (Sec. Numerical Method; no convergence test, so
the map is smooth):

    b   = u^n - (1 - theta) dt D(u^n)                  (eq. TrapRule)
    u_0 = u^n
    u_{k+1} = u_k + v_k,  A_y(u_k) v_k = w_k,  A_x(u_k) w_k = -G(u_k),
    G(u) = u + theta dt D(u) - b                        (eqs. JacobianSystem1-3)

with A_x = I + theta dt J_x and A_y = I + theta dt J_y the line operators
of the ADI split (x lines first).  Its adjoint maps a cotangent g of u_K to
J_u^T g (and J_kappa^T g for the strength kappa of Pi).

Method: a plain NumPy restatement of the forward map that accepts complex
values (the discretisation of eq. GovEqnCell2 with the face mobilities and
no-flux walls, the line bands of the direction split, dense solves), and
complex-step differentiation of it: for a real-analytic map F,
Im F(x + i eps e_j) / eps is the j-th column of its Jacobian to rounding
(no subtraction, eps = 1e-30).  The full Jacobian is formed column by column
and transposed, so the oracle shares nothing with a reverse sweep.  A
trajectory of N such steps chains the steps' transposed Jacobians in
reverse order (its pin: the complex-step Jacobian of the whole trajectory).  Only
the power-law and linear models are covered (the maps whose complex
extension is a plain rational function).  Every forward function is pinned
against the C oracle on real inputs; the derivatives against central finite
differences of the C oracle.
"""
from __future__ import annotations

import numpy as np

from . import MODEL_LINEAR, MODEL_POWERLAW, Model

EPS_CS = 1e-30


def mobility(M: Model, h, kappa=None):
    """f0, f1, f0', f1' of Sec. Thin Film Models (f0 = C h^3, f1 = h^3 Pi'),
    elementwise; h (and kappa) may be complex."""
    kap = M.kappa if kappa is None else kappa
    if M.model == MODEL_LINEAR:
        z = np.zeros_like(h)
        return z + M.c0, z + M.c1, z, z
    if M.model != MODEL_POWERLAW:
        raise NotImplementedError("the adjoint oracle covers the power-law and linear models")
    r = M.b / h
    rm, rn = r ** M.m, r ** M.n
    dpi = kap * (M.m * rm - M.n * rn) / h
    d2pi = kap * (M.n * (M.n + 1) * rn - M.m * (M.m + 1) * rm) / (h * h)
    f0 = M.cap_C * h ** 3
    f1 = h ** 3 * dpi
    return f0, f1, 3.0 * M.cap_C * h * h, 3.0 * h * h * dpi + h ** 3 * d2pi


def laplacian(M: Model, u):
    """Five-point Laplacian with even reflection at the walls."""
    s = np.zeros_like(u)
    s[:, :-1] += u[:, 1:] - u[:, :-1]
    s[:, 1:] += u[:, :-1] - u[:, 1:]
    s[:-1, :] += u[1:, :] - u[:-1, :]
    s[1:, :] += u[:-1, :] - u[1:, :]
    return s / (M.ds * M.ds)


def operator_D(M: Model, u, kappa=None):
    """D = [F_x(i+1/2) - F_x(i-1/2) + F_y(j+1/2) - F_y(j-1/2)] / ds with face
    fluxes F = fbar0 dL/ds + fbar1 du/ds, fbar the mean of the two cells'
    mobilities, zero flux through the walls."""
    f0, f1, _, _ = mobility(M, u, kappa)
    L = laplacian(M, u)
    ds = M.ds
    Fx = 0.5 * (f0[:, :-1] + f0[:, 1:]) * (L[:, 1:] - L[:, :-1]) / ds \
        + 0.5 * (f1[:, :-1] + f1[:, 1:]) * (u[:, 1:] - u[:, :-1]) / ds
    Fy = 0.5 * (f0[:-1, :] + f0[1:, :]) * (L[1:, :] - L[:-1, :]) / ds \
        + 0.5 * (f1[:-1, :] + f1[1:, :]) * (u[1:, :] - u[:-1, :]) / ds
    D = np.zeros_like(u)
    D[:, :-1] += Fx
    D[:, 1:] -= Fx
    D[:-1, :] += Fy
    D[1:, :] -= Fy
    return D / ds


def line_matrix(M: Model, u, L, dt, kappa=None):
    """Dense I + theta dt J along one line (u, L: the line's values and full
    Laplacian).  For the face between line cells p and q = p + 1 the flux
    derivative is f0'/2 gL and f1'/2 gU on the two cells (gL, gU the explicit
    differences), plus fbar0 times the along-line third difference and fbar1
    times the first difference; row p gets +dF/ds, row q -dF/ds."""
    n = len(u)
    ds = M.ds
    f0, f1, d0, d1 = mobility(M, u, kappa)
    A = np.eye(n, dtype=np.result_type(u, 1.0 if kappa is None else kappa))
    # along-line second difference with reflection: dLxx_c / du_col
    S = np.zeros((n, n))
    for c in range(n):
        if c + 1 < n:
            S[c, c + 1] += 1.0
            S[c, c] -= 1.0
        if c > 0:
            S[c, c - 1] += 1.0
            S[c, c] -= 1.0
    S /= ds * ds
    for p in range(n - 1):
        q = p + 1
        fb0, fb1 = 0.5 * (f0[p] + f0[q]), 0.5 * (f1[p] + f1[q])
        gL, gU = (L[q] - L[p]) / ds, (u[q] - u[p]) / ds
        dF = fb0 * (S[q] - S[p]) / ds
        dF = dF.astype(A.dtype)
        dF[p] += 0.5 * d0[p] * gL + 0.5 * d1[p] * gU - fb1 / ds
        dF[q] += 0.5 * d0[q] * gL + 0.5 * d1[q] * gU + fb1 / ds
        A[p] += M.theta * dt * dF / ds
        A[q] -= M.theta * dt * dF / ds
    return A


def newton_iteration(M: Model, uk, bn, dt, kappa=None):
    """(w, v, u_{k+1}) of one iteration, x lines then y lines."""
    G = uk + M.theta * dt * operator_D(M, uk, kappa) - bn
    L = laplacian(M, uk)
    w = np.empty_like(G)
    for j in range(uk.shape[0]):
        w[j, :] = np.linalg.solve(line_matrix(M, uk[j, :], L[j, :], dt, kappa), -G[j, :])
    v = np.empty_like(G)
    for i in range(uk.shape[1]):
        v[:, i] = np.linalg.solve(line_matrix(M, uk[:, i], L[:, i], dt, kappa), w[:, i])
    return w, v, uk + v


def step_fixed(M: Model, un, dt, K, kappa=None):
    """u_K of the time step with exactly K Newton iterations."""
    bn = un - (1.0 - M.theta) * dt * operator_D(M, un, kappa)
    u = un
    for _ in range(K):
        _, _, u = newton_iteration(M, u, bn, dt, kappa)
    return u


def jacobian(M: Model, un, dt, K):
    """Full Jacobian d u_K / d u^n, [N, N] (row-major cell order), by complex
    steps, and the column d u_K / d kappa."""
    un = np.asarray(un, dtype=np.float64)
    N = un.size
    J = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[j] = 1j * EPS_CS
        out = step_fixed(M, un + e.reshape(un.shape), dt, K)
        J[:, j] = out.imag.ravel() / EPS_CS
    outk = step_fixed(M, un.astype(np.complex128), dt, K, kappa=M.kappa + 1j * EPS_CS)
    return J, outk.imag.ravel() / EPS_CS


def vjp(M: Model, un, dt, K, g):
    """(g^T d u_K/d u^n reshaped like u^n, g^T d u_K/d kappa)."""
    J, Jk = jacobian(M, un, dt, K)
    g = np.asarray(g, dtype=np.float64).ravel()
    return (J.T @ g).reshape(np.shape(un)), float(Jk @ g)


def trajectory(M: Model, h0, dt, K, nsteps, kappa=None):
    """States u^0 .. u^N of N fixed steps (list of N + 1 grids)."""
    hs = [np.asarray(h0)]
    for _ in range(nsteps):
        hs.append(step_fixed(M, hs[-1], dt, K, kappa))
    return hs


def trajectory_vjp(M: Model, h0, dt, K, nsteps, g):
    """(g^T d u^N/d u^0, g^T d u^N/d kappa) by the chain rule over the steps:
    the cotangent passes through each step's transposed Jacobian in reverse
    order, and the kappa parts of the steps add."""
    hs = trajectory(M, np.asarray(h0, dtype=np.float64), dt, K, nsteps)
    gc = np.asarray(g, dtype=np.float64)
    gk = 0.0
    for n in range(nsteps - 1, -1, -1):
        gc, k = vjp(M, hs[n], dt, K, gc)
        gk += k
    return gc, gk


def trajectory_jacobian(M: Model, h0, dt, K, nsteps):
    """Full Jacobian of u^N with respect to u^0 and the kappa column, by
    complex steps through the whole trajectory (no chain rule)."""
    h0 = np.asarray(h0, dtype=np.float64)
    N = h0.size
    J = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N, dtype=np.complex128)
        e[j] = 1j * EPS_CS
        J[:, j] = trajectory(M, h0 + e.reshape(h0.shape), dt, K, nsteps)[-1].imag.ravel() / EPS_CS
    hk = trajectory(M, h0.astype(np.complex128), dt, K, nsteps, kappa=M.kappa + 1j * EPS_CS)[-1]
    return J, hk.imag.ravel() / EPS_CS


def dkappa_dtheta(theta_c: float, b: float, n: int, m: int) -> float:
    """d kappa / d theta_c for the power-law strength that gives contact
    angle theta_c, kappa = (1 - cos theta_c)/(b M), M = (n - m)/((m - 1)(n - 1)):
    sin theta_c / (b M)."""
    Mf = (n - m) / ((m - 1.0) * (n - 1.0))
    return np.sin(theta_c) / (b * Mf)
