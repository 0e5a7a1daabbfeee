"""Oracle of the radial Fourier analysis of a film (App. Radial Fourier
Transform) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this module; the CUDA library never calls it.

Plain FP64 NumPy/SciPy, one function per step of the appendix, in its
order.  Where the appendix leaves a choice open, the reading taken is stated
at the step (the same readings bind the CUDA path):

1. zeta = h - H0 (the appendix removes the zero-wavenumber peak by
   subtracting the initial thickness).  Transform: the films have no-flux
   walls, so the transform taken is that of the film reflected evenly about
   its walls (a 2nx x 2ny periodic film).  Its magnitude at wave index
   (p, q), normalised by the reflected film's size, is
       A[q, p] = |C[q, p]| / (nx ny),
       C[q, p] = sum_j sum_i zeta[j, i] cos(pi p (2i+1) / (2 nx))
                                        cos(pi q (2j+1) / (2 ny)),
   the 2-D DCT-II sum; wave vector (pi p / Lx, pi q / Ly), L = n ds.  A
   single cosine mode eps cos(pi p x / Lx) cos(pi q y / Ly) with p, q > 0
   gives A = eps / 4 (its four mirror images share the power).
2. Gaussian smoothing of A in the (p, q) index plane: weights
   exp(-d^2 / (2 sigma^2)) for |d| <= R = ceil(3 sigma), normalised to sum
   1, applied along p and then along q.  Outside 0 <= k < n the spectrum of
   the reflected film continues (period 2n): index -k is k, index n is 0,
   index n + k is n - k.  sigma = 0 leaves A unchanged.
3.-4. Radial map: points with equal |wave vector| form one radial point
   (eq. FFT_radial_averaging).  Equality is decided exactly on the integer
   key (p ny/g)^2 + (q nx/g)^2, g = gcd(nx, ny), for which
   |q| = pi g sqrt(key) / (ds nx ny).  The value is the mean of the
   smoothed magnitude over the group.  Only |q| <= q_cut enters (the
   appendix restricts to [0, 5 q_m]); the cut is the integer test
   key <= floor((q_cut / scale)^2), scale = pi g / (ds nx ny).
5. Continuous piecewise-linear least-squares fit (eq. PiecewiseFunction):
   nodes t_0 = 0, t_j = |q| of radial point j * ppi (j = 1..K-1) and
   t_K = q_cut, with K = max(1, ceil((M - 1) / ppi)) for M radial points:
   every interval but the last holds ppi points and the last holds the
   remaining 2..ppi+1 (a last interval holding only its left node would
   leave its slope undetermined).  Node values a_0 = 0, a_1..a_K free (K
   unknowns, as the appendix counts).
6. The fit sampled at n_eval equispaced points of [0, q_cut] and smoothed
   by moving averages of half-widths 3, 2 and 1 in turn; at the ends the
   window is cut to the samples that exist.
7. Critical points: derivative by second-order differences (central
   inside, one-sided second-order at the ends); a root lies in
   [q_e, q_e+1) where the derivative is zero at q_e or changes sign, and
   is placed by linear interpolation (what bisection on the sampled
   derivative converges to).  The second derivative (the same differences
   applied to the derivative), interpolated to the root, is negative at a
   local maximum.  Maxima are listed by value, highest first; the first is
   the dominant wavenumber.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

PAPER_POINTS_PER_INTERVAL = 10
PAPER_EVAL_POINTS = 400
PAPER_HALF_WIDTHS = (3, 2, 1)


# ---- step 1: magnitude of the transform of the evenly reflected film -------
def cos_matrix(n_out: int, n: int) -> np.ndarray:
    """[n_out, n] with entry cos(pi k (2i+1) / (2n)); the integer k(2i+1) is
    reduced modulo 4n before scaling so the argument stays in [0, 2 pi)."""
    k = np.arange(n_out, dtype=np.int64)[:, None]
    i = np.arange(n, dtype=np.int64)[None, :]
    m = (k * (2 * i + 1)) % (4 * n)
    return np.cos(np.pi * m.astype(np.float64) / (2.0 * n))


def amplitude(h: np.ndarray, H0: float, n_p: int | None = None, n_q: int | None = None) -> np.ndarray:
    """A[q, p] = |C[q, p]| / (nx ny) for p < n_p, q < n_q (step 1)."""
    h = np.asarray(h, dtype=np.float64)
    ny, nx = h.shape
    n_p = nx if n_p is None else n_p
    n_q = ny if n_q is None else n_q
    zeta = h - H0
    C = cos_matrix(n_q, ny) @ zeta @ cos_matrix(n_p, nx).T
    return np.abs(C) / (nx * ny)


# ---- step 2: Gaussian smoothing --------------------------------------------
def gaussian_weights(sigma: float) -> np.ndarray:
    if sigma <= 0:
        return np.ones(1)
    R = int(math.ceil(3.0 * sigma))
    d = np.arange(-R, R + 1, dtype=np.float64)
    w = np.exp(-d * d / (2.0 * sigma * sigma))
    return w / w.sum()


def fold(k: int, n: int):
    """Index of the reflected film's spectrum: (index in [0, n), True) or
    (None, False) where the spectrum is zero (index n modulo 2n)."""
    m = k % (2 * n)
    if m < n:
        return m, True
    if m == n:
        return None, False
    return 2 * n - m, True


def smooth(A: np.ndarray, nx: int, ny: int, n_p: int, n_q: int, sigma: float) -> np.ndarray:
    """Smoothed block S[q, p], q < n_q, p < n_p (step 2).  A must hold every
    index the windows reach after folding: p < min(nx, n_p + R) and
    q < min(ny, n_q + R)."""
    w = gaussian_weights(sigma)
    R = (len(w) - 1) // 2
    qb = A.shape[0]
    T = np.zeros((qb, n_p))
    for p in range(n_p):
        for d in range(-R, R + 1):
            k, ok = fold(p + d, nx)
            if ok:
                T[:, p] += w[d + R] * A[:, k]
    S = np.zeros((n_q, n_p))
    for q in range(n_q):
        for d in range(-R, R + 1):
            k, ok = fold(q + d, ny)
            if ok:
                S[q, :] += w[d + R] * T[k, :]
    return S


# ---- steps 3-4: radial average ----------------------------------------------
def radial_geometry(nx: int, ny: int, ds: float, q_cut: float):
    """(ax, ay, scale, keycut, n_p, n_q): key = (p ax)^2 + (q ay)^2,
    |q| = scale sqrt(key), keys <= keycut enter, p < n_p and q < n_q hold
    every such point."""
    g = math.gcd(nx, ny)
    ax, ay = ny // g, nx // g
    scale = math.pi * g / (ds * nx * ny)
    r = q_cut / scale
    keycut = int(math.floor(r * r))
    root = math.isqrt(keycut)
    n_p = min(nx, root // ax + 1)
    n_q = min(ny, root // ay + 1)
    return ax, ay, scale, keycut, n_p, n_q


def radial_profile(S: np.ndarray, nx: int, ny: int, ds: float, q_cut: float):
    """(q_r, mean, count, key) over the distinct |q| <= q_cut, ascending."""
    ax, ay, scale, keycut, n_p, n_q = radial_geometry(nx, ny, ds, q_cut)
    q = np.arange(n_q, dtype=np.int64)[:, None]
    p = np.arange(n_p, dtype=np.int64)[None, :]
    key = (p * ax) ** 2 + (q * ay) ** 2
    sel = key <= keycut
    keys, inv = np.unique(key[sel], return_inverse=True)
    cnt = np.bincount(inv)
    tot = np.bincount(inv, weights=S[:n_q, :n_p][sel])
    return scale * np.sqrt(keys.astype(np.float64)), tot / cnt, cnt, keys


# ---- step 5: piecewise-linear least squares ----------------------------------
def fit_nodes(q_r: np.ndarray, q_cut: float, ppi: int) -> np.ndarray:
    M = len(q_r)
    if M < 2:
        raise ValueError("the fit needs at least two radial points")
    K = max(1, -(-(M - 1) // ppi))
    t = np.empty(K + 1)
    t[0] = 0.0
    for j in range(1, K):
        t[j] = q_r[j * ppi]
    t[K] = q_cut
    return t


def design_matrix(q_r: np.ndarray, t: np.ndarray, ppi: int):
    """Sparse [M, K]: column j-1 is the hat function of node j (j = 1..K)
    evaluated at the radial points; point i lies in interval
    min(i // ppi, K - 1)."""
    M, K = len(q_r), len(t) - 1
    rows, cols, vals = [], [], []
    for i in range(M):
        j = min(i // ppi, K - 1)
        s = (q_r[i] - t[j]) / (t[j + 1] - t[j])
        if j >= 1:
            rows.append(i), cols.append(j - 1), vals.append(1.0 - s)
        rows.append(i), cols.append(j), vals.append(s)
    return sp.csr_matrix((vals, (rows, cols)), shape=(M, K))


def fit(q_r: np.ndarray, y: np.ndarray, q_cut: float, ppi: int = PAPER_POINTS_PER_INTERVAL):
    """Nodes t_0..t_K and values a_0 = 0, a_1..a_K minimising
    sum_i (f(q_i) - y_i)^2 (normal equations, sparse direct solve)."""
    t = fit_nodes(q_r, q_cut, ppi)
    A = design_matrix(q_r, t, ppi)
    N = (A.T @ A).tocsc()
    a = np.zeros(len(t))
    a[1:] = spla.spsolve(N, A.T @ y)
    return t, a


# ---- step 6: sampling and moving averages -----------------------------------
def moving_average(y: np.ndarray, P: int) -> np.ndarray:
    n = len(y)
    out = np.empty(n)
    for e in range(n):
        lo, hi = max(0, e - P), min(n - 1, e + P)
        out[e] = y[lo:hi + 1].sum() / (hi - lo + 1)
    return out


def sample_and_smooth(t: np.ndarray, a: np.ndarray, q_cut: float,
                      n_eval: int = PAPER_EVAL_POINTS, half_widths=PAPER_HALF_WIDTHS):
    qe = q_cut * np.arange(n_eval) / (n_eval - 1)
    y = np.interp(qe, t, a)
    for P in half_widths:
        y = moving_average(y, P)
    return qe, y


# ---- step 7: critical points -----------------------------------------------
def derivative(y: np.ndarray, dq: float) -> np.ndarray:
    return np.gradient(y, dq, edge_order=2)


def local_maxima(qe: np.ndarray, y: np.ndarray):
    """[(q, value)] of the local maxima, highest value first."""
    dq = qe[1] - qe[0]
    d = derivative(y, dq)
    s = derivative(d, dq)
    n = len(y)
    out = []
    for e in range(n):
        if d[e] == 0.0:
            f = 0.0
        elif e + 1 < n and ((d[e] > 0 and d[e + 1] < 0) or (d[e] < 0 and d[e + 1] > 0)):
            f = d[e] / (d[e] - d[e + 1])
        else:
            continue
        e1 = min(e + 1, n - 1)
        s_root = s[e] + f * (s[e1] - s[e])
        if s_root < 0:
            out.append((qe[e] + f * (qe[e1] - qe[e]), y[e] + f * (y[e1] - y[e])))
    out.sort(key=lambda r: (-r[1], r[0]))
    return out


# ---- the whole analysis -----------------------------------------------------
def analyse(h: np.ndarray, ds: float, H0: float, q_cut: float, sigma: float = 1.0,
            ppi: int = PAPER_POINTS_PER_INTERVAL, n_eval: int = PAPER_EVAL_POINTS) -> dict:
    h = np.asarray(h, dtype=np.float64)
    ny, nx = h.shape
    _, _, _, _, n_p, n_q = radial_geometry(nx, ny, ds, q_cut)
    R = (len(gaussian_weights(sigma)) - 1) // 2
    A = amplitude(h, H0, min(nx, n_p + R), min(ny, n_q + R))
    S = smooth(A, nx, ny, n_p, n_q, sigma)
    q_r, y, cnt, keys = radial_profile(S, nx, ny, ds, q_cut)
    t, a = fit(q_r, y, q_cut, ppi)
    qe, ye = sample_and_smooth(t, a, q_cut, n_eval)
    peaks = local_maxima(qe, ye)
    return dict(amplitude=A[:n_q, :n_p], smoothed=S, radial_q=q_r, radial_value=y,
                radial_count=cnt, radial_key=keys, node_q=t, node_value=a,
                curve_q=qe, curve_value=ye, peaks=peaks,
                q_dominant=peaks[0][0] if peaks else 0.0,
                value_dominant=peaks[0][1] if peaks else 0.0)
