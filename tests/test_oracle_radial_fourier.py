"""Pins of the radial Fourier analysis oracle (App. Radial Fourier Transform).

Each step is checked against something other than itself:
- step 1: closed-form amplitudes of single cosine modes, and the magnitude of
  NumPy's FFT of the explicitly reflected film (another route to the same
  transform);
- step 2: a delta smoothed against the Gaussian written out on the full
  periodic spectrum of the reflected film;
- steps 3-4: the grouping against lattice points grouped by floating |q|
  with a tolerance, and known sums of two squares;
- step 5: exact recovery of a function in the fit's own space, and a dense
  least-squares solve (numpy lstsq) of an explicitly built design matrix;
- steps 6-7: moving averages of constants and ramps, maxima of parabolas
  and cosines placed in closed form;
- the whole chain: a film built from linear spinodal growth (each cosine
  mode amplified by exp(sigma(k) t), sigma(k) = h0^3 k^2 (Pi'(h0) - k^2))
  has its dominant wavenumber at the linear-stability q_m (Sec. Linear
  Stability Analysis, used this way in Sec. Results).
"""
import math

import numpy as np
import pytest

from oracle import radial_fourier as RF
from paper_1806_10550_gb300 import synthetic as S


# ---- step 1 ------------------------------------------------------------------
@pytest.mark.parametrize("nx,ny", [(16, 16), (24, 10), (7, 13)])
def test_single_modes_have_closed_form_amplitudes(nx, ny):
    ds, h0, eps = 0.9, 1.3, 0.02
    for px, py, expect in [(3, 2, h0 * eps / 4), (4, 0, h0 * eps / 2), (0, 5, h0 * eps / 2)]:
        if px >= nx or py >= ny:
            continue
        h = S.mode_film(nx, ny, ds, h0, eps, px, py)
        A = RF.amplitude(h, h0)
        assert abs(A[py, px] - expect) < 1e-15
        A[py, px] = 0.0
        assert np.max(A) < 1e-15
    A = RF.amplitude(np.full((ny, nx), 1.25), 1.0)  # an offset sits at the origin
    assert abs(A[0, 0] - 0.25) < 1e-15 and np.max(A[1:, :]) < 1e-15 and np.max(A[:, 1:]) < 1e-15


def _reflected(z):
    """The film mirrored about its right and top walls: [2ny, 2nx]."""
    zx = np.concatenate([z, z[:, ::-1]], axis=1)
    return np.concatenate([zx, zx[::-1, :]], axis=0)


@pytest.mark.parametrize("nx,ny", [(12, 20), (32, 32), (5, 3)])
def test_amplitude_is_fft_magnitude_of_reflected_film(nx, ny):
    rng = np.random.default_rng(nx * 7 + ny)
    h = 1.0 + 0.05 * rng.uniform(-1, 1, (ny, nx))
    F = np.abs(np.fft.fft2(_reflected(h - 1.0))) / (4 * nx * ny)
    A = RF.amplitude(h, 1.0)
    assert np.max(np.abs(A - F[:ny, :nx])) < 1e-15 * nx * ny


# ---- step 2 ------------------------------------------------------------------
@pytest.mark.parametrize("p0,q0,sigma", [(10, 9, 1.0), (1, 0, 1.5), (0, 2, 2.0), (15, 14, 1.0), (3, 3, 0.0)])
def test_smoothing_of_a_delta_matches_periodic_convolution(p0, q0, sigma):
    nx, ny = 16, 18
    A = np.zeros((ny, nx))
    A[q0, p0] = 1.0
    # full spectrum of the reflected film: period 2n, even, zero at index n
    full = np.zeros((2 * ny, 2 * nx))
    for q in range(2 * ny):
        for p in range(2 * nx):
            qq = q if q < ny else (None if q == ny else 2 * ny - q)
            pp = p if p < nx else (None if p == nx else 2 * nx - p)
            if qq is not None and pp is not None:
                full[q, p] = A[qq, pp]
    w = RF.gaussian_weights(sigma)
    R = (len(w) - 1) // 2
    ref = np.zeros((ny, nx))
    for q in range(ny):
        for p in range(nx):
            acc = 0.0
            for dq in range(-R, R + 1):
                for dp in range(-R, R + 1):
                    acc += w[dq + R] * w[dp + R] * full[(q + dq) % (2 * ny), (p + dp) % (2 * nx)]
            ref[q, p] = acc
    got = RF.smooth(A, nx, ny, nx, ny, sigma)
    assert np.max(np.abs(got - ref)) < 1e-15
    if sigma > 0:
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs(w[R + 1] / w[R] - math.exp(-0.5 / sigma ** 2)) < 1e-14


# ---- steps 3-4 -----------------------------------------------------------------
@pytest.mark.parametrize("nx,ny,ds", [(32, 32, 1.0), (64, 16, 0.5), (12, 18, 2.0)])
def test_radial_groups_equal_lattice_distances(nx, ny, ds):
    q_cut = 0.8 * math.pi / ds
    rng = np.random.default_rng(5)
    Sm = rng.uniform(0, 1, (ny, nx))
    q_r, mean, cnt, keys = RF.radial_profile(Sm, nx, ny, ds, q_cut)
    # brute force: |q| of every lattice point in floating point, grouped with a tolerance
    pts = sorted((math.hypot(math.pi * p / (nx * ds), math.pi * q / (ny * ds)), Sm[q, p])
                 for q in range(ny) for p in range(nx))
    pts = [r for r in pts if r[0] <= q_cut * (1 + 1e-12)]
    groups = []
    for r, v in pts:
        if groups and abs(r - groups[-1][0]) <= 1e-12 * max(r, 1.0):
            groups[-1][1].append(v)
        else:
            groups.append((r, [v]))
    assert len(groups) == len(q_r)
    for (r, vs), qq, m, c in zip(groups, q_r, mean, cnt):
        assert abs(r - qq) <= 1e-13 * max(r, 1.0)
        assert c == len(vs)
        assert abs(m - sum(vs) / len(vs)) < 1e-15


def test_radial_counts_of_sums_of_two_squares():
    n = 64
    q_cut = math.pi * 25.5 / n  # radius 25.5 in wave-index units
    q_r, _, cnt, keys = RF.radial_profile(np.ones((n, n)), n, n, 1.0, q_cut)
    d = dict(zip(keys.tolist(), cnt.tolist()))
    # non-negative (p, q) with p^2 + q^2 = key
    assert d[0] == 1 and d[1] == 2 and d[2] == 1 and d[25] == 4 and d[50] == 3
    assert d[625] == 6  # (0,25), (7,24), (15,20) and their mirrors
    assert 3 not in d and 7 not in d and 21 not in d


# ---- step 5 ------------------------------------------------------------------
def test_fit_recovers_a_function_in_its_space():
    rng = np.random.default_rng(1)
    q_r = np.concatenate([[0.0], np.sort(rng.uniform(0.01, 3.9, 57))])
    q_cut = 4.0
    t = RF.fit_nodes(q_r, q_cut, 10)
    a_true = np.concatenate([[0.0], rng.uniform(-1, 1, len(t) - 1)])
    y = np.interp(q_r, t, a_true)
    t2, a = RF.fit(q_r, y, q_cut, 10)
    assert np.array_equal(t, t2)
    assert np.max(np.abs(a - a_true)) < 1e-12
    # interval sizes: 10 points each, the last 2..11
    K = len(t) - 1
    assert K == math.ceil((len(q_r) - 1) / 10)


@pytest.mark.parametrize("M,ppi", [(2, 10), (11, 10), (12, 10), (57, 10), (40, 3), (9, 1)])
def test_fit_equals_dense_least_squares(M, ppi):
    rng = np.random.default_rng(M * 31 + ppi)
    q_r = np.concatenate([[0.0], np.sort(rng.uniform(0.05, 1.9, M - 1))])
    y = rng.uniform(0, 1, M)
    q_cut = 2.0
    t, a = RF.fit(q_r, y, q_cut, ppi)
    K = len(t) - 1
    # dense design matrix from the hat functions written out directly
    D = np.zeros((M, K))
    for i in range(M):
        for j in range(1, K + 1):
            lo, mid = t[j - 1], t[j]
            hi = t[j + 1] if j < K else None
            x = q_r[i]
            if lo <= x <= mid and mid > lo:
                D[i, j - 1] = (x - lo) / (mid - lo)
            elif hi is not None and mid < x < hi:
                D[i, j - 1] = (hi - x) / (hi - mid)
    ref = np.linalg.lstsq(D, y, rcond=None)[0]
    assert np.max(np.abs(a[1:] - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))
    assert a[0] == 0.0


def test_fit_needs_two_points():
    with pytest.raises(ValueError):
        RF.fit(np.array([0.0]), np.array([1.0]), 1.0, 10)


# ---- steps 6-7 ---------------------------------------------------------------
def test_moving_average_constants_ramps_and_ends():
    y = np.full(50, 2.5)
    assert np.max(np.abs(RF.moving_average(y, 3) - 2.5)) < 1e-15
    r = np.arange(50, dtype=np.float64)
    m = RF.moving_average(r, 3)
    assert np.max(np.abs(m[3:-3] - r[3:-3])) < 1e-13
    assert abs(m[0] - 1.5) < 1e-15 and abs(m[-1] - 47.5) < 1e-13  # windows cut at the ends


@pytest.mark.parametrize("q0", [0.3, 1.17, 2.0])
def test_parabola_maximum_is_exact(q0):
    qe = 3.0 * np.arange(400) / 399
    y = 5.0 - (qe - q0) ** 2
    peaks = RF.local_maxima(qe, y)
    assert len(peaks) == 1
    assert abs(peaks[0][0] - q0) < 1e-12
    assert abs(peaks[0][1] - 5.0) < 0.5 * (qe[1] - qe[0]) ** 2 + 1e-12


def test_cosine_maxima_in_order():
    qe = 10.0 * np.arange(400) / 399
    y = np.cos(qe) * np.exp(-0.1 * qe)  # maxima at tan(q) = -0.1, q = 2 pi k - atan(0.1)
    peaks = RF.local_maxima(qe, y)
    expect = [2 * math.pi * k - math.atan(0.1) for k in (1,)]
    assert len(peaks) == 1  # q = 0 is a boundary, not a root of the derivative
    assert abs(peaks[0][0] - expect[0]) < 2e-4


# ---- the whole chain ---------------------------------------------------------
def test_linear_spinodal_film_peaks_at_qm():
    # power-law model of the 8192^2 workloads, theta_c = 20 deg, b = 0.1: q_m from the
    # linear theory, 16 lambda_m square at lambda_m / 16 spacing
    b, theta = 0.1, math.radians(20.0)
    kappa = (1 - math.cos(theta)) / (b * 0.5)
    dpi = kappa * (2 * b ** 2 - 3 * b ** 3)  # Pi'(1) = kappa (m b^m - n b^n), n=3, m=2
    qm = math.sqrt(dpi / 2)
    lam = 2 * math.pi / qm
    n, ds = 256, lam / 16
    rng = np.random.default_rng(11)
    noise = rng.uniform(-1, 1, (n, n))
    # amplify each cosine mode of the noise by exp(sigma(k) t), sigma_max t = 6
    C = RF.cos_matrix(n, n) @ noise @ RF.cos_matrix(n, n).T
    k = np.pi * np.arange(n) / (n * ds)
    kk = k[None, :] ** 2 + k[:, None] ** 2
    sig = kk * (dpi - kk)
    smax = dpi ** 2 / 4
    C *= np.exp(sig / smax * 6.0)
    # back to the film (inverse of the cosine sums: orthogonality weights 2/n, 1/n at k = 0)
    wv = np.full(n, 2.0 / n)
    wv[0] = 1.0 / n
    zeta = RF.cos_matrix(n, n).T @ (C * wv[:, None] * wv[None, :]) @ RF.cos_matrix(n, n)
    h = 1.0 + 1e-6 * zeta / np.max(np.abs(zeta))
    r = RF.analyse(h, ds, 1.0, 5 * qm)
    assert abs(r["q_dominant"] - qm) < 0.05 * qm
    assert len(r["radial_q"]) == len(r["radial_value"]) and r["node_value"][0] == 0.0


def test_derivative_is_second_order_to_the_ends():
    # second-order differences (one-sided at the ends) differentiate quadratics exactly
    qe = 2.0 * np.arange(40) / 39
    dq = qe[1] - qe[0]
    y = 3.0 * qe ** 2 - qe + 0.5
    d = RF.derivative(y, dq)
    assert np.max(np.abs(d - (6.0 * qe - 1.0))) < 1e-12
    # and halve the error of a cubic's end slope four times per halving of dq
    e = []
    for n in (41, 81):
        q = np.arange(n) / (n - 1)
        e.append(abs(RF.derivative(q ** 3, q[1] - q[0])[0]))
    assert 3.5 < e[0] / e[1] < 4.5
