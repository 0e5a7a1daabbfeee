"""Seeded synthetic initial films for the thin-film workloads.

This module holds no arithmetic of the numerical method: it only draws the
initial heights that both the CUDA path and the CPU oracle consume, so that
the two sides see bit-identical inputs.

* Spinodal films (Sec. Simulations, the random-perturbation runs): a flat
  film ``h0 (1 + eps U[-1, 1])`` with one uniform draw per cell from NumPy's
  ``default_rng(seed)``, generated once on the host in float64.
* Nucleation films (Sec. Simulations, localized plus global perturbations):
  the same noise at ``eps = 1e-4`` plus Gaussian depressions
  ``-depth * exp(-|x - c_k|^2 / w^2)`` with seeded centres, summed where they
  overlap.
* Single cosine modes ``h0 (1 + eps cos(kx x) cos(ky y))`` with
  ``k = pi p / L`` (compatible with the no-flux walls), for validation.
* Ring films: a stand-in for a film whose spinodal pattern has developed
  (Sec. Results, the films the radial Fourier analysis is applied to):
  ``n_modes`` wall-compatible cosine modes whose wavenumbers scatter about
  ``k0`` (relative spread ``spread``, uniform direction), seeded amplitudes
  in [0, 1] and signs, scaled to ``eps`` at the largest excursion, plus
  ``noise`` U[-1, 1] per cell.

Cell ``(i, j)`` has its centre at ``((i + 1/2) ds, (j + 1/2) ds)``; arrays
are row-major ``[ny, nx]``.
"""
from __future__ import annotations

import numpy as np


def cell_centres(n: int, ds: float) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) * ds


def spinodal_film(nx: int, ny: int, h0: float, eps: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return h0 * (1.0 + eps * rng.uniform(-1.0, 1.0, size=(ny, nx)))


def nucleation_film(nx: int, ny: int, ds: float, h0: float, eps: float,
                    n_holes: int, depth: float, width: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1.0, 1.0, size=(ny, nx))
    cx = rng.uniform(0.0, nx * ds, size=n_holes)
    cy = rng.uniform(0.0, ny * ds, size=n_holes)
    xc = cell_centres(nx, ds)
    yc = cell_centres(ny, ds)
    dip = np.zeros((ny, nx))
    # each depression within 8 widths of its centre: beyond, exp(-64) ~ 1e-28
    # is far below the last bit of h
    R = 8.0 * width
    for k in range(n_holes):
        i0 = max(0, int(np.floor((cx[k] - R) / ds)) - 1)
        i1 = min(nx, int(np.ceil((cx[k] + R) / ds)) + 1)
        j0 = max(0, int(np.floor((cy[k] - R) / ds)) - 1)
        j1 = min(ny, int(np.ceil((cy[k] + R) / ds)) + 1)
        x = xc[None, i0:i1]
        y = yc[j0:j1, None]
        dip[j0:j1, i0:i1] += np.exp(-((x - cx[k]) ** 2 + (y - cy[k]) ** 2) / (width * width))
    return h0 * (1.0 + eps * noise - depth * dip)


def mode_film(nx: int, ny: int, ds: float, h0: float, eps: float,
              px: int, py: int) -> np.ndarray:
    kx = np.pi * px / (nx * ds)
    ky = np.pi * py / (ny * ds)
    x = cell_centres(nx, ds)[None, :]
    y = cell_centres(ny, ds)[:, None]
    return h0 * (1.0 + eps * np.cos(kx * x) * np.cos(ky * y))


def film_ensemble_sizes(n_films: int, choices, seed: int):
    rng = np.random.default_rng(seed)
    return [int(c) for c in rng.choice(np.asarray(choices), size=n_films)]


def ring_film(nx: int, ny: int, ds: float, h0: float, eps: float, k0: float, spread: float,
              n_modes: int, noise: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    k = k0 * (1.0 + spread * rng.standard_normal(n_modes))
    ang = rng.uniform(0.0, 0.5 * np.pi, n_modes)
    p = np.clip(np.rint(k * np.cos(ang) * nx * ds / np.pi), 0, nx - 1)
    q = np.clip(np.rint(k * np.sin(ang) * ny * ds / np.pi), 0, ny - 1)
    amp = rng.uniform(0.0, 1.0, n_modes) * rng.choice([-1.0, 1.0], n_modes)
    cx = np.cos(np.pi * p[:, None] * cell_centres(nx, ds)[None, :] / (nx * ds))
    cy = np.cos(np.pi * q[:, None] * cell_centres(ny, ds)[None, :] / (ny * ds))
    pattern = cy.T @ (amp[:, None] * cx)
    pattern /= np.max(np.abs(pattern))
    return h0 * (1.0 + eps * pattern + noise * rng.uniform(-1.0, 1.0, size=(ny, nx)))
