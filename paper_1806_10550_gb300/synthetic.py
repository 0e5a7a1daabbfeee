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
    x = cell_centres(nx, ds)[None, :]
    y = cell_centres(ny, ds)[:, None]
    dip = np.zeros((ny, nx))
    for k in range(n_holes):
        dip += np.exp(-((x - cx[k]) ** 2 + (y - cy[k]) ** 2) / (width * width))
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
