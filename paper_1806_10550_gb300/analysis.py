"""Film analysis on the host: dominant wavenumber of a film pattern.

A simplified form of the paper's radial Fourier analysis (App. Radial
Fourier Transform): the film minus its mean is expanded in the cosine modes
of the no-flux box (a 2-D DCT-II, the modes the walls allow), the power is
averaged over rings of equal wavenumber k = pi |(p, q)| / L, and the ring
with the largest mean power gives the dominant wavenumber.  Used to check
that the FP32-bulk and FP64 modes select the same pattern scale.
"""
from __future__ import annotations

import numpy as np
from scipy.fft import dctn


def radial_spectrum(h: np.ndarray, ds: float, nbins: int | None = None):
    """(k_centres, mean power per ring) of a square film [n, n] with spacing ds."""
    h = np.asarray(h, dtype=np.float64)
    n = h.shape[0]
    assert h.shape == (n, n)
    c = dctn(h - h.mean(), type=2, norm="ortho")
    L = n * ds
    p = np.arange(n)
    kk = np.pi * np.hypot(p[:, None], p[None, :]) / L
    nbins = nbins or n // 2
    dk = np.pi / L
    idx = np.rint(kk / dk).astype(int)
    power = np.bincount(idx.ravel(), weights=(c * c).ravel(), minlength=nbins + 1)
    count = np.bincount(idx.ravel(), minlength=nbins + 1)
    sel = slice(1, nbins + 1)  # drop the mean (k = 0)
    with np.errstate(invalid="ignore", divide="ignore"):
        mean_power = power[sel] / np.maximum(count[sel], 1)
    return np.arange(1, nbins + 1) * dk, mean_power


def dominant_wavenumber(h: np.ndarray, ds: float) -> float:
    k, pw = radial_spectrum(h, ds)
    return float(k[int(np.argmax(pw))])
