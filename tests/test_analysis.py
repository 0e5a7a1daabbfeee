"""CPU checks of the radial-spectrum analysis used by the precision tests."""
import math

import numpy as np

from paper_1806_10550_gb300 import analysis as A
from paper_1806_10550_gb300 import synthetic as S


def test_single_mode_peak_is_exact():
    n, ds = 128, 0.7
    L = n * ds
    for px, py in [(6, 8), (10, 0), (3, 4)]:
        h = S.mode_film(n, n, ds, 1.0, 0.05, px, py)
        k = A.dominant_wavenumber(h, ds)
        assert abs(k - math.pi * math.hypot(px, py) / L) <= 0.5 * math.pi / L


def test_ring_average_prefers_stronger_ring():
    n, ds = 96, 1.0
    h = S.mode_film(n, n, ds, 1.0, 0.01, 12, 0) + (S.mode_film(n, n, ds, 1.0, 0.03, 0, 5) - 1.0)
    assert abs(A.dominant_wavenumber(h, ds) - math.pi * 5 / (n * ds)) < 1e-12
