"""The seeded input recipes (paper_1806_10550_gb300/synthetic.py) that the
CUDA path and the oracle both consume: ranges, reproducibility, wall
compatibility of the cosine modes, and the windowing of the nucleation
film's Gaussian depressions against the plain sum over the whole film."""
import numpy as np

from paper_1806_10550_gb300 import synthetic as S


def test_spinodal_film_range_and_seed():
    h = S.spinodal_film(48, 40, 2.0, 0.01, seed=1234)
    assert h.shape == (40, 48) and h.dtype == np.float64
    assert np.all(np.abs(h / 2.0 - 1.0) <= 0.01)
    assert np.array_equal(h, S.spinodal_film(48, 40, 2.0, 0.01, seed=1234))
    assert not np.array_equal(h, S.spinodal_film(48, 40, 2.0, 0.01, seed=1235))
    # one U[-1, 1] draw per cell, row-major [ny, nx]
    u = np.random.default_rng(1234).uniform(-1.0, 1.0, size=(40, 48))
    assert np.array_equal(h, 2.0 * (1.0 + 0.01 * u))


def test_nucleation_film_windows_equal_the_full_sum():
    nx, ny, ds, h0, eps, nh, depth, width, seed = 96, 80, 1.5, 1.0, 1e-4, 9, 0.3, 4.0, 77
    h = S.nucleation_film(nx, ny, ds, h0, eps, nh, depth, width, seed)
    rng = np.random.default_rng(seed)
    noise = rng.uniform(-1.0, 1.0, size=(ny, nx))
    cx = rng.uniform(0.0, nx * ds, size=nh)
    cy = rng.uniform(0.0, ny * ds, size=nh)
    x = (np.arange(nx) + 0.5) * ds
    y = (np.arange(ny) + 0.5) * ds
    dip = np.zeros((ny, nx))
    for k in range(nh):
        dip += np.exp(-((x[None, :] - cx[k]) ** 2 + (y[:, None] - cy[k]) ** 2) / width ** 2)
    full = h0 * (1.0 + eps * noise - depth * dip)
    # the depressions are cut at 8 widths, where exp(-64) is below the last bit
    assert np.max(np.abs(h - full)) <= 1e-15 * h0
    assert np.min(h) < h0 * (1.0 - 0.5 * depth)  # at least one full depression


def test_mode_film_is_wall_compatible():
    nx, ny, ds = 36, 28, 0.7
    h = S.mode_film(nx, ny, ds, 1.0, 0.1, px=3, py=2)
    x = (np.arange(nx) + 0.5) * ds
    y = (np.arange(ny) + 0.5) * ds
    L, H = nx * ds, ny * ds

    def fx(s):
        return np.cos(np.pi * 3 * s / L)

    def fy(s):
        return np.cos(np.pi * 2 * s / H)

    assert np.allclose(h, 1.0 + 0.1 * np.outer(fy(y), fx(x)), rtol=0, atol=1e-15)
    # each factor is even about both walls, so the film reflected across a
    # wall continues it (what the no-flux reflection of the method assumes)
    assert np.allclose(fx(x), fx(-x), rtol=0, atol=1e-15)
    assert np.allclose(fx(x), fx(2 * L - x), rtol=0, atol=1e-13)
    assert np.allclose(fy(y), fy(-y), rtol=0, atol=1e-15)
    assert np.allclose(fy(y), fy(2 * H - y), rtol=0, atol=1e-13)


def test_ring_film_amplitude_and_sizes():
    h = S.ring_film(64, 48, 1.0, 1.0, 0.05, 2 * np.pi / 16, 0.05, 32, 0.0, seed=7)
    assert abs(np.max(np.abs(h - 1.0)) - 0.05) <= 1e-15
    hn = S.ring_film(64, 48, 1.0, 1.0, 0.05, 2 * np.pi / 16, 0.05, 32, 0.002, seed=7)
    assert np.max(np.abs(hn - h)) <= 0.002 + 1e-15
    sizes = S.film_ensemble_sizes(50, [128, 256, 512, 1024], seed=3)
    assert len(sizes) == 50 and set(sizes) <= {128, 256, 512, 1024}
