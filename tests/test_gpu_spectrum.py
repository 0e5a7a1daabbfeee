"""GPU parity of the radial Fourier analysis (App. Radial Fourier Transform)
against the oracle, stage by stage, through the C ABI.

Tolerances:
- amplitude and smoothed spectra: the GPU transform is FP32.  A radix-2 FFT
  of length n has ||error||_2 <= log2(n) eta ||X||_2 with eta ~ 6.7 u for
  twiddles correct to u = 2^-24; two passes, the rounding of zeta to FP32 and
  the Makhoul pre/post steps give at most (log2(nx ny) + 6) eta.  With
  ||C||_2 <= sqrt(nx ny) ||zeta||_2 every entry of A = |C| / (nx ny) is off by
  at most (log2(nx ny) + 6) * 8u * rms(zeta).  Smoothing and radial means are
  convex combinations, so the bound carries over.
- later stages take the GPU's own previous stage as the oracle's input
  (FP64 on both sides): radial means sum the same values in the same order
  (1e-15 relative); the fit differs only by the elimination order of the
  normal equations (1e-10 of the largest node value); curve and maxima to
  rounding.
"""
import math

import numpy as np
import pytest

import oracle.radial_fourier as RF
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    tf.library()
    return T


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def fft_bound(h, H0):
    # FP32 transform (see the module docstring) plus the formation of zeta
    # in FP32 pieces: within 2^-24 |zeta| + 2^-45 (|h| + |H0|) per cell
    ny, nx = h.shape
    rms = math.sqrt(np.mean((h - H0) ** 2))
    return (math.log2(nx * ny) + 6) * 8 * U32 * rms + 2.0 ** -45 * (np.max(np.abs(h)) + abs(H0))


def run_gpu(torch, h, ds, **kw):
    ny, nx = h.shape
    sp = tf.tf_spectrum_params_default(**kw)
    plan = tf.SpectrumPlan(nx, ny, ds, sp)
    g = dev(torch, h)
    r = tf.tf_spectrum_run(plan, g, peak_cap=4096)
    assert np.array_equal(g.cpu().numpy(), h)  # the film is read only
    return plan, r


def check_stages(r, h, ds, H0, q_cut, sigma, ppi, n_eval):
    """Each GPU stage against the oracle step fed with the GPU's previous stage."""
    ny, nx = h.shape
    n_p, n_q = r["n_p"], r["n_q"]
    _, _, _, _, op, oq = RF.radial_geometry(nx, ny, ds, q_cut)
    assert (n_p, n_q) == (op, oq)
    R = (len(RF.gaussian_weights(sigma)) - 1) // 2
    A = RF.amplitude(h, H0, min(nx, n_p + R), min(ny, n_q + R))
    bound = fft_bound(h, H0)
    assert np.max(np.abs(r["amplitude"] - A[:n_q, :n_p])) <= bound
    Sm = RF.smooth(A, nx, ny, n_p, n_q, sigma)
    assert np.max(np.abs(r["smoothed"] - Sm)) <= bound
    # radial means of the GPU's smoothed block
    q_r, y, cnt, keys = RF.radial_profile(r["smoothed"], nx, ny, ds, q_cut)
    assert r["n_radii"] == len(q_r)
    assert np.max(np.abs(r["radial_q"] - q_r)) <= 1e-15 * q_cut
    assert np.max(np.abs(r["radial_value"] - y)) <= 1e-15 * np.max(np.abs(y))
    # fit of the GPU's radial means
    t, a = RF.fit(r["radial_q"], r["radial_value"], q_cut, ppi)
    assert r["n_intervals"] == len(t) - 1
    assert np.array_equal(r["node_q"], t)
    assert r["node_value"][0] == 0.0
    assert np.max(np.abs(r["node_value"] - a)) <= 1e-10 * max(np.max(np.abs(a)), 1e-300)
    # curve from the GPU's nodes
    qe, ye = RF.sample_and_smooth(r["node_q"], r["node_value"], q_cut, n_eval)
    assert np.max(np.abs(r["curve_q"] - qe)) <= 1e-15 * q_cut
    assert np.max(np.abs(r["curve_value"] - ye)) <= 1e-13 * max(np.max(np.abs(ye)), 1e-300)
    # maxima of the GPU's curve
    pk = RF.local_maxima(r["curve_q"], r["curve_value"])
    assert r["n_peaks"] == len(pk)
    for (gq, gv), (oq_, ov) in zip(r["peaks"], pk):
        assert abs(gq - oq_) <= 1e-9 * q_cut
        assert abs(gv - ov) <= 1e-12 * max(abs(ov), 1e-300)
    return pk


CASES = [
    # nx, ny, ds, k0 (ring wavenumber), q_cut / k0, sigma, ppi, n_eval
    (64, 64, 1.0, 2 * math.pi / 8, 3.0, 1.0, 10, 400),
    (128, 32, 0.7, 2 * math.pi / 10, 5.0, 1.0, 10, 400),
    (32, 256, 1.3, 2 * math.pi / 12, 5.0, 1.5, 10, 400),
    (256, 256, 1.0, 2 * math.pi / 16, 5.0, 1.0, 10, 400),
    (512, 128, 2.0, 2 * math.pi / 24, 4.0, 0.0, 1, 25),
    (1, 64, 1.0, 2 * math.pi / 8, 5.0, 1.0, 3, 50),
    (64, 1, 1.0, 2 * math.pi / 8, 5.0, 2.0, 10, 100),
    (2, 2, 1.0, math.pi / 2, 2.5, 1.0, 10, 10),
    (1024, 1024, 0.5, 2 * math.pi / 16, 5.0, 1.0, 10, 400),
    (4096, 64, 1.0, 2 * math.pi / 32, 5.0, 1.0, 10, 400),
]


@pytest.mark.parametrize("nx,ny,ds,k0,fcut,sigma,ppi,n_eval", CASES)
def test_stagewise_parity(torch, nx, ny, ds, k0, fcut, sigma, ppi, n_eval):
    H0 = 1.0
    h = S.ring_film(nx, ny, ds, H0, 0.05, k0, 0.05, 64, 0.002, seed=nx + 3 * ny)
    q_cut = fcut * k0
    _, r = run_gpu(torch, h, ds, H0=H0, q_cut=q_cut, sigma=sigma, points_per_interval=ppi,
                   n_eval=n_eval)
    check_stages(r, h, ds, H0, q_cut, sigma, ppi, n_eval)


@pytest.mark.parametrize("nx,ny", [(256, 256), (1024, 512)])
def test_dominant_wavenumber_matches_oracle_end_to_end(torch, nx, ny):
    ds, H0 = 1.0, 1.0
    k0 = 2 * math.pi / 20
    h = S.ring_film(nx, ny, ds, H0, 0.05, k0, 0.03, 128, 0.001, seed=7)
    q_cut = 5 * k0
    _, r = run_gpu(torch, h, ds, H0=H0, q_cut=q_cut)
    o = RF.analyse(h, ds, H0, q_cut)
    assert r["n_peaks"] >= 1
    assert abs(r["q_dominant"] - o["q_dominant"]) <= 1e-6 * q_cut
    assert abs(r["q_dominant"] - k0) <= 0.1 * k0


def test_single_mode_amplitude(torch):
    nx, ny, ds, eps = 128, 64, 0.8, 0.02
    h = S.mode_film(nx, ny, ds, 1.0, eps, 9, 5)
    q_cut = 1.5 * math.pi * math.hypot(9 / (nx * ds), 5 / (ny * ds))
    _, r = run_gpu(torch, h, ds, H0=1.0, q_cut=q_cut, sigma=0.0)
    A = r["amplitude"]
    assert abs(A[5, 9] - eps / 4) <= 4 * U32 * eps
    A[5, 9] = 0.0
    assert np.max(A) <= 16 * U32 * eps


def test_runs_are_bit_identical(torch):
    h = S.ring_film(512, 512, 1.0, 1.0, 0.05, 2 * math.pi / 16, 0.05, 64, 0.002, seed=4)
    plan, r1 = run_gpu(torch, h, 1.0, H0=1.0, q_cut=1.5)
    r2 = tf.tf_spectrum_run(plan, dev(torch, h), peak_cap=4096)
    for k in ("amplitude", "smoothed", "radial_value", "node_value", "curve_value"):
        assert np.array_equal(r1[k], r2[k]), k
    assert r1["peaks"] == r2["peaks"]


def test_three_samples_give_a_flat_curve(torch):
    # n_eval = 3: every moving-average window spans the whole curve, which is
    # then constant (the mean of the three samples); its maxima are undefined
    h = S.ring_film(64, 64, 1.0, 1.0, 0.05, 2 * math.pi / 8, 0.05, 32, 0.002, seed=9)
    _, r = run_gpu(torch, h, 1.0, H0=1.0, q_cut=2.0, n_eval=3)
    qe, ye = RF.sample_and_smooth(r["node_q"], r["node_value"], 2.0, 3)
    assert np.max(np.abs(r["curve_value"] - ye)) <= 1e-15 * np.max(np.abs(ye))
    assert r["curve_value"][0] == r["curve_value"][1] == r["curve_value"][2]


def test_too_few_radial_points_rejected(torch):
    sp = tf.tf_spectrum_params_default(q_cut=0.5 * math.pi / 64)  # below the first ring
    with pytest.raises(RuntimeError):
        tf.SpectrumPlan(64, 64, 1.0, sp)


def test_full_size_workload(torch):
    # the benchmarked analysis: an 8192^2 film at the 8192^2 workloads' spacing
    # (lambda_m / 128), pattern at q_m, q_cut = 5 q_m
    import json
    import os
    W = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))
    w = W["spectrum8k"]
    N, ds = w["N"], w["ds"]
    qm = 2 * math.pi / w["lambda_m"]
    h = S.ring_film(N, N, ds, 1.0, w["eps"], qm, w["spread"], w["modes"], w["noise"], seed=w["seed"])
    q_cut = w["q_cut"]
    plan, r = run_gpu(torch, h, ds, H0=1.0, q_cut=q_cut, sigma=w["sigma"],
                      points_per_interval=w["points_per_interval"], n_eval=w["n_eval"])
    n_p, n_q = r["n_p"], r["n_q"]
    # sampled amplitudes, each an oracle sum over the whole film
    rng = np.random.default_rng(1)
    ps = np.unique(np.concatenate([[0, 1, n_p - 1], rng.integers(0, n_p, 20)]))
    qs = np.unique(np.concatenate([[0, 1, n_q - 1], rng.integers(0, n_q, 20)]))
    rows = (h - 1.0) @ RF.cos_matrix(n_p, N)[ps].T          # [N, len(ps)]
    A = np.abs(RF.cos_matrix(n_q, N)[qs] @ rows) / (N * N)   # [len(qs), len(ps)]
    assert np.max(np.abs(r["amplitude"][np.ix_(qs, ps)] - A)) <= fft_bound(h, 1.0)
    # later stages from the GPU's smoothed block
    q_r, y, _, _ = RF.radial_profile(r["smoothed"], N, N, ds, q_cut)
    assert np.max(np.abs(r["radial_value"] - y)) <= 1e-15 * np.max(np.abs(y))
    t, a = RF.fit(r["radial_q"], r["radial_value"], q_cut)
    assert np.max(np.abs(r["node_value"] - a)) <= 1e-10 * np.max(np.abs(a))
    pk = RF.local_maxima(*RF.sample_and_smooth(r["node_q"], r["node_value"], q_cut))
    assert abs(r["q_dominant"] - pk[0][0]) <= 1e-9 * q_cut
    assert abs(r["q_dominant"] - qm) <= 0.05 * qm


def test_heights_outside_the_fast_conversion_range(torch):
    # zero, negative and tiny heights take the FP64 route for zeta (the
    # transform is FP32: heights beyond its range are not representable)
    nx, ny, ds = 128, 64, 1.0
    h = S.ring_film(nx, ny, ds, 1.0, 0.05, 2 * math.pi / 8, 0.05, 32, 0.002, seed=21)
    h[3, 5], h[10, 77], h[40, 1], h[63, 127], h[0, 0] = 0.0, -0.5, 1e-25, 1e30, 2.0 ** -70
    q_cut = 0.5 * math.pi / ds
    _, r = run_gpu(torch, h, ds, H0=1.0, q_cut=q_cut)
    A = RF.amplitude(h, 1.0, r["n_p"], r["n_q"])
    assert np.max(np.abs(r["amplitude"] - A)) <= fft_bound(h, 1.0)
