"""FP32-bulk against FP64 on a developing nucleation film (GPU).

The precision mode computes the correction solves and stencils in FP32 and
the residual, update and norms in double-float; Newton then refines to the
FP64-class fixed point.  On a 1024^2 film at the nucleation workload's
spacing (lambda_m / 32), with 1e-4 noise plus Gaussian depressions of depth
0.3 h0 and width lambda_m / 4, FP64 runs the adaptive controller to 6/sigma_max
(or rupture) and FP32-bulk replays its step sizes.  Required: relative mass
error <= 1e-6 in both modes, the same dominant wavenumber in both (the
radial Fourier analysis of App. Radial Fourier Transform, on the GPU,
checked against the oracle's), and that wavenumber near the
linear-stability k_m.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle.radial_fourier as RF
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

W = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    return T


def test_fp32_bulk_keeps_mass_and_dominant_wavelength(torch):
    w = dict(W["nucl8k"])
    N = 1024
    lam, sm = w["lambda_m"], w["sigma_max"]
    w["N"], w["P"] = N, 32
    w["ds"] = w["P"] * lam / N  # = lambda_m / 32, the nucleation workload's spacing
    h0 = S.nucleation_film(N, N, w["ds"], w["h0"], 1e-4, 16, 0.3, lam / 4, seed=w["seed"])
    T_end = 6.0 / sm
    ctx64 = tf.Context(tf.params_for_workload(w, tf.TF_FP64))
    h64 = torch.from_numpy(h0).cuda()
    info64, rec64 = tf.tf_advance(ctx64, h64, 0.0, T_end, w["dt0"], 4000)
    assert info64["status"] in (tf.TF_ADV_DONE, tf.TF_ADV_RUPTURE), info64
    acc = [r for r in rec64 if r["accepted"]]
    ctx32 = tf.Context(tf.params_for_workload(w, tf.TF_FP32_BULK))
    h32 = torch.from_numpy(h0).cuda()
    info32, rec32 = tf.tf_advance(ctx32, h32, 0.0, 1e30, 1.0, len(acc),
                                  dt_replay=[r["dt"] for r in acc])
    assert info32["accepted"] == len(acc), info32
    a64, a32 = h64.cpu().numpy(), h32.cpu().numpy()
    m0 = h0.sum()
    assert abs(a64.sum() - m0) <= 1e-6 * m0
    assert abs(a32.sum() - m0) <= 1e-6 * m0
    km = 2 * math.pi / lam
    q_cut = 5 * km
    plan = tf.SpectrumPlan(N, N, w["ds"], tf.tf_spectrum_params_default(H0=w["h0"], q_cut=q_cut))
    k64 = tf.tf_spectrum_run(plan, h64, outputs=False)["q_dominant"]
    k32 = tf.tf_spectrum_run(plan, h32, outputs=False)["q_dominant"]
    ko = RF.analyse(a64, w["ds"], w["h0"], q_cut)["q_dominant"]
    assert abs(k64 - ko) <= 1e-6 * q_cut
    assert abs(k64 - k32) <= 1e-3 * km
    assert abs(k64 - km) <= 0.25 * km
    # the film itself: FP32-bulk within Newton-tolerance accumulation of FP64
    assert np.max(np.abs(a32 - a64)) <= 1e-5
    print(f"steps={len(acc)} t={info64['t']:.1f} k_dom={k64:.5f} k_m={km:.5f} "
          f"max|h32-h64|={np.max(np.abs(a32 - a64)):.3e} "
          f"mass err 64={abs(a64.sum() - m0) / m0:.2e} 32={abs(a32.sum() - m0) / m0:.2e}")


def test_fp32_bulk_against_fp64_at_full_size(torch):
    """The precision workload at its full size: 8192^2 on 256 lambda_m
    (lambda_m / 32), 1e-4 noise plus 64 depressions of depth 0.3 h0 and
    width lambda_m / 4.  FP64 runs the adaptive controller to 6/sigma_max;
    FP32-bulk replays its step sizes.  The same requirements as above."""
    w = W["nucl8k"]
    N, lam, sm = w["N"], w["lambda_m"], w["sigma_max"]
    h0 = S.nucleation_film(N, N, w["ds"], w["h0"], w["eps"], w["holes"], w["depth"], w["width"], seed=w["seed"])
    ctx64 = tf.Context(tf.params_for_workload(w, tf.TF_FP64))
    h64 = torch.from_numpy(h0).cuda()
    info64, rec64 = tf.tf_advance(ctx64, h64, 0.0, 6.0 / sm, w["dt0"], 4000)
    assert info64["status"] in (tf.TF_ADV_DONE, tf.TF_ADV_RUPTURE), info64
    acc = [r for r in rec64 if r["accepted"]]
    ctx64.close()
    ctx32 = tf.Context(tf.params_for_workload(w, tf.TF_FP32_BULK))
    h32 = torch.from_numpy(h0).cuda()
    info32, _ = tf.tf_advance(ctx32, h32, 0.0, 1e30, 1.0, len(acc), dt_replay=[r["dt"] for r in acc])
    assert info32["accepted"] == len(acc), info32
    m0 = float(np.sum(h0))
    m64, m32 = float(h64.sum()), float(h32.sum())
    assert abs(m64 - m0) <= 1e-6 * m0
    assert abs(m32 - m0) <= 1e-6 * m0
    km = 2 * math.pi / lam
    q_cut = 5 * km
    plan = tf.SpectrumPlan(N, N, w["ds"], tf.tf_spectrum_params_default(H0=w["h0"], q_cut=q_cut))
    k64 = tf.tf_spectrum_run(plan, h64, outputs=False)["q_dominant"]
    k32 = tf.tf_spectrum_run(plan, h32, outputs=False)["q_dominant"]
    assert abs(k64 - k32) <= 1e-3 * km
    assert abs(k64 - km) <= 0.25 * km
    dmax = float(torch.max(torch.abs(h32 - h64)))
    assert dmax <= 1e-5
    print(f"steps={len(acc)} t={info64['t']:.1f} k_dom={k64:.5f} k_m={km:.5f} max|h32-h64|={dmax:.3e} "
          f"mass err 64={abs(m64 - m0) / m0:.2e} 32={abs(m32 - m0) / m0:.2e}")
