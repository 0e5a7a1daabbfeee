"""GPU parity for the NLC and polymer models (Sec. Thin Film Models) against
the FP64 oracle: the whole path with only the mobilities changed.

Tolerances are those of test_gpu_parity.py.  In FP32-bulk the models'
mobilities are evaluated in FP64 inside the double-float residual and in FP32
for the Jacobian.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

MODES = [tf.TF_FP64, tf.TF_FP32_BULK]
CASES = {
    # model, C, b, flat height (Sec. Validation)
    "nlc": (tf.TF_MODEL_NLC, O.MODEL_NLC, 0.0857, 0.01, 0.5),
    "pol": (tf.TF_MODEL_POLYMER, O.MODEL_POLYMER, 0.00581, 0.1, 3.9),
}


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    tf.library()
    return T


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def setup(which, nx, ny, mode, cells_per_lambda=8.0):
    gm, om_id, C, b, h0 = CASES[which]
    probe = O.Model(nx=4, ny=4, ds=1.0, model=om_id, cap_C=C, b=b)
    qm, wm = O.lsa(probe, h0)
    ds = 2 * math.pi / qm / cells_per_lambda
    om = O.Model(nx=nx, ny=ny, ds=ds, model=om_id, cap_C=C, b=b)
    p = tf.tf_params_default(nx=nx, ny=ny, ds=ds, model=gm, cap_C=C, b=b, precision=mode)
    return om, p, h0, wm


@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nx,ny", [(5, 7), (37, 53), (130, 97)])
def test_residual_parity(torch, which, mode, nx, ny):
    om, p, h0, wm = setup(which, nx, ny, mode)
    dt = 0.05 / wm
    h_old = S.spinodal_film(nx, ny, h0, 0.05, seed=nx * 1000 + ny)
    h_k = h_old + 0.01 * h0 * S.spinodal_film(nx, ny, 0.0, 1.0, seed=7)
    ctx = tf.Context(p)
    G = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    tf.tf_residual(ctx, dev(torch, h_k), dev(torch, h_old), dt, G)
    ref = O.residual(om, h_k, O.explicit_part(om, h_old, dt), dt)
    scale = h0 * 1e-13 if mode == tf.TF_FP64 else h0 * 1e-12
    assert np.max(np.abs(host(G) - ref)) <= scale


@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nx,ny", [(3, 2), (37, 53), (203, 151)])
def test_one_iteration_parity(torch, which, mode, nx, ny):
    om, p, h0, wm = setup(which, nx, ny, mode)
    dt = 0.001 / wm  # these grids are stiff: (q_max / q_m)^4 = 4096
    h_old = S.spinodal_film(nx, ny, h0, 0.02, seed=3 + nx)
    ctx = tf.Context(p)
    shape = (ny, nx)
    w, v, hn = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3))
    hk = dev(torch, h_old)
    info = tf.tf_newton_iteration(ctx, hk, hk, dt, hn, w=w, v=v)
    r = O.newton_iteration(om, h_old, O.explicit_part(om, h_old, dt), dt)
    sw = max(np.max(np.abs(r["w"])), 1e-300)
    sv = max(np.max(np.abs(r["v"])), 1e-300)
    tol = 1e-11 if mode == tf.TF_FP64 else 2e-4
    assert np.max(np.abs(host(w) - r["w"])) <= tol * sw
    assert np.max(np.abs(host(v) - r["v"])) <= tol * sv
    assert np.max(np.abs(host(hn) - r["unew"])) <= 1e-14 * h0 + tol * sv


@pytest.mark.parametrize("which", list(CASES))
@pytest.mark.parametrize("mode", MODES)
def test_step_parity(torch, which, mode):
    nx, ny = 48, 40
    om, p, h0, wm = setup(which, nx, ny, mode)
    dt = 0.001 / wm
    h = S.spinodal_film(nx, ny, h0, 0.01, seed=5)
    ctx = tf.Context(p)
    hn = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    info = tf.tf_newton_adi_step(ctx, dev(torch, h), hn, dt)
    ref, ri = O.step(om, O.Control(), h, dt)
    assert ri["status"] == 0 and info["status"] == tf.TF_STEP_CONVERGED
    if mode == tf.TF_FP64:
        assert info["iterations"] == ri["iterations"]
        assert np.max(np.abs(host(hn) - ref)) <= 1e-13 * h0
    else:
        assert abs(info["iterations"] - ri["iterations"]) <= 2
        assert np.max(np.abs(host(hn) - ref)) <= 1e-9 * h0
    assert abs(host(hn).sum() - h.sum()) <= 1e-12 * h.sum()


@pytest.mark.parametrize("which", list(CASES))
def test_adaptive_run_parity(torch, which):
    # 40 adaptive attempts on a 64^2 film (8 wavelengths), FP64: the same
    # accept/reject decisions and iteration counts as the oracle, films to
    # 1e-10 relative.
    nx = ny = 64
    om, p, h0, wm = setup(which, nx, ny, tf.TF_FP64)
    h = S.spinodal_film(nx, ny, h0, 0.01, seed=11)
    ctl = O.Control()
    dt0, t_end = 0.001 / wm, 1e30
    ref = O.advance(om, ctl, h, 0.0, t_end, dt0, max_attempts=40)
    ctx = tf.Context(p)
    g = dev(torch, h)
    out, recs = tf.tf_advance(ctx, g, 0.0, t_end, dt0, max_attempts=40)
    assert out["attempts"] == len(ref.records) == 40
    assert [r["accepted"] for r in recs] == [r["accepted"] for r in ref.records]
    assert [r["iterations"] for r in recs] == [r["iterations"] for r in ref.records]
    assert np.max(np.abs(host(g) - ref.h)) <= 1e-10 * h0
