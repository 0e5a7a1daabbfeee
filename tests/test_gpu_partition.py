"""Parity of the partitioned line solver (TF_SOLVER_PARTITIONED: FP32-bulk,
(3, 2) power law) at the edges of its segment geometry.

x lines are cut into segments of 64 cells and y lines into segments of 32,
with two-cell separators between segments; a last segment that would hold
fewer than 4 cells starts at n - 4 instead.  Each shape below puts a line
length at or next to one of those cases (a single segment, a full segment,
one to four cells past it, several segments with a ragged tail), and one
Newton iteration (w, v, u_{k+1}, the Newton error and mass) is compared with
the FP64 oracle at the tolerances of the FP32 solves, at two step sizes (the
stiffer one makes the reduced systems carry most of the solution).
"""
import numpy as np
import pytest

import oracle as O
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

KAPPA = 1.2061475842818314

SHAPES = [(64, 32), (65, 33), (66, 34), (67, 35), (68, 36), (69, 37), (63, 31), (129, 65), (131, 67),
          (132, 96), (190, 98), (7, 129), (130, 5), (1, 70), (70, 1), (2, 2), (4, 300), (300, 4)]


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    tf.library()
    return T


@pytest.mark.parametrize("dt", [2.0, 200.0])
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_partitioned_iteration_matches_oracle(torch, nx, ny, dt):
    ds = 1.9
    om = O.Model(nx=nx, ny=ny, ds=ds, kappa=KAPPA)
    p = tf.tf_params_default(nx=nx, ny=ny, ds=ds, kappa=KAPPA, precision=tf.TF_FP32_BULK,
                             line_solver=tf.TF_SOLVER_PARTITIONED)
    h_old = S.spinodal_film(nx, ny, 1.0, 0.05, seed=11 * nx + ny)
    ctx = tf.Context(p)
    w, v, hn = (torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3))
    hk = torch.from_numpy(h_old).cuda()
    info = tf.tf_newton_iteration(ctx, hk, hk, dt, hn, w=w, v=v)
    r = O.newton_iteration(om, h_old, O.explicit_part(om, h_old, dt), dt)
    sw = max(np.max(np.abs(r["w"])), 1e-300)
    sv = max(np.max(np.abs(r["v"])), 1e-300)
    assert np.max(np.abs(w.cpu().numpy() - r["w"])) <= 2e-4 * sw
    assert np.max(np.abs(v.cpu().numpy() - r["v"])) <= 2e-4 * sv
    assert np.max(np.abs(hn.cpu().numpy() - r["unew"])) <= 1e-15 + 2e-4 * sv
    assert info["err"] == pytest.approx(r["err"], rel=1e-3)
    if np.min(r["unew"]) > 0.0:
        assert info["status"] in (tf.TF_STEP_CONVERGED, tf.TF_STEP_NOT_CONVERGED)
        # FP32 solves: the update's sum to the solves' relative accuracy
        mtol = nx * ny * 2.0 ** -37 + 1e-13 * r["unew"].sum() + 1e-4 * np.abs(r["v"]).sum()
        assert abs(info["mass"] - r["unew"].sum()) <= mtol
    else:  # the large step overshoots: the iterate leaves the model's domain
        assert info["status"] == tf.TF_STEP_NONPOSITIVE
    ctx.close()


@pytest.mark.parametrize("nx,ny", [(131, 67), (260, 130)])
def test_partitioned_step_converges_to_oracle_step(torch, nx, ny):
    """A whole converged step: the partitioned FP32 solves change only the
    path of the iteration, not its FP64-class fixed point."""
    ds, dt = 3.9, 2.0
    om = O.Model(nx=nx, ny=ny, ds=ds, kappa=KAPPA)
    p = tf.tf_params_default(nx=nx, ny=ny, ds=ds, kappa=KAPPA, precision=tf.TF_FP32_BULK,
                             line_solver=tf.TF_SOLVER_PARTITIONED)
    h0 = S.spinodal_film(nx, ny, 1.0, 0.01, seed=nx + ny)
    ref, ri = O.step(om, O.Control(), h0, dt)
    assert ri["status"] == 0
    ctx = tf.Context(p)
    h = torch.from_numpy(h0).cuda()
    hn = torch.empty_like(h)
    info = tf.tf_newton_adi_step(ctx, h, hn, dt)
    assert info["status"] == tf.TF_STEP_CONVERGED
    assert np.max(np.abs(hn.cpu().numpy() - ref)) <= 1e-9
    ctx.close()
