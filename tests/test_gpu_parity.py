"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 mode is compared element by element with the oracle.  The tolerance is
1e-10 relative L-infinity on film heights over whole runs (the target the
method's FP64 implementation is held to).  Single operators are held to
round-off-level bounds.  FP32-bulk mode: the residual is double-float and
must match the oracle's FP64 residual to 1e-12 absolute.  The FP32 solves
must match to single-precision tolerances.  Converged steps must match to
Newton-tolerance level and conserve mass to 1e-12.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

W = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))
KAPPA = W["small"]["kappa"]
MODES = [tf.TF_FP64, tf.TF_FP32_BULK]


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


def models(nx, ny, ds, precision=tf.TF_FP64, **kw):
    om = O.Model(nx=nx, ny=ny, ds=ds, kappa=KAPPA, **{k: v for k, v in kw.items()
                                                    if k in ("model", "c0", "c1", "theta")})
    p = tf.tf_params_default(nx=nx, ny=ny, ds=ds, kappa=KAPPA, precision=precision)
    for k, v in kw.items():
        setattr(p, k, v)
    return om, p


SHAPES = [(1, 1), (40, 1), (1, 40), (2, 3), (5, 7), (37, 53), (64, 64), (130, 97)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nx,ny", SHAPES)
def test_residual_parity(torch, mode, nx, ny):
    ds, dt = 1.7, 3.0
    om, p = models(nx, ny, ds, mode)
    h_old = S.spinodal_film(nx, ny, 1.0, 0.05, seed=nx * 1000 + ny)
    h_k = h_old + 0.01 * S.spinodal_film(nx, ny, 0.0, 1.0, seed=7) + 0.001
    ctx = tf.Context(p)
    G = torch.zeros((ny, nx), dtype=torch.float64, device="cuda")
    norms = tf.tf_residual(ctx, dev(torch, h_k), dev(torch, h_old), dt, G)
    ref = O.residual(om, h_k, O.explicit_part(om, h_old, dt), dt)
    err = np.max(np.abs(host(G) - ref))
    tol = 1e-13 if mode == tf.TF_FP64 else 1e-12
    assert err <= tol, err
    assert norms["gnorm"] == pytest.approx(np.max(np.abs(ref)), rel=1e-6, abs=1e-13)
    assert norms["hmin"] == np.min(h_k)
    # the mass is a sum of values rounded to multiples of 2^-36
    assert abs(norms["mass"] - h_k.sum()) <= nx * ny * 2.0 ** -37 + 1e-13 * h_k.sum()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nx,ny", [(1, 40), (40, 1), (3, 2), (37, 53), (64, 64), (130, 97), (203, 151)])
def test_one_iteration_parity(torch, mode, nx, ny):
    ds, dt = 1.9, 20.0
    om, p = models(nx, ny, ds, mode)
    h_old = S.spinodal_film(nx, ny, 1.0, 0.05, seed=3 + nx)
    ctx = tf.Context(p)
    shape = (ny, nx)
    w, v, hn = (torch.empty(shape, dtype=torch.float64, device="cuda") for _ in range(3))
    hk = dev(torch, h_old)
    info = tf.tf_newton_iteration(ctx, hk, hk, dt, hn, w=w, v=v)
    r = O.newton_iteration(om, h_old, O.explicit_part(om, h_old, dt), dt)
    sw = max(np.max(np.abs(r["w"])), 1e-300)
    sv = max(np.max(np.abs(r["v"])), 1e-300)
    if mode == tf.TF_FP64:
        assert np.max(np.abs(host(w) - r["w"])) <= 1e-11 * sw
        assert np.max(np.abs(host(v) - r["v"])) <= 1e-11 * sv
        assert np.max(np.abs(host(hn) - r["unew"])) <= 1e-14 + 1e-11 * sv
        assert info["err"] == pytest.approx(r["err"], rel=1e-9)
    else:
        assert np.max(np.abs(host(w) - r["w"])) <= 2e-4 * sw
        assert np.max(np.abs(host(v) - r["v"])) <= 2e-4 * sv
        assert np.max(np.abs(host(hn) - r["unew"])) <= 1e-15 + 2e-4 * sv
        assert info["err"] == pytest.approx(r["err"], rel=1e-3)
    assert info["status"] in (tf.TF_STEP_CONVERGED, tf.TF_STEP_NOT_CONVERGED)
    assert info["gnorm"] == pytest.approx(r["gnorm"], rel=1e-6)
    # FP64: mass conserved per iterate to round-off; FP32-bulk: the FP32
    # solves conserve it to single precision of the update (restored as the
    # iteration converges, see test_step_parity).
    mtol = nx * ny * 2.0 ** -37 + 1e-13 * r["unew"].sum()
    if mode != tf.TF_FP64:
        mtol += 1e-5 * np.abs(r["v"]).sum()
    assert abs(info["mass"] - r["unew"].sum()) <= mtol


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("nx,ny", [(65536, 40), (40, 65536), (65536, 3), (3, 65536)])
def test_longest_lines_one_iteration(torch, mode, nx, ny):
    """Lines of the largest length the library takes (65536 cells: halves of
    32768 in the twisted solves, 1366 chunks of 24): one Newton iteration
    against the oracle over the whole grid, with the tolerances above."""
    ds, dt = 1.9, 20.0
    om, p = models(nx, ny, ds, mode)
    h_old = S.spinodal_film(nx, ny, 1.0, 0.05, seed=nx + 7 * ny)
    ctx = tf.Context(p)
    w, v, hn = (torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3))
    hk = dev(torch, h_old)
    info = tf.tf_newton_iteration(ctx, hk, hk, dt, hn, w=w, v=v)
    r = O.newton_iteration(om, h_old, O.explicit_part(om, h_old, dt), dt)
    sw, sv = np.max(np.abs(r["w"])), np.max(np.abs(r["v"]))
    rt = 1e-11 if mode == tf.TF_FP64 else 2e-4
    assert np.max(np.abs(host(w) - r["w"])) <= rt * sw
    assert np.max(np.abs(host(v) - r["v"])) <= rt * sv
    assert np.max(np.abs(host(hn) - r["unew"])) <= 1e-14 + rt * sv
    assert info["gnorm"] == pytest.approx(r["gnorm"], rel=1e-6)


@pytest.mark.parametrize("mode", MODES)
def test_step_parity(torch, mode):
    nx, ny, ds, dt = 48, 40, 3.2, 1.0
    om, p = models(nx, ny, ds, mode)
    h0 = S.spinodal_film(nx, ny, 1.0, 0.01, seed=5)
    ctx = tf.Context(p)
    hn = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    info = tf.tf_newton_adi_step(ctx, dev(torch, h0), hn, dt)
    ref, ri = O.step(om, O.Control(), h0, dt)
    assert ri["status"] == 0 and info["status"] == tf.TF_STEP_CONVERGED
    if mode == tf.TF_FP64:
        assert info["iterations"] == ri["iterations"]
        assert np.max(np.abs(host(hn) - ref)) <= 1e-13
    else:
        assert abs(info["iterations"] - ri["iterations"]) <= 2
        assert np.max(np.abs(host(hn) - ref)) <= 1e-9
    assert abs(host(hn).sum() - h0.sum()) <= 1e-12 * h0.sum()


def _workload(name, N=None):
    w = dict(W[name])
    if N is not None:
        w["N"] = N
        w["ds"] = w["P"] * w["lambda_m"] / N
    return w


def _oracle_model(w):
    return O.Model(nx=w["N"], ny=w["N"], ds=w["ds"], kappa=w["kappa"], b=w["b"], n=w["n"],
                   m=w["m"], cap_C=w["cap_C"], theta=w["theta"])


def _oracle_control(w):
    return O.Control(tol=w["tol"], max_iter=w["max_iter"], dt_min=w["dt_min"],
                     dt_max=w["dt_max"], dt_shrink=w["dt_shrink"], dt_grow=w["dt_grow"],
                     grow_after=w["grow_after"], rupture_h=w["rupture_h"])


def test_small_workload_full_run_fp64(torch):
    """64^2 on 4 lambda_m to T = 5/sigma_max with adaptive dt: the GPU makes
    the oracle's decisions and ends within 1e-10 relative L-infinity."""
    w = _workload("small")
    h0 = S.spinodal_film(w["N"], w["N"], w["h0"], w["eps"], w["seed"])
    ref = O.advance(_oracle_model(w), _oracle_control(w), h0, 0.0, w["T"], w["dt0"], 5000)
    assert ref.status == 0
    ctx = tf.Context(tf.params_for_workload(w, tf.TF_FP64))
    h = dev(torch, h0)
    info, recs = tf.tf_advance(ctx, h, 0.0, w["T"], w["dt0"], 5000)
    assert info["status"] == tf.TF_ADV_DONE and info["t"] == w["T"]
    assert [r["accepted"] for r in recs] == [r["accepted"] for r in ref.records]
    assert [r["iterations"] for r in recs] == [r["iterations"] for r in ref.records]
    rel = np.max(np.abs(host(h) - ref.h)) / np.max(np.abs(ref.h))
    assert rel <= 1e-10, rel
    # replaying the oracle's accepted steps gives the same film
    acc = ref.accepted()
    h2 = dev(torch, h0)
    info2, _ = tf.tf_advance(ctx, h2, 0.0, 1e30, 1.0, len(acc),
                             dt_replay=[r["dt"] for r in acc],
                             iter_replay=[r["iterations"] for r in acc], records=False)
    assert info2["accepted"] == len(acc)
    assert np.max(np.abs(host(h2) - ref.h)) / np.max(np.abs(ref.h)) <= 1e-10
    assert abs(host(h).sum() - h0.sum()) <= 1e-12 * h0.sum()


def test_small_workload_fp32_bulk(torch):
    """FP32-bulk on the 64^2 run, replaying the FP64 step sizes: mass kept to
    1e-12 and the film within 1e-6 of the FP64 oracle (Newton acts as
    iterative refinement of the FP64-class residual)."""
    w = _workload("small")
    h0 = S.spinodal_film(w["N"], w["N"], w["h0"], w["eps"], w["seed"])
    ref = O.advance(_oracle_model(w), _oracle_control(w), h0, 0.0, w["T"], w["dt0"], 5000)
    acc = ref.accepted()
    ctx = tf.Context(tf.params_for_workload(w, tf.TF_FP32_BULK))
    h = dev(torch, h0)
    info, recs = tf.tf_advance(ctx, h, 0.0, 1e30, 1.0, len(acc),
                               dt_replay=[r["dt"] for r in acc])
    assert info["accepted"] == len(acc)
    hh = host(h)
    assert abs(hh.sum() - h0.sum()) <= 1e-12 * h0.sum()
    assert np.max(np.abs(hh - ref.h)) <= 1e-6
    its32 = sum(r["iterations"] for r in recs)
    its64 = sum(r["iterations"] for r in acc)
    assert its32 <= 1.2 * its64 + 5


def test_scale2k_prefix_parity_fp64(torch):
    """2048^2 on 64 lambda_m, the first 50 step attempts of the adaptive run:
    the same iteration counts and the state within 1e-10 of the oracle."""
    w = _workload("scale2k")
    h0 = S.spinodal_film(w["N"], w["N"], w["h0"], w["eps"], w["seed"])
    ref = O.advance(_oracle_model(w), _oracle_control(w), h0, 0.0, w["T"], w["dt0"], 50)
    ctx = tf.Context(tf.params_for_workload(w, tf.TF_FP64))
    h = dev(torch, h0)
    info, recs = tf.tf_advance(ctx, h, 0.0, w["T"], w["dt0"], 50)
    assert [r["iterations"] for r in recs] == [r["iterations"] for r in ref.records]
    rel = np.max(np.abs(host(h) - ref.h)) / np.max(np.abs(ref.h))
    assert rel <= 1e-10, rel


def test_scale2k_full_run_to_rupture(torch):
    """The plain method at scale in full: 2048^2 on 64 lambda_m, FP64, the
    adaptive controller until min h < 2b (rupture).  Mass stays conserved to
    round-off over the whole run, the run stops on rupture with min h below
    2b, and FP32-bulk replaying the accepted step sizes stays within 1e-6 of
    the FP64 film with the same mass and the same dominant wavenumber.
    Near rupture some replayed steps need more than the 10 iterations FP64
    takes at most (the FP32 solves slow the contraction a little, and the
    large steps there contract slowly already), so the replay may take up
    to 20."""
    w = _workload("scale2k")
    N = w["N"]
    h0 = S.spinodal_film(N, N, w["h0"], w["eps"], w["seed"])
    m0 = float(np.sum(h0))
    ctx = tf.Context(tf.params_for_workload(w, tf.TF_FP64))
    h = dev(torch, h0)
    info, recs = tf.tf_advance(ctx, h, 0.0, w["T"], w["dt0"], 5000)
    assert info["status"] == tf.TF_ADV_RUPTURE, info
    acc = [r for r in recs if r["accepted"]]
    assert len(acc) == info["accepted"] and len(acc) > 100
    assert acc[-1]["hmin"] < 2 * w["b"] <= min(r["hmin"] for r in acc[:-1])
    assert float(torch.min(h)) == acc[-1]["hmin"]
    assert max(abs(r["mass"] - m0) for r in acc) <= 1e-12 * m0
    ctx32 = tf.Context(tf.params_for_workload(w, tf.TF_FP32_BULK, newton_max_iter=20))
    h32 = dev(torch, h0)
    info32, rec32 = tf.tf_advance(ctx32, h32, 0.0, 1e30, 1.0, len(acc), dt_replay=[r["dt"] for r in acc])
    assert info32["accepted"] == len(acc), info32
    assert abs(float(h32.sum()) - m0) <= 1e-6 * m0
    it64 = [r["iterations"] for r in acc]
    it32 = [r["iterations"] for r in rec32]
    print(f"iterations FP64 {sum(it64)} (max {max(it64)}), FP32-bulk {sum(it32)} (max {max(it32)}, "
          f"{sum(i > 10 for i in it32)} steps over 10)")
    assert float(torch.max(torch.abs(h32 - h))) <= 1e-6
    km = 2 * math.pi / w["lambda_m"]
    plan = tf.SpectrumPlan(N, N, w["ds"], tf.tf_spectrum_params_default(H0=w["h0"], q_cut=5 * km))
    k64 = tf.tf_spectrum_run(plan, h, outputs=False)["q_dominant"]
    k32 = tf.tf_spectrum_run(plan, h32, outputs=False)["q_dominant"]
    assert abs(k64 - k32) <= 1e-3 * km
    assert abs(k64 - km) <= 0.25 * km
    print(f"attempts={info['attempts']} accepted={len(acc)} t={info['t']:.1f} hmin={acc[-1]['hmin']:.4f} "
          f"k_dom={k64:.5f} k_m={km:.5f} max|h32-h64|={float(torch.max(torch.abs(h32 - h))):.3e}")


@pytest.mark.parametrize("mode", MODES)
def test_full_size_one_iteration(torch, mode):
    """8192^2 (the benchmark's grid and launch configuration): one Newton
    iteration compared over the whole grid with the oracle."""
    w = _workload("scale8k")
    N = w["N"]
    h0 = S.spinodal_film(N, N, w["h0"], w["eps"], w["seed"])
    dt = w["dt0"]
    ctx = tf.Context(tf.params_for_workload(w, mode))
    hk = dev(torch, h0)
    wv, vv, hn = (torch.empty((N, N), dtype=torch.float64, device="cuda") for _ in range(3))
    info = tf.tf_newton_iteration(ctx, hk, hk, dt, hn, w=wv, v=vv)
    om = _oracle_model(w)
    r = O.newton_iteration(om, h0, O.explicit_part(om, h0, dt), dt)
    sw, sv = np.max(np.abs(r["w"])), np.max(np.abs(r["v"]))
    rt = 1e-11 if mode == tf.TF_FP64 else 2e-4
    assert np.max(np.abs(host(wv) - r["w"])) <= rt * sw
    assert np.max(np.abs(host(vv) - r["v"])) <= rt * sv
    assert np.max(np.abs(host(hn) - r["unew"])) <= 1e-14 + rt * sv
    assert info["gnorm"] == pytest.approx(r["gnorm"], rel=1e-6)


# ----------------------------------------------------------------------------
# edge cases and failure reporting

@pytest.mark.parametrize("mode", MODES)
def test_flat_film(torch, mode):
    om, p = models(33, 17, 2.0, mode)
    ctx = tf.Context(p)
    h = torch.full((17, 33), 0.7, dtype=torch.float64, device="cuda")
    hn = torch.empty_like(h)
    info = tf.tf_newton_adi_step(ctx, h, hn, 50.0)
    assert info["status"] == 0 and info["iterations"] == 1 and info["err"] == 0.0
    assert torch.equal(hn, h)


@pytest.mark.parametrize("mode", MODES)
def test_nonpositive_height_reported(torch, mode):
    om, p = models(16, 16, 1.0, mode)
    ctx = tf.Context(p)
    h0 = np.full((16, 16), 1.0)
    h0[5, 7] = -0.5
    hn = torch.empty((16, 16), dtype=torch.float64, device="cuda")
    info = tf.tf_newton_adi_step(ctx, dev(torch, h0), hn, 1.0)
    assert info["status"] in (tf.TF_STEP_NONPOSITIVE, tf.TF_STEP_ZERO_PIVOT)


def test_rupture_and_replay_failure(torch):
    w = _workload("small")
    h0 = S.spinodal_film(64, 64, 1.0, 0.01, 9)
    p = tf.params_for_workload(w, tf.TF_FP64, rupture_h=0.9999)
    ctx = tf.Context(p)
    h = dev(torch, h0)
    info, recs = tf.tf_advance(ctx, h, 0.0, 1e9, 1.0, 100)
    assert info["status"] == tf.TF_ADV_RUPTURE and recs[-1]["hmin"] < 0.9999
    # a replayed step that cannot converge ends the run with TF_ADV_DT_MIN
    p2 = tf.params_for_workload(w, tf.TF_FP64, newton_max_iter=1, newton_tol=1e-30)
    ctx2 = tf.Context(p2)
    info2, _ = tf.tf_advance(ctx2, dev(torch, h0), 0.0, 1e9, 1.0, 3, dt_replay=[1.0, 1.0, 1.0])
    assert info2["status"] == tf.TF_ADV_DT_MIN and info2["accepted"] == 0


def test_linear_model_mode_amplification(torch):
    nx, ny, ds, dt, eps = 24, 20, 0.7, 0.3, 0.2
    om, p = models(nx, ny, ds, tf.TF_FP64, model=tf.TF_MODEL_LINEAR, c0=1.0, c1=1.0,
                   newton_tol=1e-14, newton_max_iter=200)
    ctx = tf.Context(p)
    u = S.mode_film(nx, ny, ds, 1.0, eps, 2, 3)
    hn = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    info = tf.tf_newton_adi_step(ctx, dev(torch, u), hn, dt)
    ref, ri = O.step(om, O.Control(tol=1e-14, max_iter=200), u, dt)
    assert info["status"] == 0
    assert np.max(np.abs(host(hn) - ref)) <= 1e-13


def test_kappa_from_contact_angle(torch):
    p = tf.tf_params_default(nx=8, ny=8, ds=1.0, kappa=0.0, contact_angle=math.radians(20.0))
    ctx = tf.Context(p)
    assert ctx.kappa == pytest.approx(O.kappa_from_contact_angle(math.radians(20.0), 0.1, 3, 2),
                                      rel=1e-15)


@pytest.mark.parametrize("mode", [tf.TF_FP64, tf.TF_FP32_BULK])
def test_fused_first_iteration_is_bit_identical(torch, mode):
    # a step's first iteration forms b^n and its right side in one kernel
    # (FP32-bulk); tf_newton_iteration forms them in two: the same bits
    nx, ny = 300, 200
    p = tf.tf_params_default(nx=nx, ny=ny, ds=2.0, precision=mode, newton_fixed_iter=1)
    h = torch.from_numpy(S.spinodal_film(nx, ny, 1.0, 0.01, seed=31)).cuda()
    a, b = torch.empty_like(h), torch.empty_like(h)
    ctx = tf.Context(p)
    tf.tf_newton_adi_step(ctx, h, a, 0.5)
    tf.tf_newton_iteration(ctx, h, h, 0.5, b)
    assert torch.equal(a, b)
