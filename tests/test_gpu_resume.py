"""Resumable step control (Fig. FlowChartTime): a run split over several
calls, each handed the previous call's time, step size and accept streak,
must make the same decisions and leave the same bits as one call.

The 64^2 workload (4 lambda_m, adaptive dt from 1e-3) is advanced for 200
attempts in one tf_advance call and in two calls split near attempt 100, in
both precision modes: records (t, dt, accepted, iterations), the next dt and the film must
be identical.  The same split of tf_ensemble_advance over three films must
give each film the bits of the unsplit ensemble.
"""
import json
import os

import numpy as np
import pytest

import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu

W = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "workloads.json")))


@pytest.fixture(scope="module")
def torch():
    import torch as T
    if not T.cuda.is_available():
        pytest.skip("no CUDA device")
    tf.library()
    return T


def _rec_key(r):
    return (r["t"], r["dt"], r["accepted"], r["iterations"], r["status"])


@pytest.mark.parametrize("mode", [tf.TF_FP64, tf.TF_FP32_BULK])
def test_two_calls_of_100_equal_one_call_of_200(torch, mode):
    w = W["small"]
    h0 = S.spinodal_film(w["N"], w["N"], w["h0"], w["eps"], w["seed"])
    ctx = tf.Context(tf.params_for_workload(w, mode))
    h1 = torch.from_numpy(h0).cuda()
    info1, rec1 = tf.tf_advance(ctx, h1, 0.0, w["T"], w["dt0"], 200)
    assert info1["attempts"] == 200
    # split near attempt 100, inside a streak (so that dropping it would
    # change the run)
    for split in range(100, 110):
        h2 = torch.from_numpy(h0).cuda()
        ia, ra = tf.tf_advance(ctx, h2, 0.0, w["T"], w["dt0"], split)
        if ia["streak"] > 0:
            break
    assert 0 < ia["streak"] < w["grow_after"]
    ib, rb = tf.tf_advance(ctx, h2, ia["t"], w["T"], ia["dt"], 200 - split, streak=ia["streak"])
    assert [_rec_key(r) for r in ra + rb] == [_rec_key(r) for r in rec1]
    assert (ib["t"], ib["dt"], ib["streak"]) == (info1["t"], info1["dt"], info1["streak"])
    assert ia["accepted"] + ib["accepted"] == info1["accepted"]
    assert torch.equal(h1, h2)
    # without the streak the second half grows dt at other attempts
    h3 = torch.from_numpy(h0).cuda()
    ic, _ = tf.tf_advance(ctx, h3, 0.0, w["T"], w["dt0"], split)
    _, rd = tf.tf_advance(ctx, h3, ic["t"], w["T"], ic["dt"], 200 - split)
    assert [r["dt"] for r in rd] != [r["dt"] for r in rb]
    ctx.close()


def test_split_ensemble_equals_unsplit(torch):
    w = W["small"]
    films, ctxs, streams = [], [], []
    for k, n in enumerate((64, 48, 40)):
        films.append(S.spinodal_film(n, n, w["h0"], w["eps"], w["seed"] + k))
        p = tf.params_for_workload(dict(w, N=n), tf.TF_FP32_BULK)
        s = torch.cuda.Stream()
        streams.append(s)
        ctxs.append(tf.Context(p, stream=s))
    dt0 = [w["dt0"]] * 3
    ga = [torch.from_numpy(f).cuda() for f in films]
    one = tf.tf_ensemble_advance(ctxs, ga, 0.0, w["T"], dt0, 120)
    gb = [torch.from_numpy(f).cuda() for f in films]
    first = tf.tf_ensemble_advance(ctxs, gb, 0.0, w["T"], dt0, 70)
    second = tf.tf_ensemble_advance(ctxs, gb, [i["t"] for i in first], w["T"], [i["dt"] for i in first], 50,
                                    streak=[i["streak"] for i in first])
    torch.cuda.synchronize()
    for a, b, c, x, y in zip(one, first, second, ga, gb):
        assert (c["t"], c["dt"], c["streak"]) == (a["t"], a["dt"], a["streak"])
        assert b["accepted"] + c["accepted"] == a["accepted"]
        assert b["newton_iterations"] + c["newton_iterations"] == a["newton_iterations"]
        assert torch.equal(x, y)
    for c in ctxs:
        c.close()
