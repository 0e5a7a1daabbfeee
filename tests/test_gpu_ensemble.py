"""Ensembles of independent films (tf_ensemble_advance): every film must
come out exactly as tf_advance leaves it -- the same attempts, decisions,
iteration counts and bit-identical grids -- and, through that, match the
oracle.  Films of one ensemble may use different line solvers (the tuner
picks one per grid shape); each solver's films match the oracle."""
import math

import numpy as np
import pytest

import oracle as O
import paper_1806_10550_gb300 as tf
from paper_1806_10550_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


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


# (nx, ny, contact angle [deg], seed, dt0 factor, t_end factor, attempts);
# times in units of 1/sigma_max of the film's own flat state
FILMS = [
    (32, 24, 12.0, 1, 1e-3, 1e30, 25),
    (48, 48, 20.0, 2, 1e-3, 1e30, 30),
    (64, 40, 35.0, 3, 5.0, 1e30, 20),      # starts too large: rejections
    (17, 33, 27.0, 4, 1e-3, 2e-3, 40),     # reaches t_end (clipped last step)
    (96, 80, 16.0, 5, 1e-2, 1e30, 15),
    (1, 40, 22.0, 6, 1e-3, 1e30, 20),
    (40, 1, 22.0, 7, 1e-3, 1e30, 0),       # no attempts at all
]


def film_params(nx, ny, th, mode, solver=tf.TF_SOLVER_TWISTED):
    kappa = O.kappa_from_contact_angle(math.radians(th), 0.1, 3, 2)
    qm, sm = O.lsa(O.Model(nx=1, ny=1, ds=1.0, kappa=kappa), 1.0)
    ds = 2 * math.pi / qm / 8
    p = tf.tf_params_default(nx=nx, ny=ny, ds=ds, contact_angle=math.radians(th), precision=mode,
                             line_solver=solver)
    return p, sm, kappa, ds


@pytest.mark.parametrize("mode,mixed", [(tf.TF_FP64, False), (tf.TF_FP32_BULK, False), (tf.TF_FP32_BULK, True)])
def test_ensemble_matches_per_film_advance(torch, mode, mixed):
    ctxs, grids, h0s, t_end, dt0, att, params = [], [], [], [], [], [], []
    for i, (nx, ny, th, seed, fdt, fend, na) in enumerate(FILMS):
        # mixed: every other film on the partitioned solver
        solver = tf.TF_SOLVER_PARTITIONED if mixed and i % 2 else tf.TF_SOLVER_TWISTED
        p, sm, _, _ = film_params(nx, ny, th, mode, solver)
        h = S.spinodal_film(nx, ny, 1.0, 0.01, seed=seed)
        ctxs.append(tf.Context(p, stream=torch.cuda.Stream()))
        grids.append(dev(torch, h))
        h0s.append(h)
        t_end.append(fend / sm)
        dt0.append(fdt / sm)
        att.append(na)
        params.append(p)
    infos = tf.tf_ensemble_advance(ctxs, grids, 0.0, t_end, dt0, att)
    torch.cuda.synchronize()
    for i, (info, g) in enumerate(zip(infos, grids)):
        ctx = tf.Context(params[i])
        ref = dev(torch, h0s[i])
        rinfo, _ = tf.tf_advance(ctx, ref, 0.0, t_end[i], dt0[i], att[i], records=False)
        assert info == rinfo, (i, info, rinfo)
        assert np.array_equal(host(g), host(ref)), i
    # the films exercise the paths they were chosen for
    assert infos[2]["attempts"] > infos[2]["accepted"]          # rejections
    assert infos[3]["status"] == tf.TF_ADV_DONE                  # reached t_end
    assert infos[3]["t"] == t_end[3]
    assert infos[6]["attempts"] == 0


def test_graph_engine_matches_host_engine(torch):
    """The graph engine (each film's run one CUDA graph, its controller on
    the device) against the host engine on the same FP32-bulk films: the
    same infos and bit-identical grids, over a first call and a second call
    on the same contexts (the graphs reused) that continues from the first
    call's t, dt and streak."""
    runs = {}
    for engine in (tf.TF_ENSEMBLE_HOST, tf.TF_ENSEMBLE_AUTO):
        ctxs, grids, t_end, dt0, att = [], [], [], [], []
        for nx, ny, th, seed, fdt, fend, na in FILMS:
            p, sm, _, _ = film_params(nx, ny, th, tf.TF_FP32_BULK)
            ctxs.append(tf.Context(p, stream=torch.cuda.Stream()))
            grids.append(dev(torch, S.spinodal_film(nx, ny, 1.0, 0.01, seed=seed)))
            t_end.append(fend / sm)
            dt0.append(fdt / sm)
            att.append(na)
        for c in ctxs:
            tf.tf_timing_enable(c, True)
        first = tf.tf_ensemble_advance(ctxs, grids, 0.0, t_end, dt0, att, engine=engine)
        g1 = [host(g).copy() for g in grids]
        timing = [tf.tf_timing_get(c) for c in ctxs]
        second = tf.tf_ensemble_advance(ctxs, grids, [i["t"] for i in first], t_end, [i["dt"] for i in first],
                                        [max(1, a // 2) for a in att], streak=[i["streak"] for i in first],
                                        engine=engine)
        runs[engine] = (first, g1, second, [host(g) for g in grids], timing)
    h1, hg1, h2, hg2, ht = runs[tf.TF_ENSEMBLE_HOST]
    a1, ag1, a2, ag2, at = runs[tf.TF_ENSEMBLE_AUTO]
    assert a1 == h1 and a2 == h2
    for i in range(len(FILMS)):
        assert np.array_equal(ag1[i], hg1[i]), i
        assert np.array_equal(ag2[i], hg2[i]), i
        # which engine ran: the graph engine counts launches but times no kernel
        if FILMS[i][6] > 0:
            assert at[i]["launches"] > 0 and at[i]["x_launches"] == 0, (i, at[i])
            assert ht[i]["x_launches"] > 0, (i, ht[i])
    assert sum(i["attempts"] for i in a2) > 0


def test_graph_engine_stops_as_tf_advance(torch):
    """The graph engine's other exits, each against the host engine: a film
    that ruptures (min h below rupture_h after its first accepted step), one
    whose step size falls below dt_min after rejections, and one on a fixed
    iteration count."""
    def film(engine, mutate, fdt):
        p, sm, _, _ = film_params(40, 32, 25.0, tf.TF_FP32_BULK)
        mutate(p, sm)
        ctx = tf.Context(p, stream=torch.cuda.Stream())
        g = dev(torch, S.spinodal_film(40, 32, 1.0, 0.01, seed=11))
        info = tf.tf_ensemble_advance([ctx], [g], 0.0, 1e30, fdt / sm, 30, engine=engine)[0]
        return info, host(g)

    def rupture(p, sm):
        p.rupture_h = 0.999

    def dt_floor(p, sm):  # one iteration never meets the tolerance: 5, 2.5, 1.25, then 0.625 < dt_min
        p.newton_max_iter = 1
        p.dt_min = 1.0 / sm

    def fixed(p, sm):
        p.newton_fixed_iter = 3

    for mutate, fdt, status in ((rupture, 1e-3, tf.TF_ADV_RUPTURE), (dt_floor, 5.0, tf.TF_ADV_DT_MIN),
                                (fixed, 1e-3, None)):
        ih, gh = film(tf.TF_ENSEMBLE_HOST, mutate, fdt)
        ia, ga = film(tf.TF_ENSEMBLE_AUTO, mutate, fdt)
        assert ia == ih, (mutate.__name__, ia, ih)
        assert np.array_equal(ga, gh), mutate.__name__
        if status is not None:
            assert ia["status"] == status, (mutate.__name__, ia)
        else:
            assert ia["newton_iterations"] == 3 * ia["attempts"] > 0


def test_ensemble_film_matches_oracle(torch):
    nx, ny, th, seed, fdt, fend, na = FILMS[2]
    p, sm, kappa, ds = film_params(nx, ny, th, tf.TF_FP64)
    h = S.spinodal_film(nx, ny, 1.0, 0.01, seed=seed)
    others = [FILMS[0], FILMS[4]]
    ctxs = [tf.Context(p, stream=torch.cuda.Stream())]
    grids = [dev(torch, h)]
    for onx, ony, oth, osd, _, _, _ in others:
        op, _, _, _ = film_params(onx, ony, oth, tf.TF_FP64)
        ctxs.append(tf.Context(op, stream=torch.cuda.Stream()))
        grids.append(dev(torch, S.spinodal_film(onx, ony, 1.0, 0.01, seed=osd)))
    infos = tf.tf_ensemble_advance(ctxs, grids, 0.0, 1e30, [fdt / sm, 1e-3 / sm, 1e-2 / sm], na)
    om = O.Model(nx=nx, ny=ny, ds=ds, kappa=kappa)
    ref = O.advance(om, O.Control(), h, 0.0, 1e30, fdt / sm, na)
    assert infos[0]["attempts"] == len(ref.records)
    assert infos[0]["accepted"] == sum(r["accepted"] for r in ref.records)
    assert infos[0]["newton_iterations"] == sum(r["iterations"] for r in ref.records)
    assert np.max(np.abs(host(grids[0]) - ref.h)) <= 1e-10


def test_ensemble_rejects_shared_context(torch):
    p, sm, _, _ = film_params(16, 16, 20.0, tf.TF_FP64)
    ctx = tf.Context(p)
    g1 = dev(torch, S.spinodal_film(16, 16, 1.0, 0.01, seed=1))
    g2 = dev(torch, S.spinodal_film(16, 16, 1.0, 0.01, seed=2))
    with pytest.raises(RuntimeError):
        tf.tf_ensemble_advance([ctx, ctx], [g1, g2], 0.0, 1e30, 1e-3 / sm, 3)


@pytest.mark.parametrize("solver", [tf.TF_SOLVER_TWISTED, tf.TF_SOLVER_PARTITIONED])
def test_fp32_bulk_solvers_match_oracle_replay(torch, solver):
    """An FP32-bulk film of 150 x 70 cells (three x segments and three y
    segments of the partitioned solver) replaying the oracle's accepted
    steps ends within Newton-tolerance level of the FP64 oracle, with
    either line solver."""
    nx, ny, th, seed = 150, 70, 25.0, 8
    p, sm, kappa, ds = film_params(nx, ny, th, tf.TF_FP32_BULK, solver)
    h = S.spinodal_film(nx, ny, 1.0, 0.01, seed=seed)
    om = O.Model(nx=nx, ny=ny, ds=ds, kappa=kappa)
    ref = O.advance(om, O.Control(), h, 0.0, 1e30, 1e-3 / sm, 12)
    acc = ref.accepted()
    assert len(acc) >= 8
    ctx = tf.Context(p)
    assert ctx.line_solver == solver
    g = dev(torch, h)
    info, _ = tf.tf_advance(ctx, g, 0.0, 1e30, 1.0, len(acc), dt_replay=[r["dt"] for r in acc],
                            records=False)
    assert info["accepted"] == len(acc)
    assert np.max(np.abs(host(g) - ref.h)) <= 1e-9


def test_tuner_picks_a_solver_per_shape_and_auto_contexts_follow_it(torch):
    picks = {}
    for n in (64, 256):
        p, sm, _, _ = film_params(n, n, 20.0, tf.TF_FP32_BULK, tf.TF_SOLVER_AUTO)
        assert tf.tf_tuned_line_solver(p) in (-1, tf.TF_SOLVER_TWISTED, tf.TF_SOLVER_PARTITIONED)
        h = dev(torch, S.spinodal_film(n, n, 1.0, 0.01, seed=n))
        h_before = h.clone()
        r = tf.tf_tune_line_solver(p, h, 1e-3 / sm, iters=2, copies=1 if n == 64 else 4)
        assert torch.equal(h, h_before)  # the film is only read
        assert r["best"] in (tf.TF_SOLVER_TWISTED, tf.TF_SOLVER_PARTITIONED)
        assert r["ms"][0] > 0.0 and r["ms"][1] > 0.0
        assert r["best"] == (tf.TF_SOLVER_PARTITIONED if r["ms"][1] < r["ms"][0] else tf.TF_SOLVER_TWISTED)
        assert tf.tf_tuned_line_solver(p) == r["best"]
        assert tf.Context(p).line_solver == r["best"]
        picks[n] = r["best"]
    # FP64 has one solver: the tuner reports the other as not applicable
    p, sm, _, _ = film_params(32, 32, 20.0, tf.TF_FP64, tf.TF_SOLVER_AUTO)
    r = tf.tf_tune_line_solver(p, dev(torch, S.spinodal_film(32, 32, 1.0, 0.01, seed=1)), 1e-3 / sm, iters=1)
    assert r["best"] == tf.TF_SOLVER_TWISTED and r["ms"][1] == -1.0
    assert tf.Context(p).line_solver == tf.TF_SOLVER_TWISTED
