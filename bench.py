"""Benchmark: grid cell-updates per second of the Newton--ADI thin-film step.

Workload (default): the 8192^2 spinodal film on a 64 lambda_m square
(b = 0.1, n = 3, m = 2, contact angle 20 deg, h0 = 1, noise 0.01 U[-1,1]
from seed 1235), Crank--Nicolson, tol 1e-10, K = 10, adaptive dt from 1e-3.
W untimed warm-up steps, then K timed steps.  FP64 mode runs the adaptive
controller and records its step sizes; FP32-bulk mode replays them, so
both modes do the same steps.  The headline value is FP32-bulk:
8192^2 * (accepted steps) / (timed seconds), summed over ranks.

One JSON line on rank 0.  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (each step a 512^2 sample of the same workload).
Under torchrun each rank runs an independent replica of the workload on its
own GPU (the single-grid step has no data-parallel split without a halo
exchange), timed with a barrier and the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = os.path.join(ROOT, "tests", "golden", "workloads.json")


def load_workload(name: str) -> dict:
    with open(WORKLOADS) as f:
        return json.load(f)[name]


def peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured")
    return dict(hbm_gbs=6800.0, source="fallback")


# The FP64 peak of the FP64-mode roofline is measured live by the library's
# FMA throughput probe (tf_probe_fma: 8 independent FMA chains per thread,
# 8 blocks of 256 threads per SM); no measured FP64 figure comes with the
# HBM and bf16 peaks.

# ncu counters per cell, each stored with a digest of the device sources of
# the kernel it was counted on: a counter is reported only while those
# sources are unchanged (current_counters), so an edited kernel reads null
# until it is counted again.
CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1806_10550_gb300", "csrc")
_SWEEP_SOURCES = ["tf_line_sweeps.cuh", "tf_sweeps.cuh", "tf_kernels.cuh", "tf_numeric.cuh"]
KERNEL_SOURCES = {
    ("f32b", "rhs"): ["tf_rhs_packed.cuh", "tf_kernels.cuh", "tf_numeric.cuh"],
    ("f32b", "explicit"): ["tf_rhs_packed.cuh", "tf_kernels.cuh", "tf_numeric.cuh"],
    ("f32b", "x_sweep"): _SWEEP_SOURCES,
    ("f32b", "y_sweep"): _SWEEP_SOURCES,
    ("fp64", "rhs"): ["tf_sweeps.cuh", "tf_kernels.cuh", "tf_numeric.cuh"],
    ("fp64", "x_sweep"): _SWEEP_SOURCES,
    ("fp64", "y_sweep"): _SWEEP_SOURCES,
}


def sources_digest(files, root=CSRC) -> str:
    """First 16 hex digits of the SHA-256 of the named files (name and
    contents, in the order given)."""
    import hashlib
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(root, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def current_counters(table, mode, root=CSRC) -> dict:
    """{kernel: value} from a table of (value, digest) entries, with None for
    a kernel whose sources no longer have the digest it was counted on."""
    return {k: (v if v is not None and d == sources_digest(KERNEL_SOURCES[(mode, k)], root) else None)
            for k, (v, d) in table.items()}


# FP64 operations executed per cell by each FP64-mode kernel (DFMA counted
# as 2, DADD and DMUL as 1), from an ncu capture of the FP64-mode kernels at
# 4096^2 (per cell they do not depend on the grid size).
FP64_FLOPS_PER_CELL = {"rhs": (46.14, "b7f77f9a109008d3"), "x_sweep": (85.91, "1453e94b4cd1b98b"),
                       "y_sweep": (102.91, "1453e94b4cd1b98b")}


class ClockSampler:
    """nvidia-smi clock and throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=mx,
                    reasons=sorted(reasons), samples=len(sm))


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        return rank, world, local, dist
    torch.cuda.set_device(0)
    return 0, 1, 0, None


def barrier(dist):
    import torch
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()


def _reduce(dist, x: float, op) -> float:
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(dist, x: float) -> float:
    return _reduce(dist, x, dist.ReduceOp.MAX) if dist is not None else x


def sum_over_ranks(dist, x: float) -> float:
    return _reduce(dist, x, dist.ReduceOp.SUM) if dist is not None else x


def job_rate(dist, local_units: float, local_ms: float) -> float:
    """Whole-job throughput: units of all ranks / the slowest rank's time."""
    return sum_over_ranks(dist, local_units) / (max_over_ranks(dist, local_ms) * 1e-3)


def run_mode(tf, torch, w, h0, mode, warmup, steps, dist, replay=None, e2e_steps=0, clocks=None):
    """Warm up, then time `steps` step attempts.  Returns a result dict."""
    N = w["N"]
    ctx = tf.Context(tf.params_for_workload(w, mode))
    h = torch.from_numpy(h0).cuda()
    if replay is None:
        info_w, rec_w = tf.tf_advance(ctx, h, 0.0, 1e30, w["dt0"], warmup)
        dt = info_w["dt"]
        t0 = info_w["t"]
    else:
        info_w, rec_w = tf.tf_advance(ctx, h, 0.0, 1e30, 1.0, warmup,
                                      dt_replay=replay[:warmup])
        t0 = info_w["t"]
        dt = 1.0
    h_start = h.clone()  # the e2e pass repeats the timed steps from here
    tf.tf_timing_enable(ctx, True)
    barrier(dist)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    wall0 = time.perf_counter()
    if clocks:
        clocks.__enter__()
    if replay is None:  # the controller continues from the warm-up's state
        info, recs = tf.tf_advance(ctx, h, t0, 1e30, dt, steps, streak=info_w["streak"])
    else:
        info, recs = tf.tf_advance(ctx, h, t0, 1e30, 1.0, steps,
                                   dt_replay=replay[warmup:warmup + steps])
    stop.record()
    torch.cuda.synchronize()
    if clocks:
        clocks.__exit__()
    wall = time.perf_counter() - wall0
    barrier(dist)
    ms = start.elapsed_time(stop)
    timing = tf.tf_timing_get(ctx)
    tf.tf_timing_enable(ctx, False)
    ms = max_over_ranks(dist, ms)
    out = dict(ms=ms, wall_s=wall, info=info, records=recs, timing=timing,
               warm_records=rec_w, final_mass=float(h.sum().item()))
    if e2e_steps > 0:
        # End to end through the public C-ABI call with host buffers: the
        # same accepted steps as the timed region, from the same film; each
        # step copies the film from pinned host memory, steps it, and copies
        # the new film back.
        hh = h_start.cpu().pin_memory()
        hd = torch.empty_like(h)
        hn = torch.empty_like(h)
        out_h = torch.empty_like(hh).pin_memory()
        dts = [r["dt"] for r in recs if r["accepted"]][:e2e_steps]
        barrier(dist)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        acc = 0
        for d in dts:
            hd.copy_(hh, non_blocking=True)
            st = tf.tf_newton_adi_step(ctx, hd, hn, d)
            out_h.copy_(hn, non_blocking=True)
            torch.cuda.current_stream().synchronize()
            hh, out_h = out_h, hh
            acc += st["status"] == 0
        e1.record()
        torch.cuda.synchronize()
        barrier(dist)
        out["e2e_ms"] = max_over_ranks(dist, e0.elapsed_time(e1))
        out["e2e_steps"] = acc
        out["e2e_bytes"] = N * N * 8
    ctx.close()
    return out


def kernel_table(res, N, lp):
    """Per-kernel launches, total duration and algorithmic bytes per launch.

    Algorithmic bytes per cell of one Newton iteration are those of the
    method's two passes: pass A reads u_k (8) and b^n (HP, 8) and writes w
    (LP); pass B reads w (LP) and u_k (8) and writes u_{k+1} (8), i.e. 40 B
    per cell in FP32-bulk and 48 B in FP64.  Pass A runs here as the residual
    kernel (reads u_k and b^n) and the x sweep (writes w); pass B is the y
    sweep.  The explicit part reads u^n and writes b^n (16 B) once per step;
    in tf_advance it also forms the first iteration's right side from the
    same D(u^n), so that iteration has no residual launch.  Everything else
    -- the right side and the FP32 film handed from the residual kernel to
    the sweeps, LU-factor spills, halo re-reads -- is implementation
    traffic, counted by ncu but not in the numerator.
    """
    t = res["timing"]
    cells = N * N
    return {
        "explicit": (t["explicit_launches"], t["explicit_ms"], cells * 16),
        "rhs": (t["rhs_launches"], t["rhs_ms"], cells * 16),
        "x_sweep": (t["x_launches"], t["x_ms"], cells * lp),
        "y_sweep": (t["y_launches"], t["y_ms"], cells * (16 + lp)),
    }


# DRAM bytes (read + write) per cell per launch of each FP32-bulk kernel,
# from an ncu capture of the FP32-bulk kernels at 4096^2 (traffic scales
# with the cells).
TRAFFIC_PER_CELL_F32B = {"rhs": (24.27, "7980ad0cf0226350"), "x_sweep": (31.23, "1453e94b4cd1b98b"),
                         "y_sweep": (44.37, "1453e94b4cd1b98b"), "explicit": (21.68, "7980ad0cf0226350")}


def ncu_counters_apply(w) -> bool:
    """True when workload w runs the kernels that the ncu counters of
    TRAFFIC_PER_CELL_F32B and FP64_FLOPS_PER_CELL were taken on: those of the
    (3, 2) power law.  The other models evaluate their mobilities in other
    code (an out-of-line call per cell, Pi in FP64 inside the residual)."""
    return w.get("model", 0) == 0 and (w["n"], w["m"]) == (3, 2)


def roofline_hbm(res, N, lp_bytes, pk, traffic_per_cell=None):
    """Dominant kernel (largest total time): achieved algorithmic GB/s; plus
    the whole Newton iteration (all three kernels) against the same peak."""
    tab = kernel_table(res, N, lp_bytes)
    name = max(tab, key=lambda k: tab[k][1])
    n, ms, b = tab[name]
    per = ms / max(1, n)
    ach = b / (per * 1e-3) / 1e9
    tpc = (traffic_per_cell or {}).get(name)
    traffic = None if tpc is None else round(tpc * N * N)
    # the whole Newton loop (explicit parts included) per Newton iteration
    iters = max(1, tab["y_sweep"][0])
    it_ms = sum(v[1] for v in tab.values()) / iters
    it_b = sum(v[0] * v[2] for v in tab.values()) / iters
    it_ach = it_b / (it_ms * 1e-3) / 1e9
    return dict(bound="hbm", kernel=name, achieved=round(ach, 1), peak=pk["hbm_gbs"],
                unit="GB/s", frac=round(ach / pk["hbm_gbs"], 4), traffic=traffic,
                ms_per_launch=round(per, 4), algorithmic_bytes_per_launch=b,
                peak_source=pk["source"],
                iteration=dict(ms=round(it_ms, 4), algorithmic_bytes=round(it_b),
                               achieved=round(it_ach, 1), frac=round(it_ach / pk["hbm_gbs"], 4),
                               scope="every kernel of the Newton loop, explicit parts included"))


MODEL_NAMES = {0: "power-law", 1: "linear", 2: "NLC", 3: "polymer"}


def oracle_model(O, w, n):
    """The oracle's model of a workload on an n x n grid (the workload's
    spacing); the NLC and polymer parameters are the paper's sets."""
    return O.Model(nx=n, ny=n, ds=w["ds"], model=w.get("model", 0), kappa=w["kappa"], b=w["b"],
                   n=w["n"], m=w["m"], cap_C=w["cap_C"], theta=w["theta"])


def cpu_baseline_sample(w, h0):
    """FP64 oracle on the host cores: the first time step of the workload."""
    import oracle as O
    O.build()
    N = w["N"]
    M = oracle_model(O, w, N)
    ctl = O.Control(tol=w["tol"], max_iter=w["max_iter"])
    t = time.perf_counter()
    _, info = O.step(M, ctl, h0, w["dt0"])
    el = time.perf_counter() - t
    out = dict(value=N * N / el, unit="cell-updates/s", cores=O.num_threads(), kind="oracle",
               sample=f"one time step (dt={w['dt0']}, {info['iterations']} Newton iterations) "
                      f"of the {N}x{N} film on the host cores, {el:.1f} s")
    # The same oracle on one thread (identical results), one step of a 2048^2
    # film with the workload's parameters and dt.
    n1 = min(N, 2048)
    from paper_1806_10550_gb300 import synthetic as S
    h1 = S.spinodal_film(n1, n1, w["h0"], w["eps"], w["seed"])
    cores = O.num_threads()
    try:
        O.set_num_threads(1)
        t = time.perf_counter()
        _, info1 = O.step(oracle_model(O, w, n1), ctl, h1, w["dt0"])
        el1 = time.perf_counter() - t
    finally:
        O.set_num_threads(cores)
    out["single_thread"] = dict(value=n1 * n1 / el1, unit="cell-updates/s", cores=1,
                                sample=f"one time step ({info1['iterations']} Newton iterations) "
                                       f"of a {n1}x{n1} film, one thread, {el1:.1f} s")
    return out


METRIC = "grid cell-updates/s per Newton-ADI step at 8192^2"


def headline_config(w, world, head="f32b", replayed=True):
    """The bench line's config (shared by both arms)."""
    N = w["N"]
    return dict(workload=(f"{N}x{N} spinodal film, {MODEL_NAMES[w.get('model', 0)]} model, "
                          f"{w['P']} lambda_m square, seed {w['seed']}"),
                mode=("FP32-bulk" if head == "f32b" else "FP64"),
                dt_sequence=("replayed from the FP64 run" if head == "f32b" and replayed
                             else "adaptive"),
                global_batch=world, l2="working set larger than L2 (several 8192^2 grids)",
                parallelism=f"replicas x{world}")


def reference_arm(args, w):
    """The FP64 CPU oracle as the reference arm: each step is one oracle
    time step of a 512^2 sample of the workload (same spacing, same noise)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_1806_10550_gb300 import synthetic as S
    O.build()
    n = 512
    M = oracle_model(O, w, n)
    ctl = O.Control(tol=w["tol"], max_iter=w["max_iter"], dt_min=w["dt_min"],
                    dt_max=w["dt_max"], dt_shrink=w["dt_shrink"], dt_grow=w["dt_grow"],
                    grow_after=w["grow_after"])
    h = S.spinodal_film(n, n, w["h0"], w["eps"], w["seed"])
    res = O.advance(M, ctl, h, 0.0, 1e30, w["dt0"], args.warmup)
    t0 = time.perf_counter()
    res2 = O.advance(M, ctl, res.h, res.t, 1e30, res.dt, args.steps)
    el = time.perf_counter() - t0
    acc = len(res2.accepted())
    value = n * n * acc / el
    line = dict(metric=METRIC, value=value,
                unit="cell-updates/s", n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=el * 1e3 / max(1, args.steps), higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                impl="reference",
                config=dict(headline_config(w, args.gpus, replayed="fp64" in args.modes),
                            sample=f"{n}x{n}"),
                cpu_baseline=dict(value=value, unit="cell-updates/s", cores=O.num_threads(),
                                  kind="oracle",
                                  sample=(f"{acc} accepted FP64 oracle steps of a {n}^2 sample of the "
                                          f"workload (same spacing ds={w['ds']:.6f} and noise), "
                                          f"adaptive dt after {args.warmup} warm-up attempts")),
                e2e=dict(value=value, unit="cell-updates/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line))


def ensemble_params(tf, w, f, mode, solver=0):
    """tf_params of one film of the ensemble workload."""
    import math
    return tf.tf_params_default(
        nx=f["N"], ny=f["N"], ds=f["ds"], b=w["b"], n=w["n"], m=w["m"], kappa=f["kappa"],
        contact_angle=math.radians(f["theta_c_deg"]), theta=w["theta"], newton_tol=w["tol"],
        newton_max_iter=w["max_iter"], dt_min=w["dt_min"], dt_max=f["dt_max"],
        dt_shrink=w["dt_shrink"], dt_grow=w["dt_grow"], grow_after=w["grow_after"], precision=mode,
        line_solver=solver)


ENSEMBLE_METRIC = "film cell-updates/s over a 256-film ensemble"


def ensemble_config(w, A, world):
    sizes = sorted({f["N"] for f in w["films"]})
    return dict(workload=(f"{len(w['films'])} spinodal films, N drawn from {sizes}, contact angle "
                          f"10-40 deg, {w['cells_per_lambda']} cells per lambda_m of each film, "
                          f"{A} attempts each"),
                mode="FP32-bulk", global_batch=len(w["films"]),
                l2="working set larger than L2 (5 GB of films and workspace)",
                parallelism=f"films sharded over {world} rank(s)")


def oracle_ensemble_sample(w, A, budget_s):
    """The FP64 oracle on the host cores: the ensemble's films in order, all
    their attempts, until budget_s seconds of CPU work."""
    import oracle as O
    from paper_1806_10550_gb300 import synthetic as S
    O.build()
    done_cells, el, nf = 0, 0.0, 0
    for f in w["films"]:
        M = O.Model(nx=f["N"], ny=f["N"], ds=f["ds"], kappa=f["kappa"], b=w["b"], n=w["n"], m=w["m"])
        ctl = O.Control(tol=w["tol"], max_iter=w["max_iter"], dt_max=f["dt_max"])
        h = S.spinodal_film(f["N"], f["N"], w["h0"], w["eps"], f["seed"])
        t = time.perf_counter()
        r = O.advance(M, ctl, h, 0.0, 1e30, f["dt0"], A)
        el += time.perf_counter() - t
        done_cells += f["N"] ** 2 * sum(x["accepted"] for x in r.records)
        nf += 1
        if el >= budget_s:
            break
    return dict(value=done_cells / el, unit="cell-updates/s", cores=O.num_threads(), kind="oracle",
                sample=f"the first {nf} film(s) of the ensemble, {A} attempts each, {el:.1f} s")


def reference_ensemble(args, w):
    """The FP64 oracle as the reference arm of the ensemble workload: each
    step the ensemble's films in order until 5 s of CPU work."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    A = w["attempts"]
    K = min(args.steps, 3)
    t0 = time.perf_counter()
    vals = [oracle_ensemble_sample(w, A, 5.0) for _ in range(K)]
    ms = (time.perf_counter() - t0) * 1e3 / K
    value = sum(v["value"] for v in vals) / K
    line = dict(metric=ENSEMBLE_METRIC, value=value, unit="cell-updates/s", n_gpus=args.gpus, steps=K,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=ensemble_config(w, A, args.gpus),
                cpu_baseline=dict(vals[-1], value=value),
                e2e=dict(value=value, unit="cell-updates/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def run_ensemble(args, w):
    """Many independent films of uneven sizes advanced together on one GPU
    (tf_ensemble_advance), against the same films advanced one after another
    (tf_advance).  Films are sharded across ranks (weak scaling)."""
    import torch
    import paper_1806_10550_gb300 as tf
    from paper_1806_10550_gb300 import synthetic as S
    rank, world, local, dist = dist_setup()
    tf.library(build_if_missing=True)
    mode = tf.TF_FP32_BULK
    films = w["films"][rank::world]
    A = args.steps if args.steps != 200 else w["attempts"]
    init = [torch.from_numpy(S.spinodal_film(f["N"], f["N"], w["h0"], w["eps"], f["seed"])).cuda()
            for f in films]
    grids = [torch.empty_like(h) for h in init]
    dt0 = [f["dt0"] for f in films]
    # the line-solver tuner: once per film size, on that size's first film,
    # with as many copies running at once as the ensemble has films of that
    # size (at most 32): the throughput the films will see
    tuned = {}
    count = {}
    for f in films:
        count[f["N"]] = count.get(f["N"], 0) + 1
    for f, h in zip(films, init):
        if f["N"] not in tuned:
            r = tf.tf_tune_line_solver(ensemble_params(tf, w, f, mode, tf.TF_SOLVER_AUTO), h, f["dt0"], iters=5,
                                       copies=min(32, count[f["N"]]))
            tuned[f["N"]] = dict(solver=("partitioned" if r["best"] == tf.TF_SOLVER_PARTITIONED else "twisted"),
                                 copies=min(32, count[f["N"]]),
                                 ms_per_film_iteration=dict(twisted=round(r["ms"][0], 5),
                                                            partitioned=round(r["ms"][1], 5)))

    def contexts(solver):
        return [tf.Context(ensemble_params(tf, w, f, mode, solver), stream=torch.cuda.Stream()) for f in films]

    def reset():
        for g, h in zip(grids, init):
            g.copy_(h)
        torch.cuda.synchronize()

    def timed(ctxs, clocks=None, engine=tf.TF_ENSEMBLE_AUTO):
        # warm-up: W attempts per film, then the timed run from the initial films
        reset()
        tf.tf_ensemble_advance(ctxs, grids, 0.0, 1e30, dt0, args.warmup, engine=engine)
        for c in ctxs:
            tf.tf_timing_enable(c, True)
        reset()
        barrier(dist)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if clocks:
            clocks.__enter__()
        e0.record()
        infos = tf.tf_ensemble_advance(ctxs, grids, 0.0, 1e30, dt0, A, engine=engine)
        e1.record()
        torch.cuda.synchronize()
        if clocks:
            clocks.__exit__()
        barrier(dist)
        return infos, e0.elapsed_time(e1)

    # the fixed shape (every film on the twisted sweeps), then the tuned one
    fixed_ctxs = contexts(tf.TF_SOLVER_TWISTED)
    infos_fixed, ms_fixed = timed(fixed_ctxs)
    cells_fixed = sum(f["N"] ** 2 * i["accepted"] for f, i in zip(films, infos_fixed))
    for c in fixed_ctxs:
        c.close()
    ctxs = contexts(tf.TF_SOLVER_AUTO)
    clocks = ClockSampler(local)
    infos, ms = timed(ctxs, clocks)
    launches = sum(tf.tf_timing_get(c)["launches"] for c in ctxs)
    cells = sum(f["N"] ** 2 * i["accepted"] for f, i in zip(films, infos))
    # the same films and contexts on the host engine (the controller on the
    # host, four threads polling the films' events): the same decisions
    infos_h, ms_h = timed(ctxs, engine=tf.TF_ENSEMBLE_HOST)
    assert infos_h == infos
    iters = sum(i["newton_iterations"] for i in infos)
    value = job_rate(dist, cells, ms)
    # the same films, one after another
    reset()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    seq = [tf.tf_advance(c, g, 0.0, 1e30, d, A, records=False)[0] for c, g, d in zip(ctxs, grids, dt0)]
    e3.record()
    torch.cuda.synchronize()
    ms_seq = e2.elapsed_time(e3)
    assert [i["accepted"] for i in seq] == [i["accepted"] for i in infos]
    cs = clocks.summary()
    line = dict(
        metric=ENSEMBLE_METRIC,
        value=value, unit="cell-updates/s", n_gpus=world, steps=A, warmup=args.warmup,
        ms_per_step=ms / max(1, A), higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32 solves + f32x2 double-float residual, f64 state", data="synthetic",
        config=ensemble_config(w, A, world),
        accepted_steps=sum(i["accepted"] for i in infos), newton_iterations=iters,
        sequential_value=job_rate(dist, cells, ms_seq), speedup_vs_sequential=ms_seq / ms,
        fixed_shape_value=job_rate(dist, cells_fixed, ms_fixed),
        engine="graph: each film's whole run one CUDA graph launch, Newton and step control on the device",
        host_engine_value=job_rate(dist, cells, ms_h),
        line_solver_by_size={str(k): v for k, v in sorted(tuned.items())},
        gpu_launches=launches,
        clocks=dict(sm_mhz=cs["sm_mhz"], sm_max_mhz=cs["sm_max_mhz"], reasons=cs["reasons"]),
    )
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_ensemble_sample(w, A, 10.0)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


SPECTRUM_METRIC = "film cells analysed/s, radial Fourier analysis at 8192^2"


def spectrum_film(w):
    from paper_1806_10550_gb300 import synthetic as S
    N = w["N"]
    qm = 2 * math.pi / w["lambda_m"]
    return S.ring_film(N, N, w["ds"], w["h0"], w["eps"], qm, w["spread"], w["modes"], w["noise"],
                       seed=w["seed"])


def spectrum_config(w, world):
    N = w["N"]
    return dict(workload=(f"{N}x{N} ring film about q_m ({w['modes']} modes, noise {w['noise']}), "
                          f"spacing lambda_m/{round(w['lambda_m'] / w['ds'])}, q_cut = 5 q_m, "
                          f"sigma {w['sigma']}, {w['points_per_interval']} points per interval, "
                          f"{w['n_eval']} samples"),
                global_batch=world, l2="input larger than L2 (512 MiB film)",
                parallelism=f"replicas x{world}")


def oracle_spectrum(w, h):
    """One oracle analysis of the whole film; returns (seconds, result)."""
    import oracle.radial_fourier as RF
    t = time.perf_counter()
    r = RF.analyse(h, w["ds"], w["h0"], w["q_cut"], w["sigma"], w["points_per_interval"], w["n_eval"])
    return time.perf_counter() - t, r


def run_spectrum(args, w):
    """The radial Fourier analysis of an 8192^2 film per step (all ten
    kernels), the film resident in HBM; e2e adds the copy of the film from
    pinned host memory and the read-back of the dominant maximum."""
    import torch
    import paper_1806_10550_gb300 as tf
    rank, world, local, dist = dist_setup()
    tf.library(build_if_missing=True)
    N = w["N"]
    h_host = torch.from_numpy(spectrum_film(w)).pin_memory()
    h = h_host.cuda()
    sp = tf.tf_spectrum_params_default(H0=w["h0"], q_cut=w["q_cut"], sigma=w["sigma"],
                                       points_per_interval=w["points_per_interval"],
                                       n_eval=w["n_eval"])
    stream = torch.cuda.current_stream()
    plan = tf.SpectrumPlan(N, N, w["ds"], sp, stream)
    for _ in range(args.warmup):
        tf.tf_spectrum_run(plan, h, outputs=False)
    K = args.steps if args.steps != 200 else w["steps"]
    names = ["rows", "cols", "smooth_p", "smooth_q", "radial", "fit"]
    kms = [0.0] * 6
    barrier(dist)
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clocks:
        e0.record(stream)
        for _ in range(K):
            info = tf.tf_spectrum_run(plan, h, outputs=False)
            kms = [a + b for a, b in zip(kms, tf.tf_spectrum_timing(plan))]
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(dist)
    ms = e0.elapsed_time(e1)
    value = job_rate(dist, N * N * K, ms)
    # end to end: film from pinned host memory, result read back (inside the call)
    hd = torch.empty_like(h)
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    e2.record(stream)
    for _ in range(K):
        hd.copy_(h_host, non_blocking=True)
        info_e = tf.tf_spectrum_run(plan, hd, outputs=False)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3)
    assert info_e["q_dominant"] == info["q_dominant"]
    pi = plan.info()
    Pb = min(N, pi["n_p"] + math.ceil(3 * w["sigma"]))
    per = {n: kms[i] / K for i, n in enumerate(names)}
    dom = max(per, key=per.get)
    # algorithmic bytes of the row transform: the film read once (8 B/cell)
    # and the narrow FP32 block of wave indices written (4 B x N x Pb)
    rows_bytes = N * N * 8 + N * Pb * 4
    pk = peaks()
    ach = rows_bytes / (per["rows"] * 1e-3) / 1e9
    qm = 2 * math.pi / w["lambda_m"]
    line = dict(
        metric=SPECTRUM_METRIC, value=value, unit="cells/s", n_gpus=world, steps=K,
        warmup=args.warmup, ms_per_step=ms / K, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f32 transform, f64 smoothing, grouping and fit",
        data="synthetic", config=spectrum_config(w, world),
        q_dominant=info["q_dominant"], q_m=qm, n_radii=pi["n_radii"], n_intervals=pi["n_intervals"],
        n_peaks=info["n_peaks"], kernel_ms_per_step={k: round(v, 4) for k, v in per.items()},
        roofline=dict(bound="hbm", kernel="rows", achieved=round(ach, 1), peak=pk["hbm_gbs"],
                      unit="GB/s", frac=round(ach / pk["hbm_gbs"], 4), traffic=None,
                      ms_per_launch=round(per["rows"], 4), algorithmic_bytes_per_launch=rows_bytes,
                      peak_source=pk["source"], dominant_kernel=dom),
        gpu_launches=10 * K,
        e2e=dict(value=job_rate(dist, N * N * K, ms_e2e), unit="cells/s",
                 h2d_bytes_per_step=N * N * 8, d2h_bytes_per_step=4 + 16),
    )
    cs = clocks.summary()
    line["clocks"] = dict(sm_mhz=cs["sm_mhz"], sm_max_mhz=cs["sm_max_mhz"], reasons=cs["reasons"])
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        el, r = oracle_spectrum(w, h_host.numpy())
        line["cpu_baseline"] = dict(value=N * N / el, unit="cells/s", cores=O.num_threads(),
                                    kind="oracle",
                                    sample=f"one oracle analysis of the whole {N}x{N} film, {el:.1f} s")
        line["oracle_q_dominant"] = r["q_dominant"]
    if rank == 0:
        print(json.dumps(line))
    plan.close()
    if dist is not None:
        dist.destroy_process_group()


def reference_spectrum(args, w):
    """The oracle's radial Fourier analysis as the reference arm: each step
    one analysis of the whole 8192^2 film on the host cores."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle as O
    h = spectrum_film(w)
    for _ in range(min(args.warmup, 1)):
        oracle_spectrum(w, h)
    K = min(args.steps, 3)
    el = 0.0
    for _ in range(K):
        dt, r = oracle_spectrum(w, h)
        el += dt
    N = w["N"]
    value = N * N * K / el
    line = dict(metric=SPECTRUM_METRIC, value=value, unit="cells/s", n_gpus=args.gpus, steps=K,
                warmup=args.warmup, ms_per_step=el * 1e3 / K, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=spectrum_config(w, args.gpus),
                cpu_baseline=dict(value=value, unit="cells/s", cores=O.num_threads(), kind="oracle",
                                  sample=f"{K} oracle analysis(es) of the whole {N}x{N} film"),
                e2e=dict(value=value, unit="cells/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


ADJOINT_METRIC = ("adjoint film cell-steps/s: gradient of |h(T) - h_target|^2 over 400 fixed steps "
                  "(3 Newton iterations each, forward + checkpointed reverse) at 1024^2")

# Algorithmic bytes per cell of one launch of each adjoint kernel group:
# the transposed solve reads the five band diagonals and the right side and
# writes the solution (56 B); a line derivative reads u_k, w, lambda and
# updates the cotangent (40 B); the D derivative the same without w (32 B).
# The per-iterate tables, the elimination scratch and the Laplacian
# cotangent pass are implementation traffic.
ADJ_BYTES_PER_CELL = {"solve_t": 56.0, "line_x": 40.0, "line_y": 40.0, "D": 32.0}


def adjoint_config(w, world):
    N = w["N"]
    return dict(workload=(f"{N}x{N} spinodal film, power-law model, {w['P']} lambda_m square, "
                          f"seed {w['seed']}, {w['steps']} steps of dt {w['dt_fixed']} with "
                          f"{w['fixed_iter']} Newton iterations unrolled; loss |h(T) - h_target|^2, "
                          f"h_target from seed {w['target_seed']}; gradient in h(0) and theta_c; "
                          f"checkpoints every ceil(sqrt({w['steps']})) steps"),
                mode="FP64", global_batch=world,
                l2="working set larger than L2 (about 400 grids of 8 MiB: checkpoints, two banks of iterates)",
                parallelism=f"replicas x{world}")


def oracle_adjoint_sample(w, n=12):
    """The oracle's adjoint (complex-step Jacobian, transposed) of one step
    on an n x n sample of the workload (same spacing, dt and noise)."""
    import oracle as O
    import oracle.adjoint as AD
    from paper_1806_10550_gb300 import synthetic as S
    M = O.Model(nx=n, ny=n, ds=w["ds"], kappa=w["kappa"], b=w["b"], n=w["n"], m=w["m"], cap_C=w["cap_C"],
                theta=w["theta"])
    u = S.spinodal_film(n, n, w["h0"], w["eps"], w["seed"])
    g = np.random.default_rng(1).standard_normal((n, n))
    t = time.perf_counter()
    AD.vjp(M, u, w["dt_fixed"], w["fixed_iter"], g)
    return time.perf_counter() - t, n


def run_adjoint(args, w):
    """The adjoint workload, one timed step = one loss gradient: the tape's
    forward over the trajectory (checkpoints kept), the loss cotangent
    2 (h(T) - h_target), and the checkpointed reverse; grids resident in
    HBM.  e2e adds the H2D copy of the initial film from pinned memory and
    the D2H copy of the gradient."""
    import torch
    import paper_1806_10550_gb300 as tf
    from paper_1806_10550_gb300 import synthetic as S
    rank, world, local, dist = dist_setup()
    tf.library(build_if_missing=True)
    if args.traj_steps > 0:
        w = dict(w, steps=args.traj_steps)
    N, K, dt, ns = w["N"], w["fixed_iter"], w["dt_fixed"], w["steps"]
    p = tf.params_for_workload(w, tf.TF_FP64)
    p.kappa, p.contact_angle = 0.0, w["theta_c"]  # kappa from the contact angle
    ctx = tf.Context(p)
    tape = tf.tf_tape_create(ctx, ns, K, dt)
    tinfo = tf.tf_tape_info(tape)
    h_host = torch.from_numpy(S.spinodal_film(N, N, w["h0"], w["eps"], w["seed"])).pin_memory()
    h = h_host.cuda()
    target = tf.tf_tape_forward(tape, torch.from_numpy(
        S.spinodal_film(N, N, w["h0"], w["eps"], w["target_seed"])).cuda()).clone()
    hT, gh = torch.empty_like(h), torch.empty_like(h)

    def gradient(h0):
        tf.tf_tape_forward(tape, h0, hT)
        return tf.tf_tape_backward(tape, 2.0 * (hT - target), g_h0=gh)

    for _ in range(args.warmup):
        gradient(h)
    S_ = args.steps if args.steps != 200 else 1
    groups = {k: 0.0 for k in tf.TAPE_GROUPS}
    barrier(dist)
    clocks = ClockSampler(local)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with clocks:
        e0.record()
        for _ in range(S_):
            r = gradient(h)
            for k, v in tf.tf_tape_timing(tape).items():
                groups[k] += v
        e1.record()
        torch.cuda.synchronize()
    barrier(dist)
    ms = e0.elapsed_time(e1)
    value = job_rate(dist, N * N * ns * S_, ms)
    # end to end from pinned host memory
    hd, out = torch.empty_like(h), torch.empty_like(h_host).pin_memory()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    for _ in range(S_):
        hd.copy_(h_host, non_blocking=True)
        gradient(hd)
        out.copy_(gh, non_blocking=True)
    e3.record()
    torch.cuda.synchronize()
    ms_e2e = e2.elapsed_time(e3)
    # the forward's kernels one by one: one more gradient, untimed, with the
    # context's kernel timing on (it waits after every iteration to read its
    # events, so it stays out of the timed region; the launches are the same)
    tf.tf_timing_enable(ctx, True)
    gradient(h)
    tim = tf.tf_timing_get(ctx)
    tf.tf_timing_enable(ctx, False)
    # the dominant kernel over both halves: the forward's FP64 kernels (the
    # tape's forward and the segments run again) and the reverse's groups
    # (the tape's timing, from the timed region)
    per = {k: v / S_ for k, v in groups.items()}
    fwd = kernel_table(dict(timing=tim), N, 8)
    rev_launches = {"solve_t": 2 * K * ns, "line_x": K * ns, "line_y": K * ns, "D": (K + 1) * ns}
    cand = {k: (n_, ms_, b) for k, (n_, ms_, b) in fwd.items()}
    cand.update({k: (rev_launches[k], per[k], ADJ_BYTES_PER_CELL[k] * N * N) for k in rev_launches})
    dom = max(cand, key=lambda k: cand[k][1])
    n_l, ms_k, bytes_l = cand[dom]
    ms_launch = ms_k / max(1, n_l)
    pk = peaks()
    ach = bytes_l / (ms_launch * 1e-3) / 1e9
    roof = dict(bound="hbm", kernel=dom, unit="GB/s", peak=pk["hbm_gbs"], peak_source=pk["source"],
                ms_per_launch=round(ms_launch, 4), achieved=round(ach, 1), frac=round(ach / pk["hbm_gbs"], 4),
                algorithmic_bytes_per_launch=int(bytes_l), traffic=None,
                kernel_ms_per_step={k: round(v[1], 1) for k, v in cand.items()})
    line = dict(
        metric=ADJOINT_METRIC, value=value, unit="cell-steps/s", n_gpus=world, steps=S_, warmup=args.warmup,
        ms_per_step=ms / S_, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
        data="synthetic", config=adjoint_config(w, world), g_theta=r["g_theta"], g_kappa=r["g_kappa"],
        checkpoints=dict(every=tinfo["every"], count=tinfo["checkpoints"], tape_bytes=tinfo["bytes"]),
        group_ms_per_step={k: round(v, 1) for k, v in per.items()}, roofline=roof,
        # the forward kernels as the context counts them in one gradient;
        # the reverse per step and iteration 1 tables, 2 band, 2 solve, 2
        # line and 1 D derivative, 3 Laplacian-transpose and 2 axpy kernels,
        # then 1 axpy, 1 D derivative and 1 Laplacian-transpose
        gpu_launches=S_ * (tim["launches"] + ns * (13 * K + 3)),
        e2e=dict(value=job_rate(dist, N * N * ns * S_, ms_e2e), unit="cell-steps/s",
                 h2d_bytes_per_step=N * N * 8, d2h_bytes_per_step=N * N * 8),
    )
    cs = clocks.summary()
    line["clocks"] = dict(sm_mhz=cs["sm_mhz"], sm_max_mhz=cs["sm_max_mhz"], reasons=cs["reasons"])
    if rank == 0 and not args.no_cpu_baseline:
        import oracle as O
        el, n = oracle_adjoint_sample(w)
        line["cpu_baseline"] = dict(value=n * n / el, unit="cell-steps/s", cores=O.num_threads(), kind="oracle",
                                    sample=(f"the oracle's adjoint of one step of a {n}x{n} sample "
                                            f"(complex-step Jacobian: {n * n} forward steps), {el:.1f} s"))
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def reference_adjoint(args, w):
    """The oracle's adjoint as the reference arm: each step one oracle adjoint
    of one time step of a 12 x 12 sample of the workload (cell-steps/s)."""
    if int(os.environ.get("RANK", "0")) != 0:
        return
    import oracle as O
    K = min(args.steps, 3)
    el = 0.0
    for _ in range(K):
        dt_, n = oracle_adjoint_sample(w)
        el += dt_
    value = n * n * K / el
    line = dict(metric=ADJOINT_METRIC, value=value, unit="cell-steps/s", n_gpus=args.gpus, steps=K,
                warmup=args.warmup, ms_per_step=el * 1e3 / K, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=adjoint_config(w, args.gpus),
                cpu_baseline=dict(value=value, unit="cell-steps/s", cores=O.num_threads(), kind="oracle",
                                  sample=f"{K} oracle adjoint(s) of a {n}x{n} sample"),
                e2e=dict(value=value, unit="cell-steps/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scale8k")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="steps of the end-to-end pass (default: all timed steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--traj-steps", type=int, default=0,
                    help="adjoint workload: trajectory length (default: the workload's; shorter for profiles)")
    ap.add_argument("--modes", default="fp64,f32b")
    args = ap.parse_args()
    w = load_workload(args.workload)
    if args.workload == "spectrum8k":
        (reference_spectrum if args.impl == "reference" else run_spectrum)(args, w)
        return
    if args.workload == "adjoint1k":
        (reference_adjoint if args.impl == "reference" else run_adjoint)(args, w)
        return
    if args.workload == "ensemble" and args.impl == "reference":
        reference_ensemble(args, w)
        return
    if args.workload == "ensemble" and args.impl == "ours":
        # one hardware work queue per stream (up to 32) before CUDA starts,
        # so that the films' streams do not share queues
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        run_ensemble(args, w)
        return
    if args.impl == "reference":
        reference_arm(args, w)
        return
    import torch
    import paper_1806_10550_gb300 as tf
    from paper_1806_10550_gb300 import synthetic as S
    rank, world, local, dist = dist_setup()
    if args.e2e_steps < 0:
        args.e2e_steps = args.steps
    tf.library(build_if_missing=True)
    N = w["N"]
    h0 = S.spinodal_film(N, N, w["h0"], w["eps"], w["seed"])
    pk = peaks()
    modes = args.modes.split(",")
    res = {}
    clocks = ClockSampler(local)
    if "fp64" in modes:
        res["fp64"] = run_mode(tf, torch, w, h0, tf.TF_FP64, args.warmup, args.steps, dist)
        replay = [r["dt"] for r in res["fp64"]["warm_records"] + res["fp64"]["records"]
                  if r["accepted"]]
    else:
        replay = None
    if "f32b" in modes:
        if replay is not None and len(replay) >= args.warmup + args.steps:
            res["f32b"] = run_mode(tf, torch, w, h0, tf.TF_FP32_BULK, args.warmup, args.steps,
                                   dist, replay=replay, e2e_steps=args.e2e_steps, clocks=clocks)
        else:
            res["f32b"] = run_mode(tf, torch, w, h0, tf.TF_FP32_BULK, args.warmup, args.steps,
                                   dist, e2e_steps=args.e2e_steps, clocks=clocks)
    head = "f32b" if "f32b" in res else "fp64"
    R = res[head]
    profiled = ncu_counters_apply(w)
    acc_local = R["info"]["accepted"]
    acc_all = sum_over_ranks(dist, acc_local)
    value = N * N * acc_all / (R["ms"] * 1e-3)
    lp = 4 if head == "f32b" else 8
    line = dict(
        metric=METRIC,
        value=value, unit="cell-updates/s", n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=R["ms"] / max(1, R["info"]["attempts"]), higher_is_better=True,
        scaling="weak", vs_baseline=None,
        dtype=("f32 solves + f32x2 double-float residual, f64 state" if head == "f32b" else "f64"),
        data="synthetic",
        config=headline_config(w, world, head, replayed="fp64" in res),
        accepted_steps=acc_local, attempts=R["info"]["attempts"],
        newton_iterations=R["info"]["newton_iterations"],
        cell_iterations_per_s=N * N * R["info"]["newton_iterations"] * world / (R["ms"] * 1e-3),
        roofline=roofline_hbm(R, N, lp, pk,
                              current_counters(TRAFFIC_PER_CELL_F32B, "f32b") if head == "f32b" and profiled else None),
        gpu_launches=R["timing"]["launches"],
        kernel_ms=dict(explicit=R["timing"]["explicit_ms"], rhs=R["timing"]["rhs_ms"],
                       x_sweep=R["timing"]["x_ms"], y_sweep=R["timing"]["y_ms"]),
    )
    if "e2e_ms" in R:
        line["e2e"] = dict(value=N * N * R["e2e_steps"] * world / (R["e2e_ms"] * 1e-3),
                           unit="cell-updates/s", h2d_bytes_per_step=R["e2e_bytes"],
                           d2h_bytes_per_step=R["e2e_bytes"], steps=R["e2e_steps"])
    alu = dict(fp64_tflops=tf.tf_probe_fma(tf.TF_FP64), fp32_tflops=tf.tf_probe_fma(tf.TF_FP32_BULK),
               source="measured live by tf_probe_fma (2 flops per FMA)")
    line["alu_peaks"] = {k: (round(v, 3) if isinstance(v, float) else v) for k, v in alu.items()}
    if "fp64" in res:
        F = res["fp64"]
        FP64_TFLOPS = alu["fp64_tflops"]
        v64 = N * N * sum_over_ranks(dist, F["info"]["accepted"]) / (F["ms"] * 1e-3)
        t = F["timing"]
        per = (t["rhs_ms"] + t["x_ms"] + t["y_ms"]) / max(1, t["x_launches"])
        # FP64 mode is bound by the FP64 pipe: executed FP64 flops of the
        # dominant kernel (and of the iteration's three kernels) over their
        # live CUDA-event time
        kt = {"rhs": (t["rhs_launches"], t["rhs_ms"]), "x_sweep": (t["x_launches"], t["x_ms"]),
              "y_sweep": (t["y_launches"], t["y_ms"])}
        dom64 = max(kt, key=lambda k: kt[k][1])
        n64, ms64 = kt[dom64]
        fl64 = current_counters(FP64_FLOPS_PER_CELL, "fp64")
        profiled = profiled and all(v is not None for v in fl64.values())
        ach64 = fl64[dom64] * N * N * n64 / (ms64 * 1e-3) / 1e12 if profiled else None
        it_fl = sum(fl64[k] * kt[k][0] for k in kt) * N * N if profiled else None
        it_ms = sum(kt[k][1] for k in kt)
        line["fp64"] = dict(value=v64, ms_per_step=F["ms"] / max(1, F["info"]["attempts"]),
                            accepted_steps=F["info"]["accepted"],
                            newton_iterations=F["info"]["newton_iterations"],
                            ms_per_iteration=per,
                            roofline=None if not profiled else dict(bound="alu", unit="TFLOP/s", peak=round(FP64_TFLOPS, 4),
                                          peak_source="measured live by tf_probe_fma",
                                          kernel=dom64, flops_per_cell=fl64[dom64],
                                          ms_per_launch=round(ms64 / max(1, n64), 4),
                                          achieved=round(ach64, 4), frac=round(ach64 / FP64_TFLOPS, 4),
                                          flops="executed FP64 operations per cell counted by ncu (DFMA = 2)",
                                          iteration=dict(
                                              achieved=round(it_fl / (it_ms * 1e-3) / 1e12, 4),
                                              frac=round(it_fl / (it_ms * 1e-3) / 1e12 / FP64_TFLOPS, 4),
                                              scope="residual, x and y sweeps (explicit parts excluded)")))
        if head == "f32b":
            line["speedup_f32b_vs_fp64"] = value / v64
    cs = clocks.summary()
    line["clocks"] = dict(sm_mhz=cs["sm_mhz"], sm_max_mhz=cs["sm_max_mhz"], reasons=cs["reasons"])
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(w, h0)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
