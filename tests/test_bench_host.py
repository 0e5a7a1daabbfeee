"""Host logic of bench.py: which workloads the ncu counters apply to, and the
roofline arithmetic of the bench line (algorithmic bytes per launch and per
Newton iteration, the dominant kernel, traffic only where a capture applies).
No GPU is needed: the timings are the live CUDA-event totals of a default
8192^2 run, typed in."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)

N = 8192
# 200 steps, 1073 Newton iterations; the first iteration of each step has no
# residual launch of its own (the explicit part forms its right side)
TIMING = dict(explicit_launches=200, explicit_ms=197.58, rhs_launches=873, rhs_ms=871.65,
              x_launches=1073, x_ms=792.11, y_launches=1073, y_ms=911.80)
PEAK = dict(hbm_gbs=6798.2, source="measured")


def test_counters_apply_only_to_the_power_law_workloads():
    for name in ("scale8k", "prof4k", "nucl8k", "scale2k"):
        assert bench.ncu_counters_apply(bench.load_workload(name)), name
    for name in ("nlc8k", "pol8k"):
        assert not bench.ncu_counters_apply(bench.load_workload(name)), name


def test_algorithmic_bytes_per_launch():
    tab = bench.kernel_table(dict(timing=TIMING), N, 4)
    cells = N * N
    # pass A: the residual reads u_k and b^n, the x sweep writes w (FP32);
    # pass B: the y sweep reads w and u_k and writes u_{k+1}; the explicit
    # part reads u^n and writes b^n
    assert tab["rhs"][2] == 16 * cells and tab["x_sweep"][2] == 4 * cells
    assert tab["y_sweep"][2] == 20 * cells and tab["explicit"][2] == 16 * cells
    assert bench.kernel_table(dict(timing=TIMING), N, 8)["y_sweep"][2] == 24 * cells


def test_roofline_of_the_dominant_kernel_and_the_iteration():
    traffic = {k: v for k, (v, _) in bench.TRAFFIC_PER_CELL_F32B.items()}
    r = bench.roofline_hbm(dict(timing=TIMING), N, 4, PEAK, traffic)
    assert r["kernel"] == "y_sweep" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    per_ms = 911.80 / 1073
    gbs = 20 * N * N / (per_ms * 1e-3) / 1e9
    assert abs(r["achieved"] - gbs) <= 0.05 and abs(r["frac"] - gbs / 6798.2) <= 5e-5
    assert r["traffic"] == round(traffic["y_sweep"] * N * N)
    # every launch of the Newton loop over the iterations: 16 B/cell per
    # explicit part and per residual, 4 per x sweep, 20 per y sweep
    it_bytes = (200 * 16 + 873 * 16 + 1073 * (4 + 20)) * N * N / 1073
    it_ms = (197.58 + 871.65 + 792.11 + 911.80) / 1073
    assert abs(r["iteration"]["algorithmic_bytes"] - it_bytes) <= 1
    assert abs(r["iteration"]["ms"] - it_ms) <= 5e-5
    assert abs(r["iteration"]["achieved"] - it_bytes / (it_ms * 1e-3) / 1e9) <= 0.05


def test_traffic_is_null_without_a_capture():
    r = bench.roofline_hbm(dict(timing=TIMING), N, 4, PEAK, None)
    assert r["traffic"] is None
    t = dict(TIMING, y_ms=100.0)  # another dominant kernel: the residual
    traffic = {k: v for k, (v, _) in bench.TRAFFIC_PER_CELL_F32B.items()}
    r = bench.roofline_hbm(dict(timing=t), N, 4, PEAK, dict(traffic, rhs=None))
    assert r["kernel"] == "rhs" and r["traffic"] is None


def test_counters_follow_the_kernel_sources(tmp_path):
    """A stored ncu counter is reported only while the device sources of its
    kernel still have the digest it was taken on: editing the residual's
    header nulls the residual's counters and leaves the sweeps' alone."""
    import shutil
    files = sorted({f for v in bench.KERNEL_SOURCES.values() for f in v})
    for f in files:
        shutil.copy(os.path.join(bench.CSRC, f), tmp_path / f)
    table = {k: (1.0 + i, bench.sources_digest(bench.KERNEL_SOURCES[("f32b", k)], str(tmp_path)))
             for i, k in enumerate(("rhs", "explicit", "x_sweep", "y_sweep"))}
    before = bench.current_counters(table, "f32b", str(tmp_path))
    assert before == {"rhs": 1.0, "explicit": 2.0, "x_sweep": 3.0, "y_sweep": 4.0}
    with open(tmp_path / "tf_rhs_packed.cuh", "a") as fh:
        fh.write("// edited\n")
    after = bench.current_counters(table, "f32b", str(tmp_path))
    assert after == {"rhs": None, "explicit": None, "x_sweep": 3.0, "y_sweep": 4.0}
    # a kernel counted on other sources, or never counted, reads null
    assert bench.current_counters({"x_sweep": (5.0, "0" * 16), "y_sweep": (None, None)}, "f32b") == \
        {"x_sweep": None, "y_sweep": None}
