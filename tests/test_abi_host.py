"""CPU checks of the C ABI: the library builds, loads and exports every
function that include/tf.h declares; ctypes structs match the C layout;
argument validation rejects bad input before any GPU work."""
import ctypes as C
import os
import re
import subprocess

import pytest

import paper_1806_10550_gb300 as tf

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
HDR = os.path.join(ROOT, "include", "tf.h")


def declared_functions():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tf_[a-z0-9_]+)\s*\(", src)))


def test_header_functions_exported():
    L = tf.library()
    names = declared_functions()
    assert "tf_init" in names and "tf_advance" in names
    for n in names:
        assert hasattr(L, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", tf._LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (tf_\w+)", out))
    assert set(names) <= exported, set(names) - exported


def _c_layout():
    prog = r'''
#include <stdio.h>
#include <stddef.h>
#include "tf.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("tf_params %zu\ntf_step_info %zu\ntf_step_record %zu\ntf_advance_info %zu\ntf_norms %zu\n",
         sizeof(tf_params), sizeof(tf_step_info), sizeof(tf_step_record), sizeof(tf_advance_info),
         sizeof(tf_norms));
  O(tf_params, ds); O(tf_params, kappa); O(tf_params, theta); O(tf_params, newton_fixed_iter);
  O(tf_params, grow_after); O(tf_params, rupture_h); O(tf_params, precision);
  O(tf_params, nlc_K); O(tf_params, nlc_w); O(tf_params, pol_C); O(tf_params, pol_d);
  O(tf_params, line_solver);
  O(tf_step_record, accepted); O(tf_step_record, hmin); O(tf_advance_info, dt);
  printf("tf_spectrum_params %zu\ntf_spectrum_info %zu\ntf_spectrum_out %zu\n",
         sizeof(tf_spectrum_params), sizeof(tf_spectrum_info), sizeof(tf_spectrum_out));
  O(tf_spectrum_params, sigma); O(tf_spectrum_params, n_eval);
  O(tf_spectrum_info, n_peaks); O(tf_spectrum_info, q_dominant); O(tf_spectrum_info, value_dominant);
  O(tf_spectrum_out, curve_value); O(tf_spectrum_out, peak_value); O(tf_spectrum_out, peak_cap);
  return 0;
}
'''
    d = os.path.join(ROOT, "paper_1806_10550_gb300", "_build")
    os.makedirs(d, exist_ok=True)
    src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
    open(src, "w").write(prog)
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), src, "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return dict(line.rsplit(" ", 1) for line in out.strip().splitlines())


def test_struct_layouts_match_header():
    lay = {k: int(v) for k, v in _c_layout().items()}
    assert lay["tf_params"] == C.sizeof(tf.TfParams)
    assert lay["tf_step_info"] == C.sizeof(tf.TfStepInfo)
    assert lay["tf_step_record"] == C.sizeof(tf.TfStepRecord)
    assert lay["tf_advance_info"] == C.sizeof(tf.TfAdvanceInfo)
    assert lay["tf_norms"] == C.sizeof(tf.TfNorms)
    assert lay["tf_spectrum_params"] == C.sizeof(tf.TfSpectrumParams)
    assert lay["tf_spectrum_info"] == C.sizeof(tf.TfSpectrumInfo)
    assert lay["tf_spectrum_out"] == C.sizeof(tf.TfSpectrumOut)
    for key, v in lay.items():
        if "." in key:
            T, f = key.split(".")
            cls = {"tf_params": tf.TfParams, "tf_step_record": tf.TfStepRecord,
                   "tf_advance_info": tf.TfAdvanceInfo, "tf_spectrum_params": tf.TfSpectrumParams,
                   "tf_spectrum_info": tf.TfSpectrumInfo, "tf_spectrum_out": tf.TfSpectrumOut}[T]
            assert getattr(cls, f).offset == v, key


def test_params_default():
    p = tf.tf_params_default()
    assert p.model == tf.TF_MODEL_POWERLAW and p.n == 3 and p.m == 2 and p.b == 0.1
    assert p.theta == 0.5 and p.newton_tol == 1e-10 and p.newton_max_iter == 10
    assert p.precision == tf.TF_FP64 and p.nx == 0
    assert p.line_solver == tf.TF_SOLVER_TWISTED


@pytest.mark.parametrize("bad", [dict(nx=0), dict(ny=-3), dict(ds=0.0), dict(theta=1.5),
                                 dict(newton_max_iter=0), dict(precision=7), dict(model=9),
                                 dict(n=2, m=2), dict(b=-1.0), dict(dt_shrink=1.0),
                                 dict(nx=70000, ny=70000), dict(nx=65537, ny=1), dict(nx=1, ny=65537),
                                 dict(nx=65536, ny=32768), dict(nx=46341, ny=46341),
                                 dict(line_solver=3), dict(line_solver=-1),
                                 # the partitioned solver: FP32-bulk with the (3, 2) power law only
                                 dict(line_solver=1),
                                 dict(line_solver=1, precision=1, n=4),
                                 dict(line_solver=1, precision=1, model=1)])
def test_init_rejects_bad_parameters(bad):
    p = tf.tf_params_default(nx=16, ny=16, ds=1.0)
    for k, v in bad.items():
        setattr(p, k, v)
    h = C.c_void_p(123)
    rc = tf.library().tf_init(C.byref(p), None, C.byref(h))
    assert rc == tf.TF_ERR_ARG
    assert h.value is None


def test_null_arguments_rejected():
    L = tf.library()
    assert L.tf_init(None, None, None) == tf.TF_ERR_ARG
    assert L.tf_newton_adi_step(None, None, None, 1.0, None) == tf.TF_ERR_ARG
    assert L.tf_residual(None, None, None, 1.0, None, None) == tf.TF_ERR_ARG
    assert L.tf_advance(None, None, 0.0, 1.0, 1.0, 1, None, None, None, None, None) == tf.TF_ERR_ARG
    assert tf.tf_strerror(tf.TF_ERR_ARG) == "invalid argument"
    L.tf_destroy(None)
    out = C.c_void_p(123)
    assert L.tf_tape_create(None, 10, 3, 0.01, 0, C.byref(out)) == tf.TF_ERR_ARG
    assert out.value is None
    assert L.tf_tape_create(None, 10, 3, 0.01, 0, None) == tf.TF_ERR_ARG
    assert L.tf_tape_info(None, None, None, None, None) == tf.TF_ERR_ARG
    assert L.tf_tape_forward(None, None, None) == tf.TF_ERR_ARG
    assert L.tf_tape_backward(None, None, None, None, None) == tf.TF_ERR_ARG
    assert L.tf_tape_timing(None, None, 0) == tf.TF_ERR_ARG
    L.tf_tape_destroy(None)
    # the ensemble call: a negative count, and an engine that does not exist
    assert L.tf_ensemble_advance(-1, None, None, None, None, None, None, None, None, tf.TF_ENSEMBLE_AUTO) == tf.TF_ERR_ARG
    assert L.tf_ensemble_advance(0, None, None, None, None, None, None, None, None, 7) == tf.TF_ERR_ARG


def test_tuner_and_probe_refuse_bad_arguments():
    """The line-solver tuner, its table and the FMA probe refuse their bad
    arguments on the host, before any device work."""
    L = tf.library()
    p = tf.tf_params_default(nx=64, ny=64, ds=1.0)
    best, ms = C.c_int(-7), (C.c_double * 2)(-3.0, -3.0)
    fake = C.c_void_p(16)  # never dereferenced: every call below is refused first
    for args in ((None, None, fake, 0.1, 1, 1),     # no parameters
                 (C.byref(p), None, None, 0.1, 1, 1),  # no film
                 (C.byref(p), None, fake, 0.1, 0, 1),  # no timed round
                 (C.byref(p), None, fake, 0.1, 1, 0),  # no copy
                 (C.byref(p), None, fake, 0.1, 1, 257),  # too many copies
                 (C.byref(p), None, fake, 0.0, 1, 1),  # dt not positive
                 (C.byref(p), None, fake, float("nan"), 1, 1),
                 (C.byref(p), None, fake, float("inf"), 1, 1)):
        assert L.tf_tune_line_solver(*args, C.byref(best), ms) == tf.TF_ERR_ARG, args
    assert L.tf_tune_line_solver(C.byref(p), None, fake, 0.1, 1, 1, None, ms) == tf.TF_ERR_ARG
    assert best.value == -7 and list(ms) == [-3.0, -3.0]
    # nothing tuned for this shape in this process; NULLs read as "none"
    assert L.tf_tuned_line_solver(C.byref(p)) == -1
    assert L.tf_tuned_line_solver(None) == -1
    assert L.tf_line_solver(None) == -1
    out = C.c_double(-1.0)
    assert L.tf_probe_fma(tf.TF_FP64, None, None) == tf.TF_ERR_ARG
    assert L.tf_probe_fma(5, None, C.byref(out)) == tf.TF_ERR_ARG
    assert out.value == -1.0


def test_no_cpu_fallback_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError, match="CUDA device is required"):
        tf.Context(tf.tf_params_default(nx=8, ny=8, ds=1.0))


def test_spectrum_params_default():
    sp = tf.tf_spectrum_params_default()
    assert sp.H0 == 1.0 and sp.q_cut == 0.0 and sp.sigma == 1.0
    assert sp.points_per_interval == 10 and sp.n_eval == 400


@pytest.mark.parametrize("nx,ny,ds,bad", [
    (48, 64, 1.0, {}), (64, 0, 1.0, {}), (32768, 64, 1.0, {}), (64, 64, 0.0, {}),
    (64, 64, 1.0, dict(q_cut=0.0)), (64, 64, 1.0, dict(q_cut=float("inf"))),
    (64, 64, 1.0, dict(sigma=-1.0)), (64, 64, 1.0, dict(sigma=17.0)),
    (64, 64, 1.0, dict(points_per_interval=0)), (64, 64, 1.0, dict(n_eval=2)),
    (64, 64, 1.0, dict(n_eval=5000)), (64, 64, 1.0, dict(H0=float("nan"))),
    (16384, 16384, 1.0, dict(q_cut=1e6)),  # more than 2^27 keys
])
def test_spectrum_plan_rejects_bad_arguments(nx, ny, ds, bad):
    sp = tf.tf_spectrum_params_default(q_cut=1.0)
    for k, v in bad.items():
        setattr(sp, k, v)
    h = C.c_void_p(123)
    assert tf.library().tf_spectrum_plan_create(nx, ny, ds, C.byref(sp), None, C.byref(h)) == tf.TF_ERR_ARG
    assert h.value is None
    L = tf.library()
    assert L.tf_spectrum_run(None, None, None, None) == tf.TF_ERR_ARG
    assert L.tf_spectrum_plan_info(None, None) == tf.TF_ERR_ARG
    L.tf_spectrum_plan_destroy(None)
