"""CPU tests of the FP32-bulk numeric layer (tf_numeric.cuh, host build).

The kernels and these tests compile the same header, so the integer
conversions and the double-float arithmetic are checked here against exact
NumPy float64 arithmetic without a GPU.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.abspath(os.path.join(os.path.dirname(__file__), ".."))
SRC = os.path.join(ROOT, "paper_1806_10550_gb300", "csrc", "tf_numeric_host.cpp")
HDR = os.path.join(ROOT, "paper_1806_10550_gb300", "csrc", "tf_numeric.cuh")
LIB = os.path.join(ROOT, "paper_1806_10550_gb300", "_build", "libtfnumeric_host.so")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if (not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(SRC),
                                                                os.path.getmtime(HDR))):
        subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
                        "-x", "c++", SRC, "-o", LIB], check=True)
    return C.CDLL(LIB)


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def test_f32_trunc(lib):
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-10, 10, 1000), [0.0, -0.0, 1.0, 1e-40, 1e40, np.inf, -np.inf]])
    y = np.empty(x.size, np.float32)
    lib.tfh_f32_trunc_of_f64(_p(x), _p(y), C.c_long(x.size))
    fin = np.abs(x) < 1e30
    big = (np.abs(x) >= 1e-37) & fin
    # truncation toward zero: |y| <= |x| and within one float ulp
    assert np.all(np.abs(y[big].astype(np.float64)) <= np.abs(x[big]))
    assert np.all(np.abs(x[big] - y[big]) <= np.spacing(np.abs(y[big]).astype(np.float32)))
    assert y[-4] == 0.0 and np.isinf(y[-3]) and np.isinf(y[-2]) and y[-1] == -np.inf


def test_df_of_f64_is_48_bit_accurate(lib):
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(0.01, 5, 5000), -rng.uniform(1e-6, 1e3, 2000),
                        rng.standard_normal(2000) * 1e-7])
    hi = np.empty(x.size, np.float32)
    lo = np.empty(x.size, np.float32)
    lib.tfh_df_of_f64(_p(x), _p(hi), _p(lo), C.c_long(x.size))
    rec = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.all(np.abs(rec - x) <= 2.0 ** -48 * np.abs(x))
    assert np.all(np.abs(lo) <= np.spacing(np.abs(hi)))


def test_f64_of_f32_exact_is_the_conversion(lib):
    """The integer widening of the y sweep's Newton update gives the bits of
    the native float -> double conversion for every one of the 2^32 float
    bit patterns, and NumPy's widening on named values."""
    f = lib.tfh_f64_of_f32_exact_mismatches
    f.restype = C.c_long
    f.argtypes = [C.c_ulonglong, C.c_ulonglong]
    assert f(0, 1 << 32) == 0
    x = np.array([0.0, -0.0, 1.0, -1.0, 1.5, 3.4028235e38, -1.1754944e-38, 1.1754942e-38, 1e-45,
                  np.inf, -np.inf, 0.1, -2.5e-7], np.float32)
    y = np.empty(x.size)
    lib.tfh_f64_of_f32_exact(_p(x), _p(y), C.c_long(x.size))
    assert y.view(np.uint64).tolist() == x.astype(np.float64).view(np.uint64).tolist()


def test_f64_add_f32_rounds_to_nearest(lib):
    rng = np.random.default_rng(2)
    n = 20000
    u = rng.uniform(0.05, 3, n) * rng.choice([-1, 1], n)
    scale = 10.0 ** rng.uniform(-14, 0.5, n)
    v = (rng.standard_normal(n) * scale * np.abs(u)).astype(np.float32)
    v[:50] = 0.0
    v[50:100] = -u[50:100].astype(np.float32)  # near-total cancellation
    y = np.empty(n)
    lib.tfh_f64_add_f32(_p(u), _p(v), _p(y), C.c_long(n))
    exact = u + v.astype(np.float64)  # exact in float64 except the final rounding
    # compare to the correctly rounded sum computed in higher precision
    ld = np.longdouble
    ex = (u.astype(ld) + v.astype(ld))
    err = np.abs(y.astype(ld) - ex)
    ulp = np.spacing(np.abs(exact)).astype(ld)
    assert np.all(err <= 0.5 * ulp + (ulp * ld(1e-3)))
    assert np.all(y[:50] == u[:50])


def test_df_arithmetic(lib):
    rng = np.random.default_rng(3)
    a = rng.uniform(0.1, 4, 4000)
    b = a * (1 + rng.uniform(-1e-3, 1e-3, 4000))  # close values: cancellation
    s, p, r = (np.empty(4000) for _ in range(3))
    lib.tfh_df_ops(_p(a), _p(b), _p(s), _p(p), _p(r), C.c_long(4000))
    assert np.all(np.abs(s - (a - b)) <= 2.0 ** -46 * np.abs(a))
    assert np.all(np.abs(p - a * b) <= 2.0 ** -45 * np.abs(a * b))
    assert np.all(np.abs(r - 1 / a) <= 2.0 ** -45 / a)


def test_fixed_point_mass(lib):
    u = np.array([0.0, 1.0, 0.5, 3.25, 1e-12, 100.0, -1.0])
    q = np.empty(u.size, np.int64)
    lib.tfh_fixed36(_p(u), _p(q), C.c_long(u.size))
    assert list(q[:4]) == [0, 2 ** 36, 2 ** 35, 13 * 2 ** 34]
    assert q[4] == round(1e-12 * 2 ** 36) and q[5] == 100 * 2 ** 36 and q[6] == 0


def test_fast_positive_conversions(lib):
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(1e-3, 50, 20000), 10.0 ** rng.uniform(-22, 38, 5000),
                        [1.0, 0.5, 2.0, 1.0 + 2.0 ** -52]])
    f, hi, lo = (np.empty(x.size, np.float32) for _ in range(3))
    lib.tfh_fast_conv(_p(x), _p(f), _p(hi), _p(lo), C.c_long(x.size))
    ref = np.empty(x.size, np.float32)
    lib.tfh_f32_trunc_of_f64(_p(x), _p(ref), C.c_long(x.size))
    assert np.array_equal(f, ref)  # same truncation as the general routine
    assert np.array_equal(hi, ref)
    rec = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.all(np.abs(rec - x) <= 2.0 ** -48 * x)
