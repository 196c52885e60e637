"""The FP64 exp of the step kernel (table-driven, after Tang 1989) against the
host's libm exp: within 2 ulp over its range, 0 below -707, +inf above 709,
NaN propagated."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def exp_tab(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("exp") / "libexp.so")
    subprocess.run(["nvcc", "-O3", "-std=c++17", "-gencode=arch=compute_103a,code=sm_103a", "-Xcompiler", "-fPIC",
                    "-shared", "-I", os.path.join(ROOT, "paper_1202_2355_gb300", "csrc"), "-o", so,
                    os.path.join(ROOT, "tests", "kernels", "exp_check.cu")], check=True)
    lib = C.CDLL(so)
    lib.exp_check.restype = C.c_int
    lib.exp_check.argtypes = [C.c_void_p, C.c_void_p, C.c_longlong]

    def f(x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        assert lib.exp_check(x.ctypes.data, y.ctypes.data, x.size) == 0
        return y
    return f


def _ulps(a, b):
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    return np.abs(ia - ib)


def test_within_two_ulp_over_the_range(exp_tab):
    rng = np.random.default_rng(7)
    L = np.log(2.0) / 32
    x = np.concatenate([
        rng.uniform(-707.0, 709.0, 400_000),
        rng.uniform(-1.0, 1.0, 200_000),
        rng.uniform(-1e-6, 1e-6, 50_000),
        # near the reduction breakpoints (N ln2/32 +- ln2/64)
        (np.arange(-2000, 2000) + 0.5) * L,
        np.arange(-2000, 2000) * L,
        np.array([0.0, -0.0, 1.0, -1.0, 700.0, -700.0, 709.0, -706.999]),
    ])
    y = exp_tab(x)
    ref = np.exp(x)
    u = _ulps(y, ref)
    assert u.max() <= 2, (u.max(), x[np.argmax(u)])
    assert np.mean(u == 0) > 0.7


def test_special_values(exp_tab):
    x = np.array([-np.inf, -1e300, -745.2, -708.0, -707.0, np.inf, 710.0, 1e300, np.nan])
    y = exp_tab(x)
    assert np.all(y[:5] == 0.0)
    assert np.all(np.isposinf(y[5:8]))
    assert np.isnan(y[8])


def test_exact_at_zero_and_monotone_near_one(exp_tab):
    assert exp_tab(np.array([0.0]))[0] == 1.0
    x = np.linspace(-1e-3, 1e-3, 20001)
    y = exp_tab(x)
    assert np.all(np.diff(y) >= 0)
