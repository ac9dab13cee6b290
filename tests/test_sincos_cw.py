"""The FP32 sine and cosine of the device code (mpt_math.cuh sincos_cw:
Cody-Waite reduction by pi/2 and Taylor series) against float64 references.

The product header is compiled for the host with g++ (the function is plain
C++: fused multiply-adds, rint, floor), so the arithmetic checked here is the
arithmetic the kernels run.
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "paper_2301_06399_gb300", "csrc")

HARNESS = r"""
#include "mpt_math.cuh"
extern "C" void run(const float* x, float* s, float* c, int n) {
  for (int i = 0; i < n; ++i) mpt::sincos_cw(x[i], s[i], c[i]);
}
"""


@pytest.fixture(scope="module")
def sincos_cw(tmp_path_factory):
    d = tmp_path_factory.mktemp("sincos")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    lib = d / "h.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-ffp-contract=off", "-I", HEADER_DIR,
                    "-o", str(lib), str(src)], check=True)
    L = C.CDLL(str(lib))
    L.run.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]

    def f(x):
        x = np.ascontiguousarray(x, np.float32)
        s = np.empty_like(x)
        c = np.empty_like(x)
        L.run(x.ctypes.data, s.ctypes.data, c.ctypes.data, len(x))
        return s, c
    return f


def test_matches_float64_within_two_ulp_on_arc_parameters(sincos_cw):
    # arc parameters: angles within a few turns, plus every quadrant boundary
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.uniform(-4 * np.pi, 4 * np.pi, 200000),
                        (np.arange(-16, 17) * np.pi / 4)]).astype(np.float32)
    s, c = sincos_cw(x)
    xd = x.astype(np.float64)
    es = np.abs(s.astype(np.float64) - np.sin(xd))
    ec = np.abs(c.astype(np.float64) - np.cos(xd))
    # a float's spacing near 1 is 2^-23 (1.19e-7); the results stay within two
    # of it (the reduced argument carries one rounding)
    assert es.max() < 2.4e-7, es.max()
    assert ec.max() < 2.4e-7, ec.max()
    # relative error where the value is not tiny
    big = np.abs(np.sin(xd)) > 1e-3
    assert (es[big] / np.abs(np.sin(xd[big]))).max() < 5e-7


def test_identities_and_special_values(sincos_cw):
    x = np.array([0.0, -0.0, np.pi / 2, np.pi, 1e-20, 1e4, -1e4, np.inf, np.nan], np.float32)
    s, c = sincos_cw(x)
    assert s[0] == 0.0 and c[0] == 1.0
    assert abs(s[2] - 1.0) < 1.2e-7 and abs(c[2]) < 1e-7
    assert abs(s[3]) < 1e-7 and abs(c[3] + 1.0) < 1.2e-7
    assert s[4] == np.float32(1e-20) and c[4] == 1.0
    # large arguments keep |s|^2 + |c|^2 = 1 and agree with float64 to ~1e-6
    for i in (5, 6):
        assert abs(float(s[i]) ** 2 + float(c[i]) ** 2 - 1.0) < 5e-7
        assert abs(float(s[i]) - np.sin(np.float64(x[i]))) < 2e-6
    assert np.isnan(s[7]) and np.isnan(c[7]) and np.isnan(s[8]) and np.isnan(c[8])


def test_pythagoras_and_odd_even_symmetry(sincos_cw):
    x = np.random.default_rng(1).uniform(0, 20, 50000).astype(np.float32)
    s, c = sincos_cw(x)
    sn, cn = sincos_cw(-x)
    assert np.abs(s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1.0).max() < 5e-7
    assert np.array_equal(sn, -s) and np.array_equal(cn, c)
