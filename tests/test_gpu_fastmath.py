"""The library's hand-written FP64 reciprocal, rsqrt and sqrt (FP32 hardware seed +
one Newton-Raphson step) and its integer-pipe f64<->f32 conversions, checked against
CUDA's IEEE operations on the GPU over the full exponent range used by the scheme."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2409_16053_gb300 import build
    so = str(tmp_path_factory.mktemp("fm") / "fastmath_check.so")
    subprocess.run([build.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3",
                    "-std=c++17", "-fmad=false", "-shared", "-Xcompiler", "-fPIC",
                    os.path.join(HERE, "fastmath_check.cu"), "-o", so], check=True)
    L = ctypes.CDLL(so)
    L.fastmath_eval.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.ratio_eval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    L.gratio_eval.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                              ctypes.c_void_p]
    return L


def test_fastmath_against_ieee(lib):
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.uniform(1.0, 2.0, 20000),
        10.0 ** rng.uniform(-300, 300, 20000) * rng.choice([-1, 1], 20000),
        10.0 ** rng.uniform(-30, 30, 20000),
        np.array([1.0, 2.0, 0.5, 3.0, 1e-12, 1e12, 1.0 - 2 ** -52, 1.0 + 2 ** -52]),
        # mantissas next to the binade edges of 1/m and 1/sqrt(m), and with large low parts
        2.0 - rng.uniform(0, 2 ** -20, 5000), 1.0 + rng.uniform(0, 2 ** -20, 5000),
        4.0 - rng.uniform(0, 2 ** -18, 5000), 1.0 + (2 ** 23 - 1) * 2 ** -23 + rng.uniform(0, 2 ** -23, 5000),
        2.0 ** rng.integers(-1000, 1000, 5000) * (2.0 - 2.0 ** -52),
    ]).astype(np.float64)
    out = np.empty((x.size, 9))
    assert lib.fastmath_eval(x.ctypes.data, x.size, out.ctypes.data) == 0
    rel = lambda a, b: np.abs(a - b) / np.abs(b)
    # one Newton step from a ~2^-22 seed: relative error below 2^-42
    assert rel(out[:, 0], out[:, 1]).max() < 2.0 ** -42
    assert rel(out[:, 2], out[:, 3]).max() < 2.0 ** -42
    assert rel(out[:, 4], out[:, 5]).max() < 2.0 ** -42
    # f64 -> f32 on the integer pipe: within one float ulp of round-to-nearest
    inr = (np.abs(x) > 1.2e-38) & (np.abs(x) < 3.0e38)
    assert (rel(out[inr, 6], out[inr, 7]) <= 2.0 ** -23).all()
    assert not np.any(out[~inr & (np.abs(x) < 1e-38), 6])        # flush to zero
    assert np.all(np.isnan(out[~inr & (np.abs(x) > 3.5e38), 6]))  # out of range -> NaN
    # f32 -> f64 is exact
    assert not np.any(out[inr, 8])


def test_sqrt_ratio_against_ieee(lib):
    """sqrt(a / b) (the sound speed sqrt(gamma p / rho)) from split mantissas: within
    2^-42 of the IEEE expression over the scheme's range, odd and even exponent
    differences, mantissa ratios on both sides of 1 and next to the binade edges
    (including ratios just below 4, whose seed can land above 2); the IEEE results for
    zero, negative and non-finite inputs."""
    rng = np.random.default_rng(1)
    n = 40000
    a = np.concatenate([10.0 ** rng.uniform(-30, 30, n), rng.uniform(1.0, 2.0, n),
                        2.0 - rng.uniform(0, 2 ** -20, 2000), 1.0 + rng.uniform(0, 2 ** -20, 2000),
                        2.0 ** rng.integers(-500, 500, 2000) * (2.0 - 2.0 ** -52),
                        (4.0 - rng.uniform(0, 2 ** -19, 2000)) * 4.0 ** rng.integers(-20, 20, 2000)])
    b = np.concatenate([10.0 ** rng.uniform(-30, 30, n), rng.uniform(1.0, 2.0, n),
                        1.0 + rng.uniform(0, 2 ** -20, 2000), 2.0 - rng.uniform(0, 2 ** -20, 2000),
                        2.0 ** rng.integers(-500, 500, 2000) * (1.0 + 2.0 ** -52),
                        1.0 + rng.uniform(0, 2 ** -20, 2000)])
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty((a.size, 2))
    assert lib.ratio_eval(a.ctypes.data, b.ctypes.data, a.size, out.ctypes.data) == 0
    assert (np.abs(out[:, 0] - out[:, 1]) / out[:, 1]).max() < 2.0 ** -42
    s = np.array([0.0, -1.0, np.inf, np.nan, 1.0, 1.0])
    t = np.array([1.0, 1.0, 1.0, 1.0, 0.0, -1.0])
    o = np.empty((s.size, 2))
    assert lib.ratio_eval(s.ctypes.data, t.ctypes.data, s.size, o.ctypes.data) == 0
    assert np.array_equal(o[:, 0], o[:, 1], equal_nan=True)


@pytest.mark.parametrize("g", [5.0 / 3.0, 1.4, 4.0 / 3.0, 1.0001, 2.0, 1.1, 7.0 / 5.0 + 1e-9])
def test_sqrt_gratio_against_ieee(lib, g):
    """sqrt(g a / b) (the sound speed with gamma split into two floats): within 2^-42 of
    the IEEE expression for the adiabatic indices in use, ratios across the binade edges
    of g a / b, and the IEEE results for zero, negative and non-finite inputs."""
    rng = np.random.default_rng(2)
    n = 40000
    a = np.concatenate([10.0 ** rng.uniform(-30, 30, n), rng.uniform(1.0, 2.0, n),
                        2.0 - rng.uniform(0, 2 ** -20, 2000), 1.0 + rng.uniform(0, 2 ** -20, 2000),
                        # g a / b next to a power of four (the square root's binade edges)
                        4.0 ** rng.integers(-20, 20, 4000) / g * (1.0 + rng.uniform(-2 ** -20, 2 ** -20, 4000))])
    b = np.concatenate([10.0 ** rng.uniform(-30, 30, n), rng.uniform(1.0, 2.0, n),
                        1.0 + rng.uniform(0, 2 ** -20, 2000), 2.0 - rng.uniform(0, 2 ** -20, 2000),
                        np.ones(4000)])
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty((a.size, 2))
    assert lib.gratio_eval(a.ctypes.data, b.ctypes.data, a.size, g, out.ctypes.data) == 0
    assert (np.abs(out[:, 0] - out[:, 1]) / out[:, 1]).max() < 2.0 ** -42
    s = np.array([0.0, -1.0, np.inf, np.nan, 1.0, 1.0])
    t = np.array([1.0, 1.0, 1.0, 1.0, 0.0, -1.0])
    o = np.empty((s.size, 2))
    assert lib.gratio_eval(s.ctypes.data, t.ctypes.data, s.size, g, o.ctypes.data) == 0
    assert np.array_equal(o[:, 0], o[:, 1], equal_nan=True)
