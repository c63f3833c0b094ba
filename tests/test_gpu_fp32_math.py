"""The FP32 step's reciprocal and square root (a hardware approximation
refined by one Newton-Raphson step) against CUDA's correctly rounded ones:
within one ulp over the argument ranges of the step (densities and
relaxation times for the reciprocal, psi^2 for the square root) and over
every binade of the normal numbers."""
import ctypes

import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm

pytestmark = pytest.mark.gpu


def _run(x):
    x = np.ascontiguousarray(x, dtype=np.float32)
    out = np.zeros(4 * x.size, np.float32)
    L = lbm.load()
    st = L.lbm_selftest_fp32_math(x.size, x.ctypes.data, out.ctypes.data)
    assert st == 0, lbm._lib.STATUS.get(st)
    return out.reshape(-1, 4)


def _ulps(a, b):
    ia = a.view(np.int32).astype(np.int64)
    ib = b.view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def test_within_one_ulp(cuda):
    rng = np.random.default_rng(0)
    x = np.concatenate([
        rng.uniform(0.5, 600.0, 200000),             # densities
        rng.uniform(0.5, 20.0, 50000),               # relaxation times
        rng.uniform(1e-3, 400.0, 200000),            # psi^2
        2.0 ** rng.uniform(-120, 120, 200000),       # every binade
        2.0 ** np.arange(-120, 121, dtype=np.float64),  # exact powers of two
    ]).astype(np.float32)
    o = _run(x)
    assert _ulps(o[:, 0], o[:, 1]).max() <= 1
    assert _ulps(o[:, 2], o[:, 3]).max() <= 1
    # most results are correctly rounded
    assert np.mean(o[:, 0] == o[:, 1]) > 0.9 and np.mean(o[:, 2] == o[:, 3]) > 0.9


def test_special_arguments(cuda):
    x = np.array([0.0, -0.0, -1.0, np.inf, np.nan], np.float32)
    o = _run(x)
    assert o[0, 2] == 0.0 and np.isnan(o[2, 2]) and np.isnan(o[4, 2])
    assert np.isinf(o[3, 2])


def test_fp64_reciprocal_within_one_ulp(cuda):
    """The FP64 step's reciprocal (hardware approximation and two
    Newton-Raphson steps) against CUDA's correctly rounded one, over the
    densities and relaxation times of the step and over the binades of the
    normal numbers the step can meet."""
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.uniform(1e-3, 600.0, 200000), rng.uniform(0.5, 20.0, 50000),
                        2.0 ** rng.uniform(-300, 300, 200000),
                        2.0 ** np.arange(-300, 301, dtype=np.float64)])
    out = np.zeros(2 * x.size)
    L = lbm.load()
    assert L.lbm_selftest_fp64_math(x.size, x.ctypes.data, out.ctypes.data) == 0
    o = out.reshape(-1, 2)
    ulps = np.abs(o[:, 0].view(np.int64) - o[:, 1].view(np.int64))
    assert ulps.max() <= 1, ulps.max()
    assert np.mean(ulps == 0) > 0.9
