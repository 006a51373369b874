"""The FP64 path's table-driven exponential and logarithm (bn_device.cuh:
exp_t, log_t, after Tang's method) against CUDA's exp and log on the GPU.

  exp: within 2 ulp of CUDA's result (itself within 1 ulp of the true value
       by its documented bound) over [-708.3, 709.7], with dense points near
       0 and near the multiples of ln2/64 where the reduction switches table
       entries; 0 below -708.3 (CUDA gives a subnormal there), +inf above
       709.7, NaN for NaN.
  log: within 2 ulp of the result's magnitude or 2^-60 absolute (near 1,
       where log x is tiny, the absolute error is what a log-domain sum
       sees), over normal and subnormal inputs, exact powers of two, the
       table's boundaries and 1 +- small; log 0 = -inf, log of a negative
       number or NaN = NaN, log +inf = +inf."""
import ctypes as C

import numpy as np
import pytest

from paper_1408_1664_gb300 import binding as B

pytestmark = pytest.mark.gpu


def run(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.zeros((x.size, 4))
    rc = B.load().bn_debug_explog(x.ctypes.data, x.size, out.ctypes.data)
    assert rc == 0
    return out[:, 0], out[:, 1], out[:, 2], out[:, 3]


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.load(build_if_missing=True)


def test_exp_within_two_ulp(lib):
    rng = np.random.default_rng(1)
    step = np.log(2.0) / 64
    x = np.concatenate([
        rng.uniform(-708.3, 709.7, 2_000_000),
        rng.uniform(-1.0, 1.0, 500_000),
        rng.uniform(-1e-8, 1e-8, 100_000),
        np.arange(-65000, 65000, 7) * step,                    # table switch points
        np.arange(-65000, 65000, 7) * step + 1e-13,
        [0.0, -0.0, 1.0, -1.0, 709.7, -708.29, 1e-300, -1e-300],
    ])
    mine, cuda, _, _ = run(x)
    ulp = np.spacing(np.abs(cuda))
    err = np.abs(mine - cuda) / ulp
    print(f"exp: max error {err.max():.2f} ulp over {x.size} points")
    assert err.max() <= 2.0


def test_exp_special_values(lib):
    x = np.array([-708.31, -745.0, -1e308, -np.inf, 709.71, 1e308, np.inf, np.nan])
    mine, _, _, _ = run(x)
    assert np.all(mine[:4] == 0.0)
    assert np.all(np.isposinf(mine[4:7]))
    assert np.isnan(mine[7])


def test_log_within_two_ulp(lib):
    rng = np.random.default_rng(2)
    exps = rng.uniform(-1074, 1023, 2_000_000)
    x = np.concatenate([
        np.exp2(exps) * rng.uniform(1.0, 2.0, exps.size),
        rng.uniform(0.5, 2.0, 1_000_000),
        1.0 + rng.uniform(-1e-6, 1e-6, 100_000),
        1.0 + (2 * np.arange(128) + 1) / 256.0,                # the table's c_j
        1.0 + np.arange(129) / 128.0,                          # its boundaries
        np.exp2(np.arange(-1074, 1024, dtype=np.float64)),     # powers of two, subnormals
        [1.0, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 5e-324, 1.7976931348623157e308],
    ])
    x = x[np.isfinite(x) & (x > 0)]
    _, _, mine, cuda = run(x)
    tol = np.maximum(2.0 * np.spacing(np.abs(cuda)), 2.0 ** -60)
    err = np.abs(mine - cuda)
    bad = err > tol
    print(f"log: max error {np.max(err / np.spacing(np.maximum(np.abs(cuda), 1e-300))):.2f} ulp, "
          f"{bad.sum()} points beyond 2 ulp / 2^-60 over {x.size}")
    assert not bad.any(), x[bad][:5]


def test_log_special_values(lib):
    x = np.array([0.0, -0.0, -1.0, -np.inf, np.nan, np.inf])
    _, _, mine, _ = run(x)
    assert np.isneginf(mine[0]) and np.isneginf(mine[1])
    assert np.isnan(mine[2]) and np.isnan(mine[3]) and np.isnan(mine[4])
    assert np.isposinf(mine[5])
