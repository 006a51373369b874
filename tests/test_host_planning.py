"""Host-side validation and planning through the C ABI, without a GPU.
bn_job_footprint checks a job as the compute entry points do (the limits and
input rules in include/bnedge.h) and returns the device bytes of its plan,
which must hold the DP arrays of Algorithm 1: A (n 2^(n-1) values, Eq. 7),
F and R' (2^n each, Eqs. 9-10) and the down-zeta rows W (n 2^(n-14) ncol
values for n >= 14, Eq. 12)."""
import math

import numpy as np
import pytest

from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen


@pytest.fixture(scope="module")
def lib():
    B.load(build_if_missing=True)


def _fp(job):
    return B.bn_job_footprint(job)


def test_footprint_holds_the_dp_arrays(lib):
    ds, d = datagen.config_large()                    # n = 26, d = 4
    n = ds.n
    ncol = sum(math.comb(13, k) for k in range(d + 1))
    values = n * 2 ** (n - 1) + 2 * 2 ** n + n * 2 ** (n - 14) * ncol
    f32 = _fp(B.Job(ds.data, ds.arity, d, precision="fp32"))
    f64 = _fp(B.Job(ds.data, ds.arity, d, precision="fp64"))
    assert 4 * values <= f32 <= 1.05 * 4 * values + 2 ** 27
    assert 8 * values <= f64 <= 1.05 * 8 * values + 2 ** 27


def test_in_degree_above_n_minus_1_is_n_minus_1(lib):
    ds = datagen.random_dag_data(9, 50, 2, 2, 1.0, seed=5)
    assert _fp(B.Job(ds.data, ds.arity, 8)) == _fp(B.Job(ds.data, ds.arity, 40))


def test_no_samples_is_valid(lib):
    assert _fp(B.Job(np.zeros((0, 6), np.uint8), [2] * 6, 2)) > 0


def _job(**kw):
    ds = datagen.random_dag_data(6, 40, 2, 2, 1.0, seed=9)
    args = dict(data=ds.data, arity=ds.arity, d=2)
    args.update(kw)
    return B.Job(**args)


K6 = sum(math.comb(5, k) for k in range(3))
BAD = {
    "value_not_below_arity": lambda: _job(data=np.full((3, 6), 2, np.uint8)),
    "negative_in_degree": lambda: _job(d=-1),
    "arity_zero": lambda: _job(data=np.zeros((3, 6), np.uint8), arity=[0, 2, 2, 2, 2, 2]),
    "ess_zero": lambda: _job(ess=0.0),
    "ess_nan": lambda: _job(ess=float("nan")),
    "log_rho_nan": lambda: _job(log_rho=[0.0, float("nan"), 0.0]),
    "log_q_nan": lambda: _job(log_q=np.full((6, 6), np.nan)),
    "log_w_plus_inf": lambda: _job(log_w=np.full((6, K6), np.inf)),
    "too_many_cells": lambda: _job(data=np.zeros((3, 6), np.uint8), arity=[255] * 6),
    "n_above_32": lambda: B.Job(np.zeros((2, 33), np.uint8), [2] * 33, 2),
}


@pytest.mark.parametrize("case", sorted(BAD))
def test_invalid_jobs_are_rejected(lib, case):
    with pytest.raises(B.BnError) as ei:
        _fp(BAD[case]())
    assert ei.value.code == B.BN_EINVAL


def test_zero_weights_are_accepted(lib):
    w = np.zeros((6, K6))
    w[:, 1:] = -np.inf                                 # -inf: a zero factor
    assert _fp(_job(log_w=w)) > 0
