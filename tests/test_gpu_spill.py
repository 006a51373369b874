"""A job whose arrays exceed the context's device budget (the space-time
trade-off of reaching larger n on one GPU): A (Eq. 7, n 2^(n-1) values, the
largest array) moves to one managed allocation whose first part stays in
device memory and whose rest lives in host memory that the kernels read and
write in place over the CPU-GPU link.  The kernels and their order are
unchanged, so the posteriors, log P(D) and A itself equal the in-core run bit
for bit.  A budget below the other arrays alone is refused (BN_ENOMEM)."""
import numpy as np
import pytest

from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B.load(build_if_missing=True)


@pytest.mark.parametrize("n,d,prec,frac", [(16, 3, "fp32", 0.5), (18, 4, "fp32", 0.9),
                                           (15, 3, "fp64", 0.5), (20, 3, "fp32", 0.25)])
def test_spilled_A_equals_in_core(lib, n, d, prec, frac):
    ds = datagen.random_dag_data(n=n, m=300, arity=2, max_parents=3, alpha=1.0, seed=70 + n)
    job = B.Job(ds.data, ds.arity, d, precision=prec)
    es = 8 if prec == "fp64" else 4
    a_bytes = n * 2 ** (n - 1) * es
    fp = B.bn_job_footprint(job)
    with B.Context(0) as ctx:
        post0, lpd0 = ctx.edge_posteriors(ds.data, ds.arity, d, precision=prec)
        A0 = B.bn_debug_stage(ctx.h, B.BN_STAGE_A, (n, 2 ** (n - 1)),
                              np.float64 if prec == "fp64" else np.float32)
    # a budget that leaves room for (1 - frac) of A in device memory
    budget = fp - int(frac * a_bytes)
    with B.Context(0, mem_budget=budget) as ctx:
        post1, lpd1 = ctx.edge_posteriors(ds.data, ds.arity, d, precision=prec)
        A1 = B.bn_debug_stage(ctx.h, B.BN_STAGE_A, (n, 2 ** (n - 1)),
                              np.float64 if prec == "fp64" else np.float32)
        post2, lpd2 = ctx.edge_posteriors(ds.data, ds.arity, d, precision=prec)   # reused
    assert np.array_equal(post0, post1) and lpd0 == lpd1
    assert np.array_equal(post0, post2) and lpd0 == lpd2
    assert np.array_equal(A0, A1)


def test_budget_below_the_other_arrays_is_refused(lib):
    ds = datagen.random_dag_data(n=16, m=100, arity=2, max_parents=2, alpha=1.0, seed=9)
    job = B.Job(ds.data, ds.arity, 3, precision="fp32")
    a_bytes = 16 * 2 ** 15 * 4
    rest = B.bn_job_footprint(job) - a_bytes
    with B.Context(0, mem_budget=rest // 2) as ctx:
        with pytest.raises(B.BnError) as e:
            ctx.edge_posteriors(ds.data, ds.arity, 3, precision="fp32")
        assert e.value.code == B.BN_ENOMEM
