"""The persistent FP32 up-zeta tile kernel (k_upzeta13p) keeps the next
tile's column sums in flight as a bulk copy counted by an mbarrier.  Its wait
for that copy is bounded: with the copy withheld (a test hook) the block
gives up after the given number of polls, leaves the timeout bit in the job's
error word and returns -- no fault, no endless wait -- and the context runs
the next job correctly.  Jobs that take the kernel agree with the oracle
(Eq. 7 through the posteriors) and with the same jobs run inside a batch,
which uses the per-tile kernel, bit for bit."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    c = B.Context(0, autotune=False)
    yield c
    c.close()


@pytest.mark.parametrize("polls", [1, 1000, 100000])
def test_withheld_copy_times_out_and_context_survives(ctx, polls):
    w = C.c_int32(-1)
    rc = B.load().bn_debug_copy_wait(polls, C.byref(w))
    assert rc == 0
    assert w.value == 2                   # the timeout bit, nothing else
    ds = datagen.random_dag_data(n=14, m=300, arity=2, max_parents=3, alpha=1.0, seed=polls % 97)
    post, _ = ctx.edge_posteriors(ds.data, ds.arity, 3, precision="fp32")
    ref = orc.edge_posteriors(ds.data, ds.arity, 3)
    np.testing.assert_allclose(post, ref["post"], atol=1e-4, rtol=0)


@pytest.mark.parametrize("n,d,arity", [(14, 4, 2), (16, 3, 3), (17, 5, 2)])
def test_persistent_tiles_match_oracle_and_per_tile_kernel(ctx, n, d, arity):
    ds = datagen.random_dag_data(n=n, m=500, arity=arity, max_parents=3, alpha=1.0, seed=11 * n + d)
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    np.testing.assert_allclose(post, ref["post"], atol=1e-4, rtol=0)
    # the same job twice in a batch group: the per-tile kernel
    jobs = [B.Job(ds.data, ds.arity, d, precision="fp32") for _ in range(2)]
    with B.Batch(ctx.h, jobs) as batch:
        batch.run()
        for k in range(2):
            bpost, blpd = batch.results(k)
            assert np.array_equal(bpost, post), k
            assert blpd == lpd
