"""Serving through bn_submit / bn_poll / bn_wait (continuous batching).

Jobs of different sizes submitted together run concurrently on the
context's slots (separate streams); each result must equal the same job run
alone through bn_edge_posteriors.  Every reduction of the library has a fixed
order, so "equal" is bit-for-bit here, which is tighter than the stated
tolerances (1e-9 FP64, 1e-4 FP32).  Each served result is also compared with
the CPU FP64 oracle within those tolerances.
"""
import time

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    return torch


def _mix():
    out = []
    for j in range(10):
        ds, d = datagen.served_job(j)
        out.append((ds, d, "fp32" if j % 3 else "fp64"))
    ds = datagen.random_dag_data(17, 400, 3, 3, 1.0, seed=91)
    out.append((ds, 3, "fp32"))
    return out


def test_results_equal_alone_and_in_the_mix(torch_cuda):
    jobs = _mix()
    refs = [orc.edge_posteriors(ds.data, ds.arity, d) for ds, d, _ in jobs]
    with B.Context(0, slots=4) as ctx:
        alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision=p) for ds, d, p in jobs]
        descs = [B.Job(ds.data, ds.arity, d, precision=p) for ds, d, p in jobs]
        ids = [B.bn_submit(ctx.h, j) for j in descs]
        for (ds, d, p), jid, (post0, lpd0), ref in zip(jobs, ids, alone, refs):
            rc, post, lpd = B.bn_wait(ctx.h, jid, ds.n, timeout_s=60.0)
            assert rc == B.BN_OK, B.bn_strerror(rc)
            assert np.array_equal(post, post0), (ds.n, p)
            assert lpd == lpd0
            tol = 1e-9 if p == "fp64" else 1e-4
            np.testing.assert_allclose(post, ref["post"], atol=tol, rtol=0)
            st = B.bn_job_stats(ctx.h, 0)
            assert st["kernels"] > 0 and st["ms_total"] > 0


def test_admission_by_memory_budget(torch_cuda):
    """With a budget just above one large job's footprint, a second job waits
    in the queue until the first has released its memory (it can still be
    canceled there); afterwards queued jobs all complete and match."""
    big, db = datagen.random_dag_data(22, 500, 2, 3, 1.0, seed=5), 3
    small, ds_ = datagen.random_dag_data(14, 300, 2, 3, 1.0, seed=15), 3
    jb = B.Job(big.data, big.arity, db, precision="fp64")
    js = B.Job(small.data, small.arity, ds_, precision="fp64")
    fb, fs = B.bn_job_footprint(jb), B.bn_job_footprint(js)
    assert fb > fs > 0
    with B.Context(0, slots=4) as probe:
        want_s, _ = probe.edge_posteriors(small.data, small.arity, ds_, precision="fp64")
    with B.Context(0, slots=4, mem_budget=fb + fs // 2) as ctx:
        first = B.bn_submit(ctx.h, jb)
        second = B.bn_submit(ctx.h, js)
        assert B.bn_cancel(ctx.h, second) == B.BN_OK          # still queued
        assert B.bn_poll(ctx.h, second, small.n)[0] == B.BN_ECANCELED
        others = [B.bn_submit(ctx.h, js) for _ in range(3)]
        assert B.bn_wait(ctx.h, first, big.n, timeout_s=120.0)[0] == B.BN_OK
        for jid in others:
            rc, post, _ = B.bn_wait(ctx.h, jid, small.n, timeout_s=60.0)
            assert rc == B.BN_OK
            assert np.array_equal(post, want_s)


def test_job_larger_than_budget_is_rejected(torch_cuda):
    ds, d = datagen.random_dag_data(20, 100, 2, 3, 1.0, seed=6), 3
    with B.Context(0, slots=2, mem_budget=8 << 20) as ctx:
        with pytest.raises(B.BnError) as ei:
            B.bn_submit(ctx.h, B.Job(ds.data, ds.arity, d, precision="fp32"))
        assert ei.value.code == B.BN_ENOMEM


def test_cancel_a_queued_job(torch_cuda):
    ds, d = datagen.random_dag_data(16, 300, 2, 3, 1.0, seed=7), 3
    with B.Context(0, slots=1) as ctx:
        first = B.bn_submit(ctx.h, B.Job(ds.data, ds.arity, d, precision="fp64"))
        second = B.bn_submit(ctx.h, B.Job(ds.data, ds.arity, d, precision="fp64"))
        rc = B.bn_cancel(ctx.h, second)
        if rc == B.BN_OK:          # it was still queued behind the single slot
            assert B.bn_poll(ctx.h, second, ds.n)[0] == B.BN_ECANCELED
        else:
            assert rc == B.BN_EAGAIN
            assert B.bn_wait(ctx.h, second, ds.n)[0] == B.BN_OK
        assert B.bn_wait(ctx.h, first, ds.n)[0] == B.BN_OK
        assert B.bn_poll(ctx.h, first, ds.n)[0] == B.BN_ENOTFOUND   # retired


def test_injected_allocation_failure(torch_cuda):
    ds, d = datagen.random_dag_data(12, 200, 2, 3, 1.0, seed=8), 3
    with B.Context(0, slots=2, fail_alloc_after=0) as ctx:
        jid = B.bn_submit(ctx.h, B.Job(ds.data, ds.arity, d, precision="fp32"))
        rc, _, _ = B.bn_wait(ctx.h, jid, ds.n, timeout_s=10.0)
        assert rc == B.BN_ENOMEM
        with pytest.raises(B.BnError) as ei:
            ctx.edge_posteriors(ds.data, ds.arity, d)
        assert ei.value.code == B.BN_ENOMEM


def test_wait_timeout_returns_etimeout(torch_cuda):
    ds, d = datagen.random_dag_data(22, 300, 2, 3, 1.0, seed=9), 3
    with B.Context(0, slots=1) as ctx:
        jid = B.bn_submit(ctx.h, B.Job(ds.data, ds.arity, d, precision="fp64"))
        rc, _, _ = B.bn_wait(ctx.h, jid, ds.n, timeout_s=0.0)
        assert rc in (B.BN_ETIMEOUT, B.BN_OK)
        t0 = time.time()
        rc, _, _ = B.bn_wait(ctx.h, jid, ds.n, timeout_s=120.0)
        assert rc == B.BN_OK and time.time() - t0 < 120.0
