"""Batches: many independent small jobs (bn_batch_create / bn_batch_run /
bn_batch_results).  Jobs with equal n, d, precision and kind of data form a
group that shares every launch of steps 1-5.  A batch exists in two forms:
a CUDA graph of those launches, and one persistent launch per precision
whose blocks take items (runs of the virtual blocks of one recorded launch)
from a device queue ordered by stage depth, each item first waiting, by
bounded polls, for the completion count of the launch before it in its
group's chain.  Without autotuning the persistent form runs; with it, the
faster of the two (BN_CTX_GRAPH_BATCH keeps the graph).

Under the default schedules each job's result equals the same job run alone
bit for bit in both forms (the same kernels, every reduction in a fixed
order).  With the graph form's autotuner on, a group may run other kernels
for a step; its results then agree with the job run alone within the stated
tolerances (1e-9 FP64, 1e-4 FP32), and are identical on every replay."""
import collections

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    return torch


def _jobs(count=20, first=0):
    return [datagen.batched_job(j) for j in range(first, first + count)]


@pytest.mark.parametrize("graph", [False, True])
@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_default_schedule_equals_alone_over_replays(torch_cuda, precision, graph):
    jobs = _jobs()
    with B.Context(0, autotune=False, graph_batch=graph) as ctx:
        alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
        descs = [B.Job(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
        with B.Batch(ctx.h, descs) as batch:
            text = batch.describe()
            assert "timed" not in text.replace("default-or-cached", "")
            assert ("in use" in text) != graph, text
            for _ in range(2):
                batch.run()
                for k, (post0, lpd0) in enumerate(alone):
                    post, lpd = batch.results(k)
                    assert np.array_equal(post, post0), k
                    assert lpd == lpd0


def test_cluster_step3_equals_alone(torch_cuda):
    """Step 3 in the persistent cluster kernel (forced for every FP32 group):
    the same 16-subset tiles as the per-level row launches, in the same
    order, so every job equals the job run alone bit for bit -- over two
    replays, with groups from n = 10 to 18 and more items than clusters."""
    jobs = _jobs(48, first=100)
    assert min(ds.n for ds, _ in jobs) <= 11 and max(ds.n for ds, _ in jobs) >= 17
    with B.Context(0, autotune=False, cluster_step3=True) as ctx:
        alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32") for ds, d in jobs]
        descs = [B.Job(ds.data, ds.arity, d, precision="fp32") for ds, d in jobs]
        with B.Batch(ctx.h, descs) as batch:
            text = batch.describe()
            assert all(" frc=1 " in line for line in text.strip().splitlines()), text
            for _ in range(2):
                batch.run()
                for k, (post0, lpd0) in enumerate(alone):
                    post, lpd = batch.results(k)
                    assert np.array_equal(post, post0), k
                    assert lpd == lpd0


def test_cluster_step3_many_jobs_one_group(torch_cuda):
    """24 jobs at n = 18 (8-block clusters): 48 work items over at most 38
    clusters, so some clusters run a second item after the first."""
    d = 3
    rng = np.random.default_rng(5)
    jobs = []
    for t in range(24):
        ds = datagen.random_dag_data(18, int(rng.integers(100, 400)), 2, d, 1.0, seed=4000 + t)
        jobs.append((ds, d))
    with B.Context(0, autotune=False, cluster_step3=True) as ctx:
        alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32") for ds, d in jobs]
        with B.Batch(ctx.h, [B.Job(ds.data, ds.arity, d, precision="fp32")
                             for ds, d in jobs]) as batch:
            batch.run()
            for k, (post0, lpd0) in enumerate(alone):
                post, lpd = batch.results(k)
                assert np.array_equal(post, post0), k
                assert lpd == lpd0


def test_persistent_tuner_and_mixed_precision(torch_cuda):
    """The persistent form's tuner times work items of 1, 2 and 4 blocks on
    the batch's own data; a batch with FP32 and FP64 jobs runs one persistent
    launch per precision.  n from 10 to 18: every job equals the job run
    alone, over two replays.  (With the tuner on, the faster form runs; the
    persistent one is forced here through the fixed-schedule context after
    timing it in an autotuned one.)"""
    jobs = _jobs(64, first=300)
    precs = ["fp32" if k % 4 else "fp64" for k in range(len(jobs))]
    with B.Context(0) as ctx:
        descs = [B.Job(ds.data, ds.arity, d, precision=p) for (ds, d), p in zip(jobs, precs)]
        with B.Batch(ctx.h, descs) as batch:
            text = batch.describe()
            lines = [x for x in text.splitlines() if x.startswith("persistent")]
            assert len(lines) == 2, text
            assert all("1:" in x and "4:" in x for x in lines), text     # item sizes timed
    with B.Context(0, autotune=False) as ctx:
        alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision=p)
                 for (ds, d), p in zip(jobs, precs)]
        descs = [B.Job(ds.data, ds.arity, d, precision=p) for (ds, d), p in zip(jobs, precs)]
        with B.Batch(ctx.h, descs) as batch:
            text = batch.describe()
            lines = [x for x in text.splitlines() if x.startswith("persistent")]
            assert len(lines) == 2 and all("in use" in x for x in lines), text
            for _ in range(2):
                batch.run()
                for k, (post0, lpd0) in enumerate(alone):
                    post, lpd = batch.results(k)
                    assert np.array_equal(post, post0), k
                    assert lpd == lpd0


def test_persistent_wait_times_out_when_a_stage_never_runs(torch_cuda):
    """Every device-side wait of the persistent kernel is bounded.  The host
    takes the work items of one stage (the per-node maxima of the scores,
    fourth in each group's sequence) out of the queue, so the items after
    them wait for results that never come; after 20000 polls the kernel
    records BN_EDEVICE_TIMEOUT, raises its abort flag and returns -- no fault,
    no endless wait -- and bn_batch_results reports the timeout."""
    import time
    jobs = _jobs(12, first=500)
    with B.Context(0, autotune=False) as ctx:
        with B.Batch(ctx.h, [B.Job(ds.data, ds.arity, d, precision="fp32")
                             for ds, d in jobs]) as batch:
            assert B.load().bn_debug_batch_drop(batch.h, 3, 20000) == B.BN_OK
            t0 = time.time()
            batch.run()
            with pytest.raises(B.BnError) as ei:
                batch.results(0)
            assert ei.value.code == B.BN_EDEVICE_TIMEOUT
            assert time.time() - t0 < 30.0
        # the context still works
        ds, d = jobs[0]
        post, _ = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
        assert np.all(np.isfinite(post))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_autotuned_batch_within_tolerance_and_cached(torch_cuda, precision):
    """The graph form's schedule tuner (kernel choices per group)."""
    jobs = _jobs(24, first=40)
    ns = {ds.n for ds, _ in jobs}
    assert min(ns) < 14 <= max(ns)             # both tile paths are in the batch
    with B.Context(0, graph_batch=True) as ctx:
        alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
        descs = [B.Job(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
        with B.Batch(ctx.h, descs) as batch:
            text = batch.describe()
            # groups are (n, d, binary data or not); the autotuner times each
            groups = collections.Counter((ds.n, d, bool(np.all(ds.arity == 2))) for ds, d in jobs)
            assert len([x for x in text.strip().splitlines() if x.startswith("n=")]) == len(groups), text
            assert text.count("timed") == len(groups), text
            first = []
            for rep in range(2):
                batch.run()
                for k, (post0, lpd0) in enumerate(alone):
                    post, lpd = batch.results(k)
                    np.testing.assert_allclose(post, post0, atol=TOL[precision], rtol=0)
                    if rep == 0:
                        first.append((post, lpd))
                    else:
                        assert np.array_equal(post, first[k][0]) and lpd == first[k][1]
        # the same group shapes again: the schedules come from the context's cache
        descs2 = [B.Job(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
        with B.Batch(ctx.h, descs2) as batch2:
            assert "timed" not in batch2.describe().replace("default-or-cached", "")
            batch2.run()
            for k in range(len(jobs)):
                post, lpd = batch2.results(k)
                assert np.array_equal(post, first[k][0]) and lpd == first[k][1]


@pytest.mark.parametrize("graph", [False, True])
def test_upload_new_data_and_download_all(torch_cuda, graph):
    """bn_batch_upload replaces every job's data (same shapes) and
    bn_batch_download returns every job's results at once: after a first
    run, new data drawn from other seeds give, in the same batch, the results
    of the new jobs run alone; data of another shape are rejected."""
    jobs = _jobs(16, first=700)
    other = [(datagen.random_dag_data(ds.n, ds.m, ds.arity, 3, 1.0, seed=9000 + k), d)
             for k, (ds, d) in enumerate(jobs)]
    with B.Context(0, autotune=False, graph_batch=graph) as ctx:
        want1 = [ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32") for ds, d in jobs]
        want2 = [ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32") for ds, d in other]
        with B.Batch(ctx.h, [B.Job(ds.data, ds.arity, d, precision="fp32")
                             for ds, d in jobs]) as batch:
            for want, src in ((want1, None), (want2, other), (want1, jobs)):
                if src is not None:
                    batch.upload([B.Job(ds.data, ds.arity, d, precision="fp32") for ds, d in src])
                batch.run()
                posts, lpds = batch.download()
                for k, (post0, lpd0) in enumerate(want):
                    assert np.array_equal(posts[k], post0), k
                    assert lpds[k] == lpd0
            bad = [B.Job(ds.data[:-1], ds.arity, d, precision="fp32") for ds, d in jobs]
            with pytest.raises(B.BnError):
                batch.upload(bad)


def test_batch_jobs_match_the_oracle(torch_cuda):
    jobs = _jobs(6, first=7)
    with B.Context(0) as ctx:
        for precision in ("fp64", "fp32"):
            descs = [B.Job(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
            with B.Batch(ctx.h, descs) as batch:
                batch.run()
                for k, (ds, d) in enumerate(jobs):
                    post, lpd = batch.results(k)
                    ref = orc.edge_posteriors(ds.data, ds.arity, d)
                    np.testing.assert_allclose(post, ref["post"], atol=TOL[precision], rtol=0)


def test_batch_rejects_device_data_and_empty(torch_cuda):
    torch = torch_cuda
    ds, d = datagen.batched_job(0)
    dev = torch.from_numpy(ds.data).cuda()
    with B.Context(0) as ctx:
        with pytest.raises(B.BnError):
            B.Batch(ctx.h, [B.Job(dev, ds.arity, d, m=ds.m)])
        with pytest.raises(B.BnError):
            B.Batch(ctx.h, [])
