"""Batches: many independent small jobs replayed as one CUDA graph
(bn_batch_create / bn_batch_run / bn_batch_results).  Each job's result must
equal the same job run alone (bit for bit: every reduction has a fixed
order), on every replay."""
import numpy as np
import pytest

from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    c = B.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_equals_alone_over_replays(ctx, precision):
    jobs = [datagen.batched_job(j) for j in range(20)]
    alone = [ctx.edge_posteriors(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
    descs = [B.Job(ds.data, ds.arity, d, precision=precision) for ds, d in jobs]
    with B.Batch(ctx.h, descs) as batch:
        for _ in range(2):
            batch.run()
            for k, (post0, lpd0) in enumerate(alone):
                post, lpd = batch.results(k)
                assert np.array_equal(post, post0), k
                assert lpd == lpd0


def test_batch_rejects_device_data_and_empty(ctx):
    torch = pytest.importorskip("torch")
    ds, d = datagen.batched_job(0)
    dev = torch.from_numpy(ds.data).cuda()
    with pytest.raises(B.BnError):
        B.Batch(ctx.h, [B.Job(dev, ds.arity, d, m=ds.m)])
    with pytest.raises(B.BnError):
        B.Batch(ctx.h, [])
