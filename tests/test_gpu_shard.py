"""A job split over W ranks (include/bnedge.h, "Shards"), all ranks in this
process on one GPU with the exchange done by device-buffer reads
(shard.run_virtual): the summed posteriors must equal the job run whole bit
for bit (every tile is computed from the same values in the same order), and
the oracle within the method's tolerances (1e-9 FP64, 1e-4 FP32).  Each
rank's matrix holds only its endpoints' columns.  The sizes span several
tile levels, ranks that own no tile of a level, and the largest split the
tile index allows (W = 2^(n-4) FP32, 2^(n-3) FP64, here capped at 32)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen
from paper_1408_1664_gb300 import shard as sh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    c = B.Context(0)
    yield torch, c
    c.close()


def run_split(torch, ctx, job, world, divide_a=False):
    n = job.n
    shards = [B.Shard(ctx.h, job, r, world, divide_a) for r in range(world)]
    try:
        nb = sh.max_step_bytes(shards[0])
        bufs = [torch.zeros(nb, dtype=torch.uint8, device="cuda") for _ in shards]
        parts = [torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
                 for _ in shards]
        lpd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        stream = torch.cuda.Stream()          # not handle 0 (= the context's stream)
        with torch.cuda.stream(stream):
            sh.run_virtual(shards, bufs, parts, lpd, stream)
        stream.synchronize()
        run_split.bytes = [x.bytes() for x in shards]
        return [p.cpu().numpy() for p in parts], float(lpd.item())
    finally:
        for s in shards:
            s.close()


CASES = [
    # n, d, arity, precision, world
    (9, 3, 2, "fp64", 2),
    (12, 3, 2, "fp64", 4),
    (12, 3, 3, "fp64", 32),
    (13, 3, 2, "fp32", 2),
    (16, 4, 2, "fp32", 4),
    (18, 3, 3, "fp32", 8),
    (14, 3, 2, "fp32", 32),
]


@pytest.mark.parametrize("n,d,arity,prec,world", CASES)
def test_split_job_equals_whole_job_and_oracle(torch_ctx, n, d, arity, prec, world):
    torch, ctx = torch_ctx
    ds = datagen.random_dag_data(n=n, m=400, arity=arity, max_parents=3, alpha=1.0, seed=n + world)
    job = B.Job(ds.data, ds.arity, d, precision=prec)
    parts, lpd = run_split(torch, ctx, job, world)
    for r, p in enumerate(parts):
        own = np.array([v % world == r for v in range(n)])
        assert np.all(p[:, ~own] == 0.0), f"rank {r} wrote another rank's endpoint"
    post = np.sum(parts, axis=0)
    whole, lpd_whole = ctx.edge_posteriors(ds.data, ds.arity, d, precision=prec)
    assert np.array_equal(post, whole), float(np.abs(post - whole).max())
    assert lpd == lpd_whole
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    tol = 1e-9 if prec == "fp64" else 1e-4
    np.testing.assert_allclose(post, ref["post"], atol=tol, rtol=0)


DIVIDED = [
    # n, d, arity, precision, world: n - log2(world) >= 14 low variables
    (15, 3, 2, "fp32", 2),
    (16, 3, 2, "fp32", 4),
    (17, 4, 3, "fp32", 8),
    (15, 3, 2, "fp64", 2),
    (16, 2, 3, "fp64", 4),
]


@pytest.mark.parametrize("n,d,arity,prec,world", DIVIDED)
def test_divided_A_split_job(torch_ctx, n, d, arity, prec, world):
    """BN_SHARD_DIVIDE_A: every rank holds only its slabs of A, computed
    from the score table folded over its top bits.  The posteriors agree
    with the whole job and the oracle within the method's tolerances, and a
    rank holds well under the undivided shard's bytes."""
    torch, ctx = torch_ctx
    ds = datagen.random_dag_data(n=n, m=400, arity=arity, max_parents=3, alpha=1.0, seed=n + 7 * world)
    job = B.Job(ds.data, ds.arity, d, precision=prec)
    parts, lpd = run_split(torch, ctx, job, world, divide_a=True)
    divided = run_split.bytes
    for r, p in enumerate(parts):
        own = np.array([v % world == r for v in range(n)])
        assert np.all(p[:, ~own] == 0.0)
    post = np.sum(parts, axis=0)
    tol = 1e-9 if prec == "fp64" else 1e-4
    whole, lpd_whole = ctx.edge_posteriors(ds.data, ds.arity, d, precision=prec)
    np.testing.assert_allclose(post, whole, atol=tol, rtol=0)
    assert abs(lpd - lpd_whole) <= (1e-9 if prec == "fp64" else 1e-3) * max(1.0, abs(lpd_whole))
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    np.testing.assert_allclose(post, ref["post"], atol=tol, rtol=0)
    run_split(torch, ctx, job, world)
    undivided = run_split.bytes
    print(f"n={n} W={world} {prec}: bytes per rank {divided[0]} divided, {undivided[0]} whole A; "
          f"max |split - whole| {np.abs(post - whole).max():.2e}")
    assert max(divided) < 0.8 * min(undivided)


def test_divided_A_needs_14_low_variables(torch_ctx):
    torch, ctx = torch_ctx
    ds = datagen.random_dag_data(n=15, m=100, arity=2, max_parents=2, alpha=1.0, seed=5)
    job = B.Job(ds.data, ds.arity, 2, precision="fp32")
    with pytest.raises(B.BnError) as e:
        B.Shard(ctx.h, job, 0, 4, divide_a=True)     # 13 low variables
    assert e.value.code == B.BN_EINVAL


def test_split_rejects_bad_worlds(torch_ctx):
    torch, ctx = torch_ctx
    ds = datagen.random_dag_data(n=8, m=100, arity=2, max_parents=2, alpha=1.0, seed=3)
    job = B.Job(ds.data, ds.arity, 2, precision="fp32")
    for rank, world in ((0, 3), (2, 2), (-1, 2), (0, 64), (0, 32)):   # n - 4 = 4: W <= 16
        with pytest.raises(B.BnError) as e:
            B.Shard(ctx.h, job, rank, world)
        assert e.value.code == B.BN_EINVAL
