"""The order prior q_i(S) (by |S|), per-family weights (a general rho_i(G))
and single modular features (Eqs. 4-9, 12) through the C ABI, against the
CPU FP64 oracle: posteriors within 1e-9 (FP64) and 1e-4 (FP32).  Sizes on
both sides of n = 14, where steps 2 and 4 switch to the 13-dimension tiles."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-9, "fp32": 1e-4}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    c = B.Context(0)
    yield c
    c.close()


def _priors(n, K, seed, zeros=0.25):
    rng = np.random.default_rng(seed)
    log_q = rng.normal(0.0, 1.5, size=(n, n))
    log_w = rng.normal(0.0, 1.0, size=(n, K))
    log_w[rng.random((n, K)) < zeros] = -math.inf
    log_w[:, 0] = 0.0                              # every node keeps a parent set
    return log_q, log_w


CASES = [(9, 3, [2, 3, 2, 2, 3, 2, 4, 2, 2], 300, 1), (12, 2, 2, 500, 2),
         (15, 3, 2, 400, 3), (16, 4, 3, 600, 4)]


@pytest.mark.parametrize("n,d,arity,m,seed", CASES)
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_order_prior_and_family_weights(ctx, n, d, arity, m, seed, precision):
    ds = datagen.random_dag_data(n, m, arity, min(d, 3), 0.8, seed=600 + seed)
    log_q, log_w = _priors(n, orc.num_families(n, d), seed)
    ref = orc.edge_posteriors(ds.data, ds.arity, d, log_q=log_q, log_w=log_w)
    post, lpd = B.bn_edge_posteriors(ctx.h, B.Job(ds.data, ds.arity, d, precision=precision,
                                                  log_q=log_q, log_w=log_w))
    np.testing.assert_allclose(post, ref["post"], atol=TOL[precision], rtol=0)
    if precision == "fp64":
        assert abs(lpd - ref["log_PD"]) <= 1e-9 * max(1.0, abs(ref["log_PD"]))


def test_scores_include_family_weights(ctx):
    ds = datagen.random_dag_data(10, 250, 3, 3, 1.0, seed=610)
    K = orc.num_families(10, 3)
    _, log_w = _priors(10, K, 11)
    masks, logB = B.bn_scores(ctx.h, B.Job(ds.data, ds.arity, 3, log_w=log_w))
    om, ol = orc.scores(ds.data, ds.arity, 3)
    np.testing.assert_array_equal(masks, om)
    fin = np.isfinite(log_w)
    np.testing.assert_allclose(logB[fin], (ol + log_w)[fin], atol=1e-10, rtol=0)
    assert np.all(logB[~fin] < -9e6)               # a zero weight held as -1e7: exp == 0
    assert np.all(np.exp(logB[~fin]) == 0.0)


def test_prior_served_equals_direct(ctx):
    """The served path uploads the priors like the direct one: identical bits,
    and both within the FP32 tolerance of the oracle."""
    ds = datagen.random_dag_data(13, 300, 2, 3, 1.0, seed=611)
    log_q, log_w = _priors(13, orc.num_families(13, 3), 12)
    ref = orc.edge_posteriors(ds.data, ds.arity, 3, log_q=log_q, log_w=log_w)
    job = B.Job(ds.data, ds.arity, 3, precision="fp32", log_q=log_q, log_w=log_w)
    post0, lpd0 = B.bn_edge_posteriors(ctx.h, job)
    jid = B.bn_submit(ctx.h, job)
    rc, post1, lpd1 = B.bn_wait(ctx.h, jid, 13)
    assert rc == 0
    assert np.array_equal(post0, post1) and lpd0 == lpd1
    np.testing.assert_allclose(post1, ref["post"], atol=TOL["fp32"], rtol=0)


def _random_feature(masks, seed, p_zero=0.4):
    rng = np.random.default_rng(seed)
    log_f = np.where(rng.random(masks.shape) < p_zero, -math.inf, 0.0)
    log_f[:, 0] = 0.0
    return log_f


@pytest.mark.parametrize("n,d,seed", [(7, 2, 20), (11, 3, 21), (15, 3, 22)])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_feature_posterior_matches_oracle(ctx, n, d, seed, precision):
    ds = datagen.random_dag_data(n, 300, 2, min(d, 3), 0.8, seed=620 + seed)
    masks, _ = orc.scores(ds.data, ds.arity, d)
    log_q, log_w = _priors(n, masks.shape[1], seed)
    log_f = _random_feature(masks, seed)
    p_ref, lpfd_ref = orc.feature_posterior(ds.data, ds.arity, d, log_f, log_q=log_q,
                                            log_w=log_w)
    p, lpfd = B.bn_feature_posterior(ctx.h, B.Job(ds.data, ds.arity, d, precision=precision,
                                                  log_q=log_q, log_w=log_w), log_f)
    assert abs(p - p_ref) <= TOL[precision]
    if precision == "fp64":
        assert abs(lpfd - lpfd_ref) <= 1e-9 * max(1.0, abs(lpfd_ref))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_edge_feature_equals_edge_posterior(ctx, precision):
    """P(u -> v | D) by the single-feature DP equals the all-edges path, on
    the GPU, at n = 14 (13-dimension tiles in step 2)."""
    n, d = 14, 3
    ds = datagen.random_dag_data(n, 500, 2, 3, 1.0, seed=630)
    K = orc.num_families(n, d)
    masks, _ = orc.scores(ds.data, ds.arity, d)
    job = B.Job(ds.data, ds.arity, d, precision=precision)
    post, _ = B.bn_edge_posteriors(ctx.h, job)
    for (u, v) in [(0, 1), (5, 9), (13, 2), (7, 6)]:
        log_f = np.zeros((n, K))
        log_f[v] = np.where((masks[v] >> u) & 1, 0.0, -math.inf)
        p, _ = B.bn_feature_posterior(ctx.h, job, log_f)
        assert abs(p - post[u, v]) <= TOL[precision], (u, v)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_trivial_and_impossible_features(ctx, precision):
    ds = datagen.random_dag_data(9, 200, 2, 2, 1.0, seed=640)
    K = orc.num_families(9, 2)
    job = B.Job(ds.data, ds.arity, 2, precision=precision)
    _, lpd = B.bn_edge_posteriors(ctx.h, B.Job(ds.data, ds.arity, 2))
    p, lpfd = B.bn_feature_posterior(ctx.h, job, np.zeros((9, K)))
    assert abs(p - 1.0) <= (1e-12 if precision == "fp64" else 1e-5)
    assert abs(lpfd - lpd) <= (1e-9 if precision == "fp64" else 1e-3) * max(1.0, abs(lpd))
    log_f = np.zeros((9, K))
    log_f[4] = -math.inf
    p, lpfd = B.bn_feature_posterior(ctx.h, job, log_f)
    assert p == 0.0 and lpfd == -math.inf


def test_invalid_priors_are_rejected(ctx):
    ds = datagen.random_dag_data(6, 50, 2, 2, 1.0, seed=650)
    K = orc.num_families(6, 2)
    bad = np.zeros((6, 6))
    bad[2, 3] = np.nan
    with pytest.raises(B.BnError):
        B.bn_edge_posteriors(ctx.h, B.Job(ds.data, ds.arity, 2, log_q=bad))
    w = np.zeros((6, K))
    w[1, 1] = math.inf
    with pytest.raises(B.BnError):
        B.bn_edge_posteriors(ctx.h, B.Job(ds.data, ds.arity, 2, log_w=w))
    f = np.zeros((6, K))
    f[0, 0] = np.nan
    with pytest.raises(B.BnError):
        B.bn_feature_posterior(ctx.h, B.Job(ds.data, ds.arity, 2), f)
    # batches do not take the priors
    with pytest.raises(B.BnError):
        B.Batch(ctx.h, [B.Job(ds.data, ds.arity, 2, log_q=np.zeros((6, 6)))])
