"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (stated by the method's contract): counts and parent masks
bit-exact; edge posteriors within 1e-9 absolute on the FP64 path and 1e-4 on
the FP32 path.  Local scores: an error delta in log B_i(G) changes every
posterior by at most about 2*delta (P = X/Y with X and Y both scaled by at
most exp(delta)), so log B is held to 1e-10 absolute.  Stage arrays (FP64)
are compared after undoing the per-node shift c_i the library applies.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu

LN2 = math.log(2.0)


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    c = B.Context(0)
    yield c
    c.close()


def _ds(n, m, arity, d, alpha=1.0, seed=0):
    return datagen.random_dag_data(n, m, arity, d, alpha, seed=seed)


# ------------------------------------------------------------------ step 1 --

@pytest.mark.parametrize("n,m,arity,seed", [
    (6, 200, 2, 1), (7, 3000, 3, 2), (8, 130, [2, 3, 4, 2, 5, 3, 2, 2], 3), (5, 64, 2, 4),
    (5, 1, 3, 5), (9, 2000, 2, 6)])
def test_counts_bit_exact(ctx, n, m, arity, seed):
    ds = _ds(n, m, arity, 3, seed=seed)
    d = min(3, n - 1)
    job = B.Job(ds.data, ds.arity, d)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        i = int(rng.integers(n))
        k = int(rng.integers(0, d + 1))
        cand = [p for p in range(n) if p != i]
        G = sum(1 << int(p) for p in rng.choice(cand, size=k, replace=False))
        want = orc.family_counts(ds.data, ds.arity, i, G)
        got = B.bn_debug_counts(ctx.h, job, i, G, want.shape[0])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("n,m,d,seed", [(10, 700, 8, 11), (12, 130, 6, 12), (9, 2000, 7, 13)])
def test_counts_bit_exact_binary_large_families(ctx, n, m, d, seed):
    """Binary data, families of 5..d parents: the counts of every cell, in
    the cell order (configuration, child value), against the oracle's."""
    ds = _ds(n, m, 2, 4, seed=seed)
    job = B.Job(ds.data, ds.arity, d)
    rng = np.random.default_rng(seed)
    for k in list(range(5, d + 1)) * 4:
        i = int(rng.integers(n))
        cand = [p for p in range(n) if p != i]
        G = sum(1 << int(p) for p in rng.choice(cand, size=k, replace=False))
        want = orc.family_counts(ds.data, ds.arity, i, G)
        got = B.bn_debug_counts(ctx.h, job, i, G, want.shape[0])
        np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("n,m,arity,d,seed,ess,rho", [
    (12, 200, 2, 3, 0, 1.0, None), (9, 700, 3, 4, 1, 1.0, None),
    (11, 300, 2, 8, 5, 1.0, None), (13, 97, 2, 6, 6, 3.0, [0.0, -0.5, -1.1, -1.6, -2.3, -2.9, -3.7]),
    (14, 500, 2, 5, 7, 1.0, None),
    (10, 333, [2, 3, 2, 4, 2, 3, 2, 2, 5, 2], 3, 2, 2.5, [0.0, -0.7, -1.9, -3.3]),
    (6, 0, 2, 2, 3, 1.0, None), (1, 50, 4, 0, 4, 1.0, None)])
def test_scores_match_oracle(ctx, n, m, arity, d, seed, ess, rho):
    ds = _ds(n, m, arity, d, seed=seed)
    masks, logB = ctx.scores(ds.data, ds.arity, d, ess=ess, log_rho=rho)
    om, ol = orc.scores(ds.data, ds.arity, d, ess=ess, log_rho=rho)
    np.testing.assert_array_equal(masks, om)
    np.testing.assert_allclose(logB, ol, atol=1e-10, rtol=0)


# -------------------------------------------------------- stages, FP64 --

@pytest.mark.parametrize("n,d,arity,m,seed", [(9, 3, 2, 150, 7), (11, 2, 3, 300, 8),
                                              (14, 4, 2, 400, 9)])
def test_stage_arrays_fp64(ctx, n, d, arity, m, seed):
    ds = _ds(n, m, arity, d, seed=seed)
    ref = orc.edge_posteriors(ds.data, ds.arity, d, stages=True)
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    K = orc.num_families(n, d)
    N = 1 << n
    full = N - 1
    c = B.bn_debug_stage(ctx.h, B.BN_STAGE_SHIFT, (n,), np.float64)
    np.testing.assert_allclose(c, ref["logB"].max(axis=1), atol=1e-10, rtol=0)
    A = B.bn_debug_stage(ctx.h, B.BN_STAGE_A, (n, N // 2), np.float64)
    F = B.bn_debug_stage(ctx.h, B.BN_STAGE_F, (N,), np.float64)
    Rc = B.bn_debug_stage(ctx.h, B.BN_STAGE_RC, (N,), np.float64)
    G = B.bn_debug_stage(ctx.h, B.BN_STAGE_GAMMA, (n, K), np.float64)
    S = np.arange(N)
    csum = np.array([sum(c[j] for j in range(n) if s >> j & 1) for s in range(N)])
    for i in range(n):
        low = (1 << i) - 1
        cidx = np.arange(N // 2)
        full_idx = (cidx & low) | ((cidx & ~low) << 1)
        np.testing.assert_allclose(A[i], ref["A"][i][full_idx] - c[i], atol=1e-9, rtol=0)
    np.testing.assert_allclose(F, ref["F"] - csum, atol=1e-9, rtol=0)
    np.testing.assert_allclose(Rc, ref["R"][full ^ S] - csum[full ^ S], atol=1e-9, rtol=0)
    # Gamma_v(G) reaches a posterior only through B_v(G) Gamma_v(G) / F(V)
    # (Eq. 11).  The 13-dimension tiles (n >= 14) may hold an output whose
    # product lies below F(V) e^-40 at a floor value instead (the relevance
    # cut, error below 2^-64 per posterior): every other entry is exact.
    shiftB = ref["logB"] - c[:, None]
    for v in range(n):
        want = ref["Gamma"][v] - (c.sum() - c[v])
        rel = shiftB[v] + want >= F[full] - 40.0
        np.testing.assert_allclose(G[v][rel], want[rel], atol=1e-9, rtol=0)
        assert np.all(shiftB[v][~rel] + G[v][~rel] < F[full] - 40.0)
        if n < 14:
            np.testing.assert_allclose(G[v], want, atol=1e-9, rtol=0)
    np.testing.assert_allclose(post, ref["post"], atol=1e-9, rtol=0)
    assert abs(lpd - ref["log_PD"]) < 1e-8


# --------------------------------------------------------- posteriors --

EDGE_CASES = [
    # n, d, arity, m, seed
    (1, 0, 2, 10, 1), (2, 1, 2, 50, 2), (2, 5, 3, 0, 3), (3, 2, 2, 0, 4), (4, 0, 2, 80, 5),
    (5, 4, 2, 120, 6), (5, 2, 3, 60, 7), (6, 3, [2, 3, 2, 4, 2, 2], 90, 8), (7, 1, 2, 1, 9),
    (8, 7, 2, 40, 10), (13, 3, 2, 250, 11), (15, 2, 3, 180, 12), (16, 3, 2, 500, 13),
]


@pytest.mark.parametrize("n,d,arity,m,seed", EDGE_CASES)
def test_posteriors_fp64_match_oracle(ctx, n, d, arity, m, seed):
    ds = _ds(n, m, arity, max(d, 1), seed=seed)
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    np.testing.assert_allclose(post, ref["post"], atol=1e-9, rtol=0)
    assert abs(lpd - ref["log_PD"]) <= 1e-9 * max(1.0, abs(ref["log_PD"]))


@pytest.mark.parametrize("n,d,arity,m,seed", EDGE_CASES)
def test_posteriors_fp32_match_oracle(ctx, n, d, arity, m, seed):
    ds = _ds(n, m, arity, max(d, 1), seed=seed)
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    np.testing.assert_allclose(post, ref["post"], atol=1e-4, rtol=0)


# In-degree bounds across the whole range on the 13-dimension tile path
# (n >= 14): no parents, single parents, bounds that make some tile columns
# long and others short, and d = n - 1 (every subset is a parent set).
TILE_CASES = [(14, 0), (14, 1), (14, 5), (15, 7), (15, 14), (17, 2)]


@pytest.mark.parametrize("n,d", TILE_CASES)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_tile_path_in_degree_range(ctx, n, d, precision, tol):
    ds = datagen.random_dag_data(n, 300, 2, min(max(d, 1), 3), 1.0, seed=40 + n + d)
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision=precision)
    np.testing.assert_allclose(post, ref["post"], atol=tol, rtol=0)
    if precision == "fp64":
        assert abs(lpd - ref["log_PD"]) <= 1e-9 * max(1.0, abs(ref["log_PD"]))


# A structure prior that grows steeply with the parent-set size spreads the
# values of an upward-zeta tile over thousands of log units: tiles whose high
# part H has few elements then span one, two, three or more single-scale
# windows of the 13-dimension tile (or fall back to its banded path),
# depending on |H|.  The windows are 206 bits (FP32) and 1300 nats (FP64).
@pytest.mark.parametrize("precision,step", [("fp64", 1000.0), ("fp32", 150.0)])
def test_stage_A_wide_spans(ctx, precision, step):
    n, d = 18, 4
    ds = _ds(n, 200, 2, 3, seed=77)
    rho = [step * k for k in range(d + 1)]
    ref = orc.edge_posteriors(ds.data, ds.arity, d, log_rho=rho, stages=True)
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, log_rho=rho, precision=precision)
    N = 1 << n
    c = B.bn_debug_stage(ctx.h, B.BN_STAGE_SHIFT, (n,), np.float64)
    dt = np.float64 if precision == "fp64" else np.float32
    A = B.bn_debug_stage(ctx.h, B.BN_STAGE_A, (n, N // 2), dt).astype(np.float64)
    assert np.all(np.isfinite(A))
    for i in range(n):
        low = (1 << i) - 1
        cidx = np.arange(N // 2)
        want = ref["A"][i][(cidx & low) | ((cidx & ~low) << 1)] - c[i]
        if precision == "fp64":
            np.testing.assert_allclose(A[i], want, atol=1e-9, rtol=0)
        else:                                   # log2 units, FP32 inputs
            want2 = want / np.log(2.0)
            np.testing.assert_allclose(A[i], want2, atol=1e-4, rtol=2e-6)
    tol = 1e-9 if precision == "fp64" else 1e-4
    np.testing.assert_allclose(post, ref["post"], atol=tol, rtol=0)


# Larger in-degree bounds on the 13-dimension tile path (the paper's d = 6
# and 8 of its sweep): other score kernels, longer row lists and more
# columns per tile, most phase-2 columns on the butterfly kernel.
LARGE_D = [(16, 6), (16, 8), (18, 6), (20, 6)]
_large_d_ref = {}


@pytest.mark.parametrize("n,d", LARGE_D)
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_large_in_degree_bounds(ctx, n, d, precision, tol):
    ds = datagen.random_dag_data(n, 500, 2, min(d, 4), 1.0, seed=300 + n + d)
    if (n, d) not in _large_d_ref:
        _large_d_ref[(n, d)] = orc.edge_posteriors(ds.data, ds.arity, d)
    ref = _large_d_ref[(n, d)]
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision=precision)
    np.testing.assert_allclose(post, ref["post"], atol=tol, rtol=0)
    if precision == "fp64":
        assert abs(lpd - ref["log_PD"]) <= 1e-9 * max(1.0, abs(ref["log_PD"]))


def test_small_config_both_paths(ctx):
    ds, d = datagen.config_small()
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    p64, l64 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    p32, l32 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    np.testing.assert_allclose(p64, ref["post"], atol=1e-9, rtol=0)
    np.testing.assert_allclose(p32, ref["post"], atol=1e-4, rtol=0)
    assert abs(l64 - ref["log_PD"]) < 1e-8


def test_mid_config_both_paths(ctx):
    ds, d = datagen.config_mid()
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    p64, l64 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    p32, l32 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    err32 = float(np.abs(p32 - ref["post"]).max())
    print(f"mid config: fp64 max err {np.abs(p64 - ref['post']).max():.3e}, fp32 {err32:.3e}")
    np.testing.assert_allclose(p64, ref["post"], atol=1e-9, rtol=0)
    np.testing.assert_allclose(p32, ref["post"], atol=1e-4, rtol=0)
    assert abs(l64 - ref["log_PD"]) <= 1e-9 * abs(ref["log_PD"])


def test_determinism(ctx):
    ds, d = datagen.config_small()
    a, _ = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    b, _ = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    c, _ = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    e, _ = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    assert np.array_equal(a, b) and np.array_equal(c, e)


def test_invalid_inputs_rejected(ctx):
    ds = _ds(5, 40, 2, 2, seed=3)
    bad = ds.data.copy()
    bad[3, 2] = 2                       # value not below its arity
    with pytest.raises(B.BnError) as ei:
        ctx.edge_posteriors(bad, ds.arity, 2)
    assert ei.value.code == B.BN_EINVAL
    with pytest.raises(B.BnError):
        ctx.edge_posteriors(ds.data, np.array([2, 2, 0, 2, 2], np.uint8), 2)
    with pytest.raises(B.BnError):
        ctx.edge_posteriors(ds.data, ds.arity, -1)
    with pytest.raises(B.BnError):
        ctx.edge_posteriors(ds.data, ds.arity, 2, ess=0.0)


def test_device_data_async_path(ctx):
    torch = pytest.importorskip("torch")
    ds, d = datagen.config_small()
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    data_dev = torch.from_numpy(ds.data).cuda()
    post_dev = torch.zeros((ds.n, ds.n), dtype=torch.float64, device="cuda")
    lpd_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    job = B.Job(data_dev, ds.arity, d, precision="fp64", m=ds.m)
    s = torch.cuda.current_stream()
    B.bn_edge_posteriors_async(ctx.h, job, post_dev, lpd_dev, s)
    torch.cuda.synchronize()
    np.testing.assert_allclose(post_dev.cpu().numpy(), ref["post"], atol=1e-9, rtol=0)
    assert abs(float(lpd_dev.item()) - ref["log_PD"]) < 1e-8


# ------------------------------------------------------- full size, n=26 --

def _lse(xs):
    m = max(xs)
    return m + math.log(sum(math.exp(x - m) for x in xs))


@pytest.fixture(scope="module")
def large_runs(ctx):
    ds, d = datagen.config_large()
    p32, l32 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    st32 = ctx.stats()
    p64, l64 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    st64 = ctx.stats()
    print("n=26 stats fp32", st32)
    print("n=26 stats fp64", st64)
    return ds, d, p32, l32, p64, l64


def test_large_properties_and_fp32_vs_fp64(large_runs):
    ds, d, p32, l32, p64, l64 = large_runs
    n = ds.n
    for P, tol in ((p32, 1e-4), (p64, 1e-9)):
        assert np.all(np.isfinite(P))
        assert np.all(P >= 0) and np.all(P <= 1 + tol)
        assert np.all(np.diag(P) == 0)
        assert np.all(P + P.T <= 1 + 2 * tol)           # acyclic: not both ways
        assert np.all(P.sum(axis=0) <= d + n * tol)     # in-degree bound
    err = float(np.abs(p32 - p64).max())
    print(f"n=26 max |fp32 - fp64| = {err:.3e}")
    assert err < 1e-4
    assert abs(l32 - l64) < 1e-3 * n


def test_large_sampled_scores_and_A(ctx, large_runs):
    """FP64 stage values at n=26 against the oracle computed one by one:
    sampled local scores, and sampled A_i(S) by direct summation over the
    parent sets inside S (Definition 1)."""
    ds, d, *_ = large_runs
    n = ds.n
    c = B.bn_debug_stage(ctx.h, B.BN_STAGE_SHIFT, (n,), np.float64)
    K = orc.num_families(n, d)
    logB = B.bn_debug_stage(ctx.h, B.BN_STAGE_LOGB, (n, K), np.float64)
    masks = B.bn_debug_stage(ctx.h, B.BN_STAGE_MASKS, (n, K), np.uint32)
    A = B.bn_debug_stage(ctx.h, B.BN_STAGE_A, (n, 1 << (n - 1)), np.float64)
    rng = np.random.default_rng(0)
    for _ in range(40):
        i = int(rng.integers(n))
        f = int(rng.integers(K))
        want = orc.family_score(ds.data, ds.arity, i, int(masks[i, f]))
        assert abs(logB[i, f] - want) < 1e-10
    for _ in range(6):
        i = int(rng.integers(n))
        members = [p for p in range(n) if p != i and rng.random() < 0.4][:9]
        S = sum(1 << p for p in members)
        terms = []
        sub = S
        while True:
            if bin(sub).count("1") <= d:
                terms.append(orc.family_score(ds.data, ds.arity, i, sub))
            if sub == 0:
                break
            sub = (sub - 1) & S
        low = (1 << i) - 1
        cidx = (S & low) | ((S >> 1) & ~low)
        assert abs(A[i, cidx] - (_lse(terms) - c[i])) < 1e-9
