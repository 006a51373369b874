"""Pins of the CPU FP64 oracle against facts that do not come from the oracle.

Each check below is an independent computation (brute force over orders or
DAGs, direct per-subset sums, sequential predictive probabilities, closed
forms, textbook invariants).  None re-types the oracle's own formula, so a
dropped term, a wrong sign or index, or a transposed operand anywhere in the
oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import datagen


def lse_list(xs):
    xs = [x for x in xs if x != -math.inf]
    if not xs:
        return -math.inf
    m = max(xs)
    return m + math.log(sum(math.exp(x - m) for x in xs))


def subsets_of(mask):
    """All submasks of ``mask``."""
    sub = mask
    while True:
        yield sub
        if sub == 0:
            return
        sub = (sub - 1) & mask


# ---------------------------------------------------------------- families --

@pytest.mark.parametrize("n,d", [(1, 0), (2, 1), (5, 2), (7, 3), (9, 9), (12, 3)])
def test_family_list_is_canonical(n, d):
    """Families of node i: every G subset V-{i}, |G|<=d, exactly once, sorted by
    (|G|, mask value)."""
    dd = min(d, n - 1)
    for i in range(n):
        got = orc.family_list(n, d, i).tolist()
        want = sorted((m for m in range(1 << n)
                       if not (m >> i) & 1 and bin(m).count("1") <= dd),
                      key=lambda m: (bin(m).count("1"), m))
        assert got == want


# ------------------------------------------------------------------ counts --

@pytest.mark.parametrize("arity", [2, 3, [2, 3, 4, 2, 5, 3]])
def test_counts_match_bincount(arity):
    ds = datagen.random_dag_data(6, 317, arity, 3, 1.0, seed=11)
    rng = np.random.default_rng(5)
    for _ in range(25):
        i = int(rng.integers(6))
        G = int(rng.integers(64)) & ~(1 << i)
        got = orc.family_counts(ds.data, ds.arity, i, G)
        idx = np.zeros(ds.m, dtype=np.int64)
        stride = 1
        for p in range(6):
            if G >> p & 1:
                idx += ds.data[:, p].astype(np.int64) * stride
                stride *= int(ds.arity[p])
        cell = idx * int(ds.arity[i]) + ds.data[:, i]
        want = np.bincount(cell, minlength=stride * int(ds.arity[i]))
        np.testing.assert_array_equal(got, want)


# -------------------------------------------------------------------- BDeu --

def polya_log_marginal(data, arity, i, G, ess):
    """BDeu marginal likelihood as the product of sequential predictive
    probabilities of a Dirichlet-multinomial (Polya urn): no lgamma."""
    n = len(arity)
    parents = [p for p in range(n) if G >> p & 1]
    q = int(np.prod([int(arity[p]) for p in parents])) if parents else 1
    r = int(arity[i])
    a_jk = ess / (q * r)
    a_j = ess / q
    Njk = {}
    Nj = {}
    total = 0.0
    for row in data:
        j = 0
        stride = 1
        for p in parents:
            j += int(row[p]) * stride
            stride *= int(arity[p])
        k = int(row[i])
        total += math.log((a_jk + Njk.get((j, k), 0)) / (a_j + Nj.get(j, 0)))
        Njk[(j, k)] = Njk.get((j, k), 0) + 1
        Nj[j] = Nj.get(j, 0) + 1
    return total


@pytest.mark.parametrize("ess", [1.0, 0.3, 7.5])
def test_bdeu_equals_sequential_predictive(ess):
    ds = datagen.random_dag_data(5, 400, [2, 3, 2, 4, 3], 2, 0.7, seed=3)
    for i in range(5):
        for G in (0, 0b00011, 0b10100, 0b11010):
            G &= ~(1 << i)
            got = orc.family_score(ds.data, ds.arity, i, G, ess=ess)
            want = polya_log_marginal(ds.data, ds.arity, i, G, ess)
            assert abs(got - want) < 1e-9 * max(1.0, abs(want))


def test_bdeu_score_equivalence():
    """Markov-equivalent DAGs get equal BDeu scores (a textbook property of
    BDeu); a v-structure is not equivalent to a chain."""
    ds = datagen.random_dag_data(3, 500, [2, 3, 4], 2, 0.8, seed=9)
    s = lambda i, *ps: orc.family_score(ds.data, ds.arity, i, sum(1 << p for p in ps))
    for a, b in itertools.permutations(range(3), 2):
        assert abs((s(a) + s(b, a)) - (s(b) + s(a, b))) < 1e-9
    chain = s(0) + s(1, 0) + s(2, 1)           # 0 -> 1 -> 2
    rev = s(2) + s(1, 2) + s(0, 1)             # 2 -> 1 -> 0
    fork = s(1) + s(0, 1) + s(2, 1)            # 0 <- 1 -> 2
    vstruct = s(0) + s(2) + s(1, 0, 2)         # 0 -> 1 <- 2
    assert abs(chain - rev) < 1e-9 and abs(chain - fork) < 1e-9
    assert abs(chain - vstruct) > 1e-6


def test_bdeu_no_data_is_zero():
    arity = np.array([2, 3, 2], dtype=np.uint8)
    data = np.zeros((0, 3), dtype=np.uint8)
    for i in range(3):
        for G in range(8):
            if not G >> i & 1:
                assert orc.family_score(data, arity, i, G) == 0.0


# ------------------------------------------------------------- zeta pins --

def _rand_int_table(n, rng, hi=9, dmax=None):
    s = rng.integers(0, hi + 1, size=1 << n).astype(np.float64)
    if dmax is not None:
        for S in range(1 << n):
            if bin(S).count("1") > dmax:
                s[S] = 0.0
    return s


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_upzeta_equals_definition_1(n):
    rng = np.random.default_rng(n)
    for d in range(0, n + 1):
        s = _rand_int_table(n, rng)
        with np.errstate(divide="ignore"):
            t = orc.upzeta(n, d, np.log(s))
        for T in range(1 << n):
            want = sum(s[S] for S in subsets_of(T) if bin(S).count("1") <= d)
            got = math.exp(t[T]) if t[T] != -math.inf else 0.0
            assert abs(got - want) <= 1e-12 * max(1.0, want)


@pytest.mark.parametrize("n", [1, 3, 5, 7])
def test_downzeta_equals_definition_2(n):
    rng = np.random.default_rng(100 + n)
    full = (1 << n) - 1
    for d in range(0, n + 1):
        s = _rand_int_table(n, rng)
        with np.errstate(divide="ignore"):
            t = orc.downzeta(n, d, np.log(s))
        for T in range(1 << n):
            if bin(T).count("1") > d:
                continue
            want = sum(s[S] for S in subsets_of(full) if S & T == T)
            got = math.exp(t[T]) if t[T] != -math.inf else 0.0
            assert abs(got - want) <= 1e-12 * max(1.0, want)


# ------------------------------------------------------------ F and R pins --

@pytest.mark.parametrize("n", [1, 2, 4, 5])
def test_forward_backward_equal_sums_over_orders(n):
    """F(S) = sum over orderings s1..sl of S of prod_t A_st({s1..s(t-1)});
    R(S) = the same with every predecessor set enlarged by V-S."""
    rng = np.random.default_rng(42 + n)
    N = 1 << n
    full = N - 1
    A = rng.normal(size=(n, N)) * 2.0
    F = orc.forward(n, A)
    R = orc.backward(n, A)
    for S in range(N):
        members = [i for i in range(n) if S >> i & 1]
        fw, bw = [], []
        for perm in itertools.permutations(members):
            pre_f, pre_b = 0, full & ~S
            wf = wb = 0.0
            for v in perm:
                wf += A[v, pre_f]
                wb += A[v, pre_b]
                pre_f |= 1 << v
                pre_b |= 1 << v
            fw.append(wf)
            bw.append(wb)
        assert abs(F[S] - lse_list(fw)) < 1e-11 * max(1.0, abs(F[S]))
        assert abs(R[S] - lse_list(bw)) < 1e-11 * max(1.0, abs(R[S]))
    assert abs(F[full] - R[full]) < 1e-11 * max(1.0, abs(F[full]))


# ------------------------------------------------------ posterior pins --

def brute_force_orders(n, d, masks, logB):
    """Eq. 3-5 written out: sum over all n! orders of the product over nodes of
    the sum over parent sets inside the predecessor set.  Returns (post,
    log P(D))."""
    fam = [dict(zip(masks[i].tolist(), logB[i].tolist())) for i in range(n)]
    tot, joint = [], {}
    for perm in itertools.permutations(range(n)):
        pre = 0
        terms_all = []
        terms_edge = {}
        pos = {}
        for v in perm:
            terms_all.append(lse_list([fam[v][G] for G in subsets_of(pre)
                                       if G in fam[v]]))
            for u in range(n):
                if pre >> u & 1:
                    terms_edge[(u, v)] = lse_list(
                        [fam[v][G] for G in subsets_of(pre) if G in fam[v] and G >> u & 1])
            pos[v] = len(pos)
            pre |= 1 << v
        w = sum(terms_all)
        tot.append(w)
        for (u, v), e in terms_edge.items():
            joint.setdefault((u, v), []).append(w - terms_all[pos[v]] + e)
    lpd = lse_list(tot)
    post = np.zeros((n, n))
    for (u, v), ws in joint.items():
        post[u, v] = math.exp(lse_list(ws) - lpd)
    return post, lpd


@pytest.mark.parametrize("n,d,arity,m,seed", [
    (3, 1, 2, 60, 1), (4, 2, 3, 80, 2), (5, 1, 2, 150, 3), (5, 3, [2, 3, 2, 2, 4], 90, 4),
    (6, 2, 2, 120, 5), (6, 5, 2, 40, 6)])
def test_posteriors_match_sum_over_all_orders(n, d, arity, m, seed):
    ds = datagen.random_dag_data(n, m, arity, min(d, 3), 0.6, seed=seed)
    out = orc.edge_posteriors(ds.data, ds.arity, d)
    masks, logB = orc.scores(ds.data, ds.arity, d)
    post, lpd = brute_force_orders(n, d, masks, logB)
    np.testing.assert_allclose(out["post"], post, atol=1e-12, rtol=0)
    assert abs(out["log_PD"] - lpd) < 1e-11 * max(1.0, abs(lpd))


def count_linear_extensions(n, parents):
    c = 0
    for perm in itertools.permutations(range(n)):
        pos = {v: k for k, v in enumerate(perm)}
        if all(pos[p] < pos[v] for v in range(n) for p in parents[v]):
            c += 1
    return c


@pytest.mark.parametrize("n,d,seed", [(3, 2, 1), (4, 1, 2), (4, 2, 3), (4, 3, 4)])
def test_posteriors_match_dag_enumeration(n, d, seed):
    """Enumerate every DAG with in-degree <= d; under the order-modular prior
    with q = 1 its weight is (number of linear extensions) * prod_i B_i(G_i)."""
    ds = datagen.random_dag_data(n, 70, 2, d, 0.5, seed=seed)
    out = orc.edge_posteriors(ds.data, ds.arity, d)
    cand = []
    for i in range(n):
        cand.append([G for G in range(1 << n)
                     if not G >> i & 1 and bin(G).count("1") <= d])
    score = {}
    for i in range(n):
        for G in cand[i]:
            score[(i, G)] = orc.family_score(ds.data, ds.arity, i, G)
    ws, edge_ws = [], {}
    for choice in itertools.product(*cand):
        parents = [[p for p in range(n) if choice[v] >> p & 1] for v in range(n)]
        ext = count_linear_extensions(n, parents)
        if ext == 0:
            continue                              # cyclic
        w = math.log(ext) + sum(score[(i, choice[i])] for i in range(n))
        ws.append(w)
        for v in range(n):
            for u in parents[v]:
                edge_ws.setdefault((u, v), []).append(w)
    Z = lse_list(ws)
    want = np.zeros((n, n))
    for (u, v), e in edge_ws.items():
        want[u, v] = math.exp(lse_list(e) - Z)
    np.testing.assert_allclose(out["post"], want, atol=1e-12, rtol=0)


def test_two_variables_closed_form():
    ds = datagen.random_dag_data(2, 300, [3, 2], 1, 0.5, seed=8)
    out = orc.edge_posteriors(ds.data, ds.arity, 1)
    b1, b1p = orc.family_score(ds.data, ds.arity, 0, 0), orc.family_score(ds.data, ds.arity, 0, 2)
    b2, b2p = orc.family_score(ds.data, ds.arity, 1, 0), orc.family_score(ds.data, ds.arity, 1, 1)
    # P(1->2) = B1(0) B2({1}) / [B1(0)(B2(0)+B2({1})) + B2(0)(B1(0)+B1({2}))]
    num = b1 + b2p
    den = lse_list([b1 + lse_list([b2, b2p]), b2 + lse_list([b1, b1p])])
    assert abs(out["post"][0, 1] - math.exp(num - den)) < 1e-13
    num21 = b2 + b1p
    assert abs(out["post"][1, 0] - math.exp(num21 - den)) < 1e-13


def empty_data_posterior(n, d):
    """m = 0 and rho = 1: every order has the same weight, so
    P(u->v) = (1/n) sum_{l=1}^{n-1} (l/(n-1)) sum_{k=1}^{d} C(l-1,k-1) / sum_{k=0}^{d} C(l,k)."""
    tot = 0.0
    for l in range(1, n):
        num = sum(math.comb(l - 1, k - 1) for k in range(1, d + 1))
        den = sum(math.comb(l, k) for k in range(0, d + 1))
        tot += (l / (n - 1)) * num / den
    return tot / n


@pytest.mark.parametrize("n,d", [(2, 1), (4, 2), (5, 1), (6, 3), (9, 2)])
def test_empty_data_closed_form(n, d):
    arity = np.full(n, 2, dtype=np.uint8)
    out = orc.edge_posteriors(np.zeros((0, n), dtype=np.uint8), arity, d)
    want = empty_data_posterior(n, d)
    off = ~np.eye(n, dtype=bool)
    np.testing.assert_allclose(out["post"][off], want, atol=1e-13, rtol=0)
    assert np.all(np.diag(out["post"]) == 0)


def test_empty_data_golden_value():
    """n=4, d=2, no data: 39/168 (closed form above, evaluated by hand)."""
    with open(__file__.replace("test_oracle_pins.py", "golden/empty_data_n4_d2.txt")) as f:
        val = float([ln for ln in f if not ln.startswith("#")][0])
    out = orc.edge_posteriors(np.zeros((0, 4), dtype=np.uint8),
                              np.full(4, 2, dtype=np.uint8), 2)
    assert abs(out["post"][0, 1] - val) < 1e-12
    assert abs(val - 39.0 / 168.0) < 1e-12


def test_in_degree_zero_gives_zero_posteriors():
    ds = datagen.random_dag_data(7, 200, 2, 2, 1.0, seed=4)
    out = orc.edge_posteriors(ds.data, ds.arity, 0)
    assert np.all(out["post"] == 0.0)


@pytest.mark.parametrize("n,d,arity,seed", [(8, 3, 2, 12), (9, 2, 3, 13), (10, 4, 2, 14)])
def test_posterior_invariants(n, d, arity, seed):
    ds = datagen.random_dag_data(n, 300, arity, d, 1.0, seed=seed)
    out = orc.edge_posteriors(ds.data, ds.arity, d, stages=True)
    P = out["post"]
    assert np.all(P >= 0) and np.all(P <= 1 + 1e-12)
    assert np.all(P + P.T <= 1 + 1e-12)                 # acyclic: not both ways
    assert np.all(P.sum(axis=0) <= d + 1e-9)            # in-degree bound
    full = (1 << n) - 1
    assert abs(out["F"][full] - out["R"][full]) < 1e-9
    for v in range(n):                                  # sum_G B_v Gamma_v = F(V)
        z = lse_list((out["logB"][v] + out["Gamma"][v]).tolist())
        assert abs(z - out["log_PD"]) < 1e-9


def test_rho_per_size_prior_matches_orders():
    """A non-uniform per-size prior rho(|G|) enters B_i (Eq. 6)."""
    ds = datagen.random_dag_data(5, 100, 2, 2, 0.5, seed=21)
    log_rho = np.array([0.0, -1.3, -2.9])
    out = orc.edge_posteriors(ds.data, ds.arity, 2, log_rho=log_rho)
    masks, logB = orc.scores(ds.data, ds.arity, 2)
    sizes = np.vectorize(lambda m: bin(int(m)).count("1"))(masks)
    post, _ = brute_force_orders(5, 2, masks, logB + log_rho[sizes])
    np.testing.assert_allclose(out["post"], post, atol=1e-12, rtol=0)


def test_golden_small_config_regression():
    """Posteriors of the n=12 workload stored by tests/golden/make_golden.py
    (which calls only the oracle)."""
    path = __file__.replace("test_oracle_pins.py", "golden/small_n12_d3_posteriors.txt")
    rows = [ln for ln in open(path) if not ln.startswith("#")]
    lpd = float(rows[0])
    want = np.array([[float(x) for x in ln.split()] for ln in rows[1:]])
    ds, d = datagen.config_small()
    out = orc.edge_posteriors(ds.data, ds.arity, d)
    assert abs(out["log_PD"] - lpd) < 1e-9
    np.testing.assert_allclose(out["post"], want, atol=1e-12, rtol=0)


# ------------------------------------- order prior q, family weights, features --

def brute_force_general(n, masks, logB, log_q=None, log_f=None):
    """Eq. 5 written out over all n! orders, with the order prior q_i(L_i) of
    Eq. 4 (log_q[i, |L_i|]) and a modular feature (log_f[i] per family, as
    logB): returns (log P(f, D), {(u, v): log P(u->v, f=1 elsewhere, D)})."""
    fam = [dict(zip(masks[i].tolist(), logB[i].tolist())) for i in range(n)]
    ff = None if log_f is None else [dict(zip(masks[i].tolist(), log_f[i].tolist()))
                                     for i in range(n)]
    tot, joint = [], {}
    for perm in itertools.permutations(range(n)):
        pre = 0
        w = 0.0
        node_terms = {}
        edge_terms = {}
        for v in perm:
            q = 0.0 if log_q is None else log_q[v][bin(pre).count("1")]
            subs = [G for G in subsets_of(pre) if G in fam[v]]
            t = q + lse_list([fam[v][G] + (0.0 if ff is None else ff[v][G]) for G in subs])
            node_terms[v] = t
            w += t
            for u in range(n):
                if pre >> u & 1:
                    edge_terms[(u, v)] = q + lse_list([fam[v][G] for G in subs if G >> u & 1])
            pre |= 1 << v
        tot.append(w)
        if ff is None:
            for (u, v), e in edge_terms.items():
                joint.setdefault((u, v), []).append(w - node_terms[v] + e)
    return lse_list(tot), {k: lse_list(ws) for k, ws in joint.items()}


def _rand_q_w(n, K, rng, zeros=0.0):
    log_q = rng.normal(0.0, 1.5, size=(n, n))
    log_w = rng.normal(0.0, 1.0, size=(n, K))
    if zeros:
        log_w[rng.random((n, K)) < zeros] = -math.inf
        log_w[:, 0] = 0.0                                  # keep every node a parent set
    return log_q, log_w


@pytest.mark.parametrize("n,d,arity,seed", [(4, 2, 3, 31), (5, 3, [2, 3, 2, 2, 4], 32),
                                            (6, 2, 2, 33)])
def test_order_prior_and_family_weights_match_orders(n, d, arity, seed):
    """q_i(S) by |S| (Eq. 4, 7, 12) and per-family weights (a general
    rho_i(G)), some of them zero: Algorithm 1 against the sum over orders."""
    ds = datagen.random_dag_data(n, 90, arity, min(d, 3), 0.6, seed=seed)
    masks, logB = orc.scores(ds.data, ds.arity, d)
    rng = np.random.default_rng(seed)
    log_q, log_w = _rand_q_w(n, masks.shape[1], rng, zeros=0.25)
    out = orc.edge_posteriors(ds.data, ds.arity, d, log_q=log_q, log_w=log_w)
    lpd, joint = brute_force_general(n, masks, logB + log_w, log_q=log_q)
    assert abs(out["log_PD"] - lpd) < 1e-11 * max(1.0, abs(lpd))
    want = np.zeros((n, n))
    for (u, v), lj in joint.items():
        want[u, v] = math.exp(lj - lpd)
    np.testing.assert_allclose(out["post"], want, atol=1e-12, rtol=0)


def test_constant_order_prior_changes_only_the_normaliser():
    """q_i(S) = c_i for every S scales every order by prod_i c_i: posteriors
    unchanged, log P(D) shifted by sum_i log c_i."""
    ds = datagen.random_dag_data(7, 200, 2, 3, 0.8, seed=34)
    c = np.linspace(-2.0, 3.0, 7)
    log_q = np.repeat(c[:, None], 7, axis=1)
    a = orc.edge_posteriors(ds.data, ds.arity, 3)
    b = orc.edge_posteriors(ds.data, ds.arity, 3, log_q=log_q)
    np.testing.assert_allclose(b["post"], a["post"], atol=1e-12, rtol=0)
    assert abs(b["log_PD"] - a["log_PD"] - c.sum()) < 1e-9


@pytest.mark.parametrize("n,d,seed", [(4, 2, 35), (5, 2, 36), (6, 3, 37)])
def test_feature_posterior_matches_orders(n, d, seed):
    """A random modular feature (each f_i a random 0/1 pattern over the parent
    sets, f_i(empty) = 1 so that f has positive probability), with q and
    weights: P(f | D) = P(f, D) / P(D) against the sum over orders."""
    ds = datagen.random_dag_data(n, 120, 2, min(d, 3), 0.7, seed=seed)
    masks, logB = orc.scores(ds.data, ds.arity, d)
    rng = np.random.default_rng(seed)
    log_q, log_w = _rand_q_w(n, masks.shape[1], rng)
    log_f = np.where(rng.random(masks.shape) < 0.4, -math.inf, 0.0)
    log_f[:, 0] = 0.0
    p, lpfd = orc.feature_posterior(ds.data, ds.arity, d, log_f, log_q=log_q, log_w=log_w)
    want_fd, _ = brute_force_general(n, masks, logB + log_w, log_q=log_q, log_f=log_f)
    want_d, _ = brute_force_general(n, masks, logB + log_w, log_q=log_q)
    assert abs(lpfd - want_fd) < 1e-11 * max(1.0, abs(want_fd))
    assert abs(p - math.exp(want_fd - want_d)) < 1e-12


def test_edge_feature_equals_forward_backward_edge_posterior():
    """The feature 'u -> v' (f_v(G) = [u in G], f_i = 1 otherwise) through the
    single-feature DP (Eqs. 5-9) equals P(u -> v | D) from the
    forward-backward path (Eqs. 10-12), with q and weights: two algorithms."""
    n, d = 8, 3
    ds = datagen.random_dag_data(n, 300, 2, 3, 0.8, seed=38)
    K = orc.num_families(n, d)
    rng = np.random.default_rng(38)
    log_q, log_w = _rand_q_w(n, K, rng)
    out = orc.edge_posteriors(ds.data, ds.arity, d, log_q=log_q, log_w=log_w)
    masks, _ = orc.scores(ds.data, ds.arity, d)
    for (u, v) in [(0, 1), (3, 7), (6, 2), (5, 4)]:
        log_f = np.zeros((n, K))
        log_f[v] = np.where((masks[v] >> u) & 1, 0.0, -math.inf)
        p, _ = orc.feature_posterior(ds.data, ds.arity, d, log_f, log_q=log_q, log_w=log_w)
        assert abs(p - out["post"][u, v]) < 1e-12


def test_trivial_and_impossible_features():
    """f = 1 gives P = 1 and log P(f, D) = log P(D); f_i = 0 for every parent
    set of one node gives P = 0."""
    ds = datagen.random_dag_data(6, 100, 2, 2, 1.0, seed=39)
    K = orc.num_families(6, 2)
    p, lpfd = orc.feature_posterior(ds.data, ds.arity, 2, np.zeros((6, K)))
    assert abs(p - 1.0) < 1e-14
    assert abs(lpfd - orc.edge_posteriors(ds.data, ds.arity, 2)["log_PD"]) < 1e-12
    log_f = np.zeros((6, K))
    log_f[4] = -math.inf
    p, lpfd = orc.feature_posterior(ds.data, ds.arity, 2, log_f)
    assert p == 0.0 and lpfd == -math.inf
