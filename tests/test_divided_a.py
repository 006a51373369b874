"""The identity behind a split job's divided A, pinned on the CPU against the
oracle's A (Eq. 7 by Algorithm 2 over the whole lattice).

With the top k variables fixed to a rank's bits r (nl = n - k low variables),
every entry a rank reads is a truncated zeta transform over the low
variables alone of the score table folded over the top bits:
  low node i:    A_i(r + L) = sum over G <= L of  sum over G_t <= r,
                 |G_t| + |G| <= d, of B_i(G_t + G);
  top variable t: A_t(r' + L), r' = r - {t}, L over all low variables, as
                 X1(L) (families without variable 0) plus, when 0 is in L,
                 X2(L - {0}) (families with variable 0).
The library's k_fold_scores / k_top_slabs compute exactly these sums on the
GPU; here they are formed from the oracle's family scores and transformed by
the oracle's own truncated up-zeta, then compared with the oracle's full A
for every rank and every entry."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import datagen


def _lse(xs):
    xs = [x for x in xs if x != -np.inf]
    if not xs:
        return -np.inf
    m = max(xs)
    return m + np.log(sum(np.exp(x - m) for x in xs))


def _subsets(x):
    t = x
    while True:
        yield t
        if t == 0:
            return
        t = (t - 1) & x


@pytest.mark.parametrize("n,d,k", [(8, 3, 1), (9, 2, 2), (9, 4, 3)])
def test_folded_slabs_equal_the_oracle_A(n, d, k):
    ds = datagen.random_dag_data(n=n, m=200, arity=2, max_parents=3, alpha=1.0, seed=40 + n + k)
    ref = orc.edge_posteriors(ds.data, ds.arity, d, stages=("A", "logB", "masks"))
    A, logB, masks = ref["A"], ref["logB"], ref["masks"]
    score = [{int(g): float(v) for g, v in zip(masks[i], logB[i])} for i in range(n)]
    nl = n - k
    NL = 1 << nl

    def folded(node, G, tops):
        if bin(G).count("1") > d:
            return -np.inf
        return _lse([score[node][G | (t << nl)] for t in _subsets(tops)
                     if bin(G).count("1") + bin(t).count("1") <= d])

    worst = 0.0
    for r in range(1 << k):
        for i in range(nl):                                    # low nodes
            s = np.array([-np.inf if L >> i & 1 else folded(i, L, r) for L in range(NL)])
            z = orc.upzeta(nl, d, s)
            for L in range(NL):
                if L >> i & 1:
                    continue
                want = A[i, L | (r << nl)]
                worst = max(worst, abs(z[L] - want))
        for q in range(k):                                     # top variables
            t, tops = nl + q, r & ~(1 << q)
            s1 = np.array([-np.inf if L & 1 else folded(t, L, tops) for L in range(NL)])
            s2 = np.array([-np.inf if L & 1 else folded(t, L | 1, tops) for L in range(NL)])
            x1, x2 = orc.upzeta(nl, d, s1), orc.upzeta(nl, d, s2)
            for L in range(NL):
                got = x1[L] if not L & 1 else np.logaddexp(x1[L], x2[L & ~1])
                want = A[t, L | (tops << nl)]
                worst = max(worst, abs(got - want))
    assert worst <= 1e-10, worst
