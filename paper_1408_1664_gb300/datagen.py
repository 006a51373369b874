"""Seeded synthetic inputs: discrete data sampled from a random DAG.

This module only draws random inputs.  It holds none of the method's
arithmetic (no scores, no transforms, no sums over orders), so both the CPU
oracle and the CUDA library can consume its output without sharing code.

The paper's experiments use synthetic discrete data sets of 500 samples
(Section 4.2) but do not state the generator.  The recipe here:

  * ``rng = numpy.random.default_rng(seed)``;
  * a random permutation ``pi`` of the n variables fixes a topological order;
  * the variable at position p draws k ~ U{0..min(max_parents, p)} parents,
    without replacement, from the variables before it;
  * every row of every conditional probability table is drawn from
    Dirichlet(alpha * 1_r);
  * samples are drawn ancestrally.

Variable i (0-based) is bit i of a subset bitmask everywhere in this project
(the paper numbers variables 1..n and uses bit i-1 for variable i, Section
3.1.1).  Parent configurations are mixed-radix numbers with the
lowest-numbered parent least significant.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Dataset:
    """m samples of n discrete variables plus the DAG they were drawn from."""

    data: np.ndarray          # (m, n) uint8, data[s, i] < arity[i]
    arity: np.ndarray         # (n,) uint8, every entry >= 1
    parents: list = field(default_factory=list)  # true parent lists (sorted)
    seed: int = 0

    @property
    def n(self) -> int:
        return int(self.arity.shape[0])

    @property
    def m(self) -> int:
        return int(self.data.shape[0])


def random_dag_data(n: int, m: int, arity, max_parents: int, alpha: float,
                    seed: int) -> Dataset:
    """Draw ``m`` samples of ``n`` variables from a seeded random DAG.

    ``arity`` is an int (all variables share it) or a length-n sequence.
    """
    rng = np.random.default_rng(seed)
    if np.isscalar(arity):
        ar = np.full(n, int(arity), dtype=np.int64)
    else:
        ar = np.asarray(arity, dtype=np.int64).copy()
        assert ar.shape == (n,)
    assert np.all(ar >= 1) and np.all(ar <= 255)
    perm = rng.permutation(n)
    parents: list = [[] for _ in range(n)]
    for pos, node in enumerate(perm):
        k = int(rng.integers(0, min(max_parents, pos) + 1))
        if k:
            chosen = rng.choice(perm[:pos], size=k, replace=False)
            parents[node] = sorted(int(c) for c in chosen)
    cpts = []
    for node in range(n):
        q = int(np.prod([ar[p] for p in parents[node]])) if parents[node] else 1
        cpts.append(rng.dirichlet(np.full(int(ar[node]), float(alpha)), size=q))
    data = np.zeros((m, n), dtype=np.uint8)
    for node in perm:
        cfg = np.zeros(m, dtype=np.int64)
        stride = 1
        for p in parents[node]:          # ascending: lowest parent least significant
            cfg += data[:, p].astype(np.int64) * stride
            stride *= int(ar[p])
        cum = np.cumsum(cpts[node], axis=1)
        cum[:, -1] = 1.0
        u = rng.random(m)
        x = (u[:, None] >= cum[cfg]).sum(axis=1)
        data[:, node] = np.minimum(x, ar[node] - 1).astype(np.uint8)
    return Dataset(data=data, arity=ar.astype(np.uint8), parents=parents, seed=seed)


# ---------------------------------------------------------------------------
# Named workloads.  Shapes follow the paper's experiments (n 21..33, d 2..8,
# 500 samples) and the stated configurations; values are synthetic.
# ---------------------------------------------------------------------------

def config_small() -> tuple[Dataset, int]:
    """n=12 binary, d=3, m=200, seed 0, Dirichlet(1,1) CPTs."""
    return random_dag_data(12, 200, 2, 3, 1.0, seed=0), 3


def config_mid() -> tuple[Dataset, int]:
    """n=20, arity 3, d=4, m=1000, seed 1, Dirichlet(0.5) CPTs."""
    return random_dag_data(20, 1000, 3, 4, 0.5, seed=1), 4


def config_large() -> tuple[Dataset, int]:
    """n=26 binary, d=4, m=2000, seed 2, Dirichlet(1) CPTs (full 2^26 lattice)."""
    return random_dag_data(26, 2000, 2, 4, 1.0, seed=2), 4


def batched_job(j: int) -> tuple[Dataset, int]:
    """Job j of the batched workload: seed 1000+j, n~U[10,18], d=3,
    arity~U{2,3} (one arity per job), m~U[100,1000], Dirichlet(1)."""
    rng = np.random.default_rng(1000 + j)
    n = int(rng.integers(10, 19))
    r = int(rng.integers(2, 4))
    m = int(rng.integers(100, 1001))
    return random_dag_data(n, m, r, 3, 1.0, seed=1000 + j), 3


def served_job(j: int, big: bool = False) -> tuple[Dataset, int]:
    """Job j of the served workload: n~U[8,22], d=3, binary, m=500; the
    periodic big job is n=29, d=3, m=2000."""
    rng = np.random.default_rng(2_000_000 + j)
    if big:
        return random_dag_data(29, 2000, 2, 3, 1.0, seed=3_000_000 + j), 3
    n = int(rng.integers(8, 23))
    return random_dag_data(n, 500, 2, 3, 1.0, seed=2_000_000 + j), 3


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int = 7) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate_per_s))
        if t >= duration_s:
            return np.asarray(out)
        out.append(t)
