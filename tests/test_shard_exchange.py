"""The exchange schedule of a job split over ranks (paper_1408_1664_gb300.shard),
run on gloo ranks on the CPU.

Each rank drives a CPU stand-in of the library's shard with the same
interface and the same partition rule: subsets S are grouped into tiles of
2^B by their low B bits, the tile index S >> B has H = n - B bits, and its top
k bits name the rank.  The stand-in computes F (Eq. 9) and R'(T) = R(V - T)
(Eq. 10) for its own tiles only, from the oracle's A, and refuses to read a
value it does not hold (NaN) -- so a schedule that computes a level before
the levels it reads have arrived, or an exchange that drops or misplaces a
row, fails here.  After both sweeps every rank must hold the oracle's F and R
in full, and its endpoints' posterior columns (Gamma_v by Eq. 12, the edge
sums by Eq. 11, written out below by brute force over subsets) summed over
the ranks must equal the oracle's posteriors.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _lse(xs):
    xs = [x for x in xs if x != -np.inf]
    if not xs:
        return -np.inf
    m = max(xs)
    return m + np.log(sum(np.exp(x - m) for x in xs))


class CpuShard:
    """The library's shard interface on numpy arrays (FP64, natural log)."""

    def __init__(self, n, d, B, A, logB, masks, rank, world):
        self.n, self.d, self.B, self.A = n, d, B, A
        self.logB, self.masks = logB, masks
        self.rank, self.world = rank, world
        self.k = world.bit_length() - 1
        self.levels = n - B                   # H: tile levels 0..H
        N = 1 << n
        self.F = np.full(N, np.nan)
        self.Rc = np.full(N, np.nan)          # R'(T) = R(V - T)
        self._acc = {}

    # the partition ----------------------------------------------------
    def owner(self, t):
        return t >> (self.levels - self.k)

    def tiles(self, hl, r):
        return [t for t in range(1 << self.levels)
                if bin(t).count("1") == hl and self.owner(t) == r]

    def _get(self, X, S):
        v = X[S]
        if np.isnan(v):
            raise AssertionError(f"rank {self.rank} read subset {S:#x} before it arrived")
        return v

    # Shard interface --------------------------------------------------
    def prepare(self, stream=None):
        pass

    def level(self, sweep, hl, stream=None):
        n, B = self.n, self.B
        full = (1 << n) - 1
        for t in self.tiles(hl, self.rank):
            subs = [(t << B) | lo for lo in range(1 << B)]
            if sweep == 0:                    # F by increasing popcount
                for S in sorted(subs, key=lambda S: bin(S).count("1")):
                    if S == 0:
                        self.F[S] = 0.0
                        continue
                    self.F[S] = _lse([self.A[i, S ^ (1 << i)] + self._get(self.F, S ^ (1 << i))
                                      for i in range(n) if S >> i & 1])
            else:                             # R' by decreasing popcount
                for T in sorted(subs, key=lambda S: -bin(S).count("1")):
                    if T == full:
                        self.Rc[T] = 0.0
                        continue
                    self.Rc[T] = _lse([self.A[i, T] + self._get(self.Rc, T | (1 << i))
                                       for i in range(n) if not T >> i & 1])

    def exchange_bytes(self, hl):
        rows = max(len(self.tiles(hl, r)) for r in range(self.world))
        return 16 + rows * (1 << self.B) * 8

    def _rows(self, hl, r):
        return np.array([(t << self.B) | lo for t in self.tiles(hl, r)
                         for lo in range(1 << self.B)], dtype=np.int64)

    def pack(self, sweep, hl, buf, stream=None):
        X = self.Rc if sweep else self.F
        idx = self._rows(hl, self.rank)
        view = buf[16:16 + 8 * len(idx)].numpy().view(np.float64)
        view[:] = X[idx]

    def unpack(self, sweep, hl, src, buf, stream=None):
        if src == self.rank:
            return
        X = self.Rc if sweep else self.F
        idx = self._rows(hl, src)
        X[idx] = buf[16:16 + 8 * len(idx)].numpy().view(np.float64)

    def finish(self, post, lpd=None, stream=None):
        n, d = self.n, self.d
        full = (1 << n) - 1
        assert not np.isnan(self.F).any() and not np.isnan(self.Rc).any()
        P = post.numpy()
        P[:] = 0.0
        lpd_v = self.F[full]
        for v in range(n):
            if v % self.world != self.rank:
                continue
            rest = full ^ (1 << v)
            for f, G in enumerate(self.masks[v]):
                G = int(G)
                # Gamma_v(G): sum over G <= S <= V - {v} of F(S) R'(S + v),
                # S = G + X for every subset X of M = V - {v} - G
                M = rest & ~G
                terms = []
                X = 0
                while True:
                    S = G | X
                    terms.append(self.F[S] + self.Rc[S | (1 << v)])
                    if X == M:
                        break
                    X = ((X | ~M) + 1) & M
                gam = _lse(terms)
                self._acc.setdefault(v, {}).update({f: self.logB[v, f] + gam})
            for u in range(n):
                if u == v:
                    continue
                P[u, v] = np.exp(_lse([x for f, x in self._acc[v].items()
                                       if int(self.masks[v][f]) >> u & 1]) - lpd_v)
        if lpd is not None:
            lpd[0] = lpd_v


def _rank(rank, world, port, n, d, B, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import oracle as orc
    from paper_1408_1664_gb300 import datagen, shard as sh
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ds = datagen.random_dag_data(n=n, m=300, arity=2, max_parents=2, alpha=1.0, seed=11)
        ref = orc.edge_posteriors(ds.data, ds.arity, d, stages=("A", "F", "R", "logB", "masks"))
        s = CpuShard(n, d, B, ref["A"], ref["logB"], ref["masks"], rank, world)
        nb = sh.max_step_bytes(s)
        buf = torch.zeros(nb, dtype=torch.uint8)
        gathered = torch.zeros(world * nb, dtype=torch.uint8)
        post = torch.zeros((n, n), dtype=torch.float64)
        lpd = torch.zeros(1, dtype=torch.float64)
        sh.run_rank(s, dist, buf, gathered, post, lpd.numpy())
        full = (1 << n) - 1
        comp = full ^ np.arange(1 << n)
        out.put((rank,
                 float(np.abs(s.F - ref["F"]).max()),
                 float(np.abs(s.Rc - ref["R"][comp]).max()),
                 float(np.abs(post.numpy() - ref["post"]).max()),
                 abs(float(lpd[0]) - ref["log_PD"])))
    except Exception as e:                    # reported to the parent
        out.put((rank, repr(e)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_job_exchange_schedule_on_gloo_ranks(world):
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    n, d, B = 8, 2, 2
    procs = [mp.Process(target=_rank, args=(r, world, port, n, d, B, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for res in got:
        assert len(res) == 5, res
        rank, dF, dR, dpost, dlpd = res
        assert dF <= 1e-12 and dR <= 1e-12, (rank, dF, dR)
        assert dpost <= 1e-9, (rank, dpost)
        assert dlpd <= 1e-9 * n


def test_steps_pair_forward_and_backward_levels():
    sys.path.insert(0, ROOT)
    from paper_1408_1664_gb300 import shard as sh
    assert sh.steps(3) == [(0, 3), (1, 2), (2, 1), (3, 0)]
