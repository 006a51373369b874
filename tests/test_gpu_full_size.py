"""Parity at the benchmark's full size: the n=26 workload (binary, d=4,
m=2000, the 2^26 subset lattice) against ONE full run of the CPU FP64 oracle,
entry by entry, and the served n=29 job (d=3, m=2000) FP32 against FP64.

Tolerances are the method's contract: edge posteriors within 1e-9 absolute
on the FP64 path and 1e-4 on the FP32 path (all n(n-1) = 650 of them here).
log P(D) = log F(V) (Algorithm 1) within 1e-9 relative on the FP64 path.  The
FP64 stage arrays F (Eq. 9) and R' (R'(T) = R(V-T), Eq. 10) are compared in
full, all 2^26 entries each, within 1e-9 absolute after undoing the per-node
shift the library applies (F(S) - sum_{j in S} c_j): a log-domain FP64 value
of magnitude below 1e5 carries rounding of about 1e-11 per level.

The FP32 run goes through bn_edge_posteriors_async with device-resident data
on a dedicated stream, the launch configuration the benchmark times.

The oracle at n=26 holds A (n 2^n doubles, 14 GB) plus per-thread scratch
of 4 * 2^n doubles; it runs when the host has that much memory available,
otherwise the test says "oracle skipped: RAM" and is skipped.  At n=29 the
oracle would need about 130 GB plus scratch and several minutes; it runs only
when the memory is there, and the FP32 path is always checked against the
GPU FP64 path, itself checked against the oracle at n=26 above.
"""
import time

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu


def mem_available() -> int:
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def oracle_bytes(n: int) -> int:
    """Peak host bytes of one oracle run: A, F, R and, per OpenMP thread, the
    four 2^n scratch arrays of the down-zeta loop."""
    N = 1 << n
    return 8 * (n * N + 2 * N + 4 * N * orc.num_threads())


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    c = B.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def oracle26():
    ds, d = datagen.config_large()
    need, have = oracle_bytes(ds.n), mem_available()
    if have < 1.2 * need:
        print(f"oracle skipped: RAM ({have / 2**30:.0f} GiB available, "
              f"{need / 2**30:.0f} GiB needed)")
        pytest.skip("oracle skipped: RAM")
    t0 = time.perf_counter()
    ref = orc.edge_posteriors(ds.data, ds.arity, d, stages=("F", "R"))
    print(f"oracle n=26: {time.perf_counter() - t0:.1f} s on {orc.num_threads()} threads")
    return ds, d, ref


def _csum(c: np.ndarray, n: int) -> np.ndarray:
    """sum_{j in S} c_j for every S of the 2^n lattice."""
    S = np.arange(1 << n, dtype=np.uint32)
    out = np.zeros(1 << n)
    for j in range(n):
        out += c[j] * ((S >> np.uint32(j)) & np.uint32(1))
    return out


def test_n26_fp64_posteriors_logPD_F_R_match_oracle(ctx, oracle26):
    ds, d, ref = oracle26
    n = ds.n
    post, lpd = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    err = float(np.abs(post - ref["post"]).max())
    print(f"n=26 FP64: max |post - oracle| = {err:.3e} over {n * (n - 1)} edges; "
          f"log P(D) {lpd:.10f} vs {ref['log_PD']:.10f}")
    np.testing.assert_allclose(post, ref["post"], atol=1e-9, rtol=0)
    assert abs(lpd - ref["log_PD"]) <= 1e-9 * abs(ref["log_PD"])
    c = B.bn_debug_stage(ctx.h, B.BN_STAGE_SHIFT, (n,), np.float64)
    N = 1 << n
    full = N - 1
    csum = _csum(c, n)
    F = B.bn_debug_stage(ctx.h, B.BN_STAGE_F, (N,), np.float64)
    dF = np.abs(F - (ref["F"] - csum))
    print(f"n=26 FP64: max |F - oracle| = {dF.max():.3e} over {N} subsets")
    assert float(dF.max()) <= 1e-9
    del F, dF
    Rc = B.bn_debug_stage(ctx.h, B.BN_STAGE_RC, (N,), np.float64)
    comp = full ^ np.arange(N, dtype=np.int64)
    dR = np.abs(Rc - (ref["R"][comp] - csum[comp]))
    print(f"n=26 FP64: max |R' - oracle| = {dR.max():.3e} over {N} subsets")
    assert float(dR.max()) <= 1e-9


def test_n26_fp32_bench_launch_config_matches_oracle(ctx, oracle26):
    torch = pytest.importorskip("torch")
    ds, d, ref = oracle26
    n = ds.n
    stream = torch.cuda.Stream()
    data_dev = torch.from_numpy(ds.data).cuda()
    post_dev = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    lpd_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    job = B.Job(data_dev, ds.arity, d, precision="fp32", m=ds.m)
    for _ in range(2):                    # the second run reuses the workspace, as the bench does
        B.bn_edge_posteriors_async(ctx.h, job, post_dev, lpd_dev, stream)
    stream.synchronize()
    post = post_dev.cpu().numpy()
    lpd = float(lpd_dev.item())
    err = float(np.abs(post - ref["post"]).max())
    print(f"n=26 FP32 (async, device data): max |post - oracle| = {err:.3e}; "
          f"log P(D) {lpd:.6f} vs {ref['log_PD']:.6f}")
    np.testing.assert_allclose(post, ref["post"], atol=1e-4, rtol=0)
    assert abs(lpd - ref["log_PD"]) < 1e-3 * n


@pytest.mark.parametrize("j", range(6))
def test_n29_served_job_fp32_vs_fp64(ctx, j):
    """The served workload's big jobs (n=29, d=3, m=2000, FP32 arrays of
    about 36 GB; one every 10 s of the 60 s trace): FP32 against the GPU FP64
    path at 1e-4, and against the oracle when the host has the memory for it.
    At this size the FP32 forward sums reach thousands in log2 units, which
    the per-level bases of F and R' keep near zero."""
    ds, d = datagen.served_job(j, big=True)
    p32, l32 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp32")
    p64, l64 = ctx.edge_posteriors(ds.data, ds.arity, d, precision="fp64")
    err = float(np.abs(p32 - p64).max())
    print(f"n=29 served job {j}: max |fp32 - fp64| = {err:.3e}")
    np.testing.assert_allclose(p32, p64, atol=1e-4, rtol=0)
    assert abs(l32 - l64) < 1e-3 * ds.n
    if j > 0:                             # the oracle, if at all, on the first of them
        return
    need, have = oracle_bytes(ds.n), mem_available()
    if have < 1.2 * need:
        print(f"oracle skipped: RAM ({have / 2**30:.0f} GiB available, "
              f"{need / 2**30:.0f} GiB needed)")
        return
    ref = orc.edge_posteriors(ds.data, ds.arity, d)
    np.testing.assert_allclose(p64, ref["post"], atol=1e-9, rtol=0)
    np.testing.assert_allclose(p32, ref["post"], atol=1e-4, rtol=0)
