"""The no-allocation entry point, bn_edge_posteriors_static.

It exists for callers that cannot let a library allocate device memory:
host applications that own and partition all GPU memory themselves, and
loops that cannot pay for cudaMalloc or for the device-wide synchronisation
of cudaFree.  It keeps every intermediate array in one fixed device array
inside the library.  These
checks call it through the C ABI, twice in a row on different jobs (the
fixed array keeps the previous call's contents), and compare each result
with bn_edge_posteriors on the same job within the tolerances used for the
oracle parity tests (1e-9 on the FP64 path, 1e-4 on the FP32 path).  This
file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1408_1664_gb300 import binding as B
from paper_1408_1664_gb300 import datagen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.load(build_if_missing=True)
    return torch


def _static(torch, job, n, stream):
    post = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    lpd = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    B.bn_edge_posteriors_static(job, post, lpd, stream)
    stream.synchronize()
    return post.cpu().numpy(), float(lpd.item())


def test_static_matches_existing_entry_point_two_calls(torch_cuda):
    torch = torch_cuda
    small, d_small = datagen.config_small()                       # n=12, FP64
    other = datagen.random_dag_data(16, 400, 3, 3, 1.0, seed=77)  # n=16, FP32
    stream = torch.cuda.Stream()
    with B.Context(0) as ctx:
        want1, lpd1 = ctx.edge_posteriors(small.data, small.arity, d_small, precision="fp64")
        want2, lpd2 = ctx.edge_posteriors(other.data, other.arity, 3, precision="fp32")
    job1 = B.Job(small.data, small.arity, d_small, precision="fp64")
    data2 = torch.from_numpy(other.data).cuda()
    job2 = B.Job(data2, other.arity, 3, precision="fp32", m=other.m)
    got1, g1 = _static(torch, job1, small.n, stream)
    got2, g2 = _static(torch, job2, other.n, stream)
    np.testing.assert_allclose(got1, want1, atol=1e-9, rtol=0)
    assert abs(g1 - lpd1) <= 1e-9 * abs(lpd1)
    np.testing.assert_allclose(got2, want2, atol=1e-4, rtol=0)
    assert abs(g2 - lpd2) <= 1e-4 * abs(lpd2)
    # and once more on the first job after the second has overwritten the scratch
    again, _ = _static(torch, job1, small.n, stream)
    np.testing.assert_allclose(again, want1, atol=1e-9, rtol=0)


def test_static_with_per_size_prior(torch_cuda):
    """A per-size structure prior (log_rho) travels to the device in its own
    small table of the fixed array: same result as the existing entry point."""
    torch = torch_cuda
    ds = datagen.random_dag_data(11, 300, 2, 3, 1.0, seed=91)
    rho = [0.0, -0.7, -1.9, -3.3]
    stream = torch.cuda.Stream()
    with B.Context(0) as ctx:
        want, lpd = ctx.edge_posteriors(ds.data, ds.arity, 3, log_rho=rho, precision="fp64")
    got, g = _static(torch, B.Job(ds.data, ds.arity, 3, precision="fp64", log_rho=rho),
                     ds.n, stream)
    np.testing.assert_allclose(got, want, atol=1e-9, rtol=0)
    assert abs(g - lpd) <= 1e-9 * abs(lpd)


def test_static_rejects_jobs_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    big, d = datagen.config_large()                                # n=26 does not fit
    post = torch.zeros((big.n, big.n), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BnError) as ei:
        B.bn_edge_posteriors_static(B.Job(big.data, big.arity, d, precision="fp32"), post)
    assert ei.value.code == B.BN_ENOMEM
