"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer
on the GPU: the small-n parity, batch (graph and persistent forms, the
bounded-wait test), split-job, serving (its scheduler thread) and prior
tests run once more in a child process that loads the ASan build of the
library (_build/libbnedge_asan.so, host code instrumented) with the
sanitizer runtimes preloaded.  Any host out-of-bounds access,
use-after-free or undefined behaviour fails the test."""
import pytest

from test_sanitizers import run_under_sanitizers

pytestmark = pytest.mark.gpu


def test_gpu_tests_under_host_sanitizers():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    run_under_sanitizers(["tests/test_gpu_parity.py", "tests/test_gpu_batch.py",
                          "tests/test_gpu_shard.py", "tests/test_gpu_serving.py",
                          "tests/test_gpu_priors.py", "-k", "not large"], "gpu")
