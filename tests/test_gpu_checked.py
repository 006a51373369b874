"""The small-n parity, split-job and batch tests once more under the
BN_CHECK_BOUNDS debug build (_build/libbnedge_checked.so): the kernels check
every global offset they form against their arrays' sizes, and each test
then also asserts that no check failed (tests/conftest.py).  A failing check
records its line and redirects the access to offset 0, so an indexing error
shows up here as a failed assertion, not as a GPU fault."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

pytestmark = pytest.mark.gpu


def test_small_cases_under_index_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, BN_CHECK_BOUNDS="1", BN_TESTING="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_parity.py", "tests/test_gpu_shard.py", "tests/test_gpu_batch.py",
           "-k", "not large"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=3000)
    print(r.stdout[-4000:], r.stderr[-2000:])
    assert r.returncode == 0
