import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


# The tests load the testing build of the library (libbnedge_testing.so), which
# adds the stage-dump and count hooks of the header's BN_TESTING section.
os.environ.setdefault("BN_TESTING", "1")


# Under the BN_CHECK_BOUNDS debug build every GPU test also asserts that no
# index check of the kernels failed while it ran (tests/test_gpu_checked.py
# runs the small parity cases that way).
import pytest  # noqa: E402


@pytest.fixture(autouse=True)
def _index_checks(request):
    yield
    if os.environ.get("BN_CHECK_BOUNDS") == "1" and request.node.get_closest_marker("gpu"):
        from paper_1408_1664_gb300 import binding as B
        line, unit = B.bn_debug_bounds()
        assert (line, unit) == (0, 0), f"index check failed: unit {unit}, line {line}"
