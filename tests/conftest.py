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
