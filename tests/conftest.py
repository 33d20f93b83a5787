import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle comparison")


@pytest.fixture(scope="session")
def aqt_lib():
    """The in-tree libaqt.so, compiled first if it is missing or older than its sources."""
    from paper_1710_03431_gb300 import build as B
    srcs = [os.path.join(B.CSRC, f) for f in os.listdir(B.CSRC)]
    if not os.path.exists(B.LIB) or max(os.path.getmtime(s) for s in srcs) > os.path.getmtime(B.LIB):
        B.build()
    from paper_1710_03431_gb300 import aqt
    aqt.lib()
    return aqt
