import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def mmplib():
    """The native library, built in-tree if out of date.  Never a fallback:
    if it cannot be built or loaded the tests fail."""
    from paper_2310_11365_gb300 import build, mmp

    build.build()
    mmp.load()
    return mmp
