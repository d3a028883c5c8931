import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a) and the built libhm.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "plants_bad_index: feeds a deliberately out-of-range index to a kernel")


# HM_TEST_LIB=checked runs the session against libhm_checked.so (the same
# kernels with every index read from a device buffer checked before use) and
# requires, after each GPU test, that no check failed -- except in the tests
# that plant an out-of-range index on purpose.
CHECKED = os.environ.get("HM_TEST_LIB", "") == "checked"


def pytest_sessionstart(session):
    if CHECKED:
        from paper_2506_06988_b300 import lib
        lib.use(lib.load_checked())


@pytest.fixture(autouse=True)
def _checked_library_status(request):
    yield
    if CHECKED and request.node.get_closest_marker("gpu") is not None:
        from paper_2506_06988_b300 import lib
        st = lib.hm_checked_status(reset=True)
        if request.node.get_closest_marker("plants_bad_index") is None:
            assert st == 0, f"an index check of the checked library failed (status {st})"
