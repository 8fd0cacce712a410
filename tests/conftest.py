import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def ora():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _no_index_violation(request):
    """With a bounds-checked library (PSORT_LIB=.../libpsort_checked.so) every
    GPU test also fails if a kernel recorded an out-of-range index."""
    yield
    if request.node.get_closest_marker("gpu") is None or "checked" not in os.environ.get("PSORT_LIB", ""):
        return
    import ctypes
    from paper_2305_05245_gb300 import _lib
    out = (ctypes.c_uint64 * 4)()
    rc = _lib.load().ps_debug_violation(out)
    assert rc == 0, "kernel index violation: site %d index %d bound %d cta %d" % tuple(out)
