import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libzda.so")
    config.addinivalue_line("markers", "slow: long CPU test")


@pytest.fixture(scope="session", autouse=True)
def _libzda_built():
    """Build libzda.so (and the oracle) once if missing or stale, so that the
    package import (which loads the library and has no fallback) works."""
    import __graft_entry__
    b = __graft_entry__._build_module()
    srcs = [os.path.join(b.CSRC, s) for s in b.SOURCES] + [os.path.join(b.CSRC, f) for f in os.listdir(b.CSRC)
                                                          if f.endswith(".h")]
    srcs.append(os.path.join(ROOT, "include", "zda.h"))
    p = b.lib_path()
    if not os.path.exists(p) or os.path.getmtime(p) < max(os.path.getmtime(s) for s in srcs):
        b.build()
    yield
