import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def _stale(lib, src_dirs):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    for d in src_dirs:
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")) and os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


@pytest.fixture(scope="session")
def libhh():
    """The CUDA library, (re)built in-tree with nvcc when missing or older than its sources."""
    from paper_2506_18694_gb300 import build, hh

    if _stale(build.LIB, [build.CSRC, os.path.join(ROOT, "include")]):
        build.build()
    return hh.load_library()
