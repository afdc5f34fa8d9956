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


def build_spp_lib():
    """Builds libspp.so (if stale) without importing the package, whose import
    needs the library."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2602_08642_gb300", "build_lib.py")
    spec = importlib.util.spec_from_file_location("spp_build_lib", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
