import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libeacg.so")


def ensure_library():
    """Build libeacg.so in-tree when it is missing (nvcc cross-compiles without a GPU)."""
    import importlib.util
    path = os.path.join(ROOT, "paper_2503_16225_gb300", "build.py")
    spec = importlib.util.spec_from_file_location("_eacg_build_for_tests", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.build()
