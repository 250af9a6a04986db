import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_sessionstart(session):
    # the package loads libdsm.so on import: build it first if it is missing
    lib = os.path.join(ROOT, "paper_2504_19941_gb300", "libdsm.so")
    if not os.path.exists(lib):
        import importlib.util
        spec = importlib.util.spec_from_file_location(
            "dsm_build", os.path.join(ROOT, "paper_2504_19941_gb300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libdsm")
    config.addinivalue_line("markers", "slow: long physics pin (still CPU, still run by default)")
