import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libns.so")


def gpu_available():
    try:
        import torch

        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def ns():
    """The ctypes binding over libns.so (GPU tests only)."""
    if not gpu_available():
        pytest.skip("no CUDA device")
    from paper_2603_08892_gb300 import binding

    return binding


@pytest.fixture
def report():
    """Record a measured error against the oracle: ``report(name, value, bound)`` appends one
    JSON line to the file named by the environment variable NS_ERROR_REPORT (nothing when it is
    unset), so that a GPU run leaves the table of errors per result behind."""
    import json

    path = os.environ.get("NS_ERROR_REPORT")

    def rec(name, value, bound=None, **extra):
        if not path:
            return
        with open(path, "a") as f:
            f.write(json.dumps(dict(name=name, value=float(value), bound=bound, **extra)) + "\n")

    return rec
