import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer oracle runs")


@pytest.fixture(scope="session")
def gpulib():
    """Build (if stale) and load libmapgb300.so; skip when no CUDA device is present."""
    import ctypes
    try:
        cudart = None
        for name in ("libcudart.so", "libcudart.so.13", "libcudart.so.12"):
            try:
                cudart = ctypes.CDLL(name)
                break
            except OSError:
                continue
        n = ctypes.c_int(0)
        if cudart is None or cudart.cudaGetDeviceCount(ctypes.byref(n)) != 0 or n.value < 1:
            import torch
            if not torch.cuda.is_available():
                pytest.skip("no CUDA device")
    except Exception:
        pytest.skip("no CUDA device")
    from paper_1204_5849_gb300 import _build
    _build.build()
    import paper_1204_5849_gb300 as pkg
    return pkg.load()
