import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: long CPU test")


def pytest_collection_finish(session):
    """Start the oracle for the full-size parity tests in the background, while the other
    GPU tests run (only when those tests are selected and a CUDA device is present)."""
    if not any("test_zy_fullsize" in item.nodeid for item in session.items):
        return
    try:
        import torch
    except ImportError:
        return
    if not torch.cuda.is_available():
        return
    import fullsize_support
    fullsize_support.start()


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("fullsize_support")
    if mod is not None:
        mod.stop()
