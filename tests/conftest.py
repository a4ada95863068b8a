import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU case")
    config.addinivalue_line("markers", "late: run after every other test (a stop-at-first-failure run then "
                                       "has run all the others first)")


def pytest_collection_modifyitems(config, items):
    items[:] = sorted(items, key=lambda it: 1 if "late" in it.keywords else 0)  # stable: order kept otherwise
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)
