import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "gpu_new: GPU test of a path whose first run on a GB300 is still "
                                       "pending; such tests run after all the others")


def pytest_collection_modifyitems(config, items):
    # keep the established GPU parity tests ahead of the not-yet-run ones, so
    # that a stop on the first failure (-x) never hides them
    items[:] = [it for it in items if "gpu_new" not in it.keywords] + \
        [it for it in items if "gpu_new" in it.keywords]
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
