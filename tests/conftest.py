import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a)")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def parity_log():
    """Record measured parity figures: appends one JSON object per call to
    the file named by ACR_PARITY_LOG (nothing when it is unset)."""
    import json
    path = os.environ.get("ACR_PARITY_LOG")

    def log(**rec):
        if path:
            with open(path, "a") as fh:
                fh.write(json.dumps(rec, default=float) + "\n")
    return log
