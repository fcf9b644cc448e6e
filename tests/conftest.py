import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running case")


def gpu_available():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture
def parity_log(request):
    """Returns log(**fields): appends one JSON line (the test id and the
    fields) to the file named by the environment variable CT_PARITY_REPORT,
    when it is set.  The solver tests record through it, per case, the
    iteration count, the oracle's own sensitivity, the tolerance in force and
    the error the GPU reached, so the tolerances can be audited case by
    case."""
    import json

    path = os.environ.get("CT_PARITY_REPORT")

    def log(**fields):
        if not path:
            return
        rec = {"test": request.node.nodeid}
        rec.update({k: (float(v) if hasattr(v, "dtype") else v) for k, v in fields.items()})
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")

    return log
