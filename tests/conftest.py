import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 and the compiled CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def mw():
    """The compiled library's binding (built in-tree if missing)."""
    lib = os.path.join(ROOT, "paper_2606_20863_gb300", "libmw.so")
    if not os.path.exists(lib):
        import __graft_entry__
        __graft_entry__.build()
    import paper_2606_20863_gb300 as mw
    return mw


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return torch.device("cuda:0")


def to_dev(x, dev):
    import numpy as np
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


# Worst observed |C - C_exact| / bound per workload, written as JSON to the
# path in MW_ERROR_REPORT at the end of the session (when set).
_WORST = {}


def record_worst(name, ratio):
    _WORST[name] = max(_WORST.get(name, 0.0), float(ratio))


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("MW_ERROR_REPORT")
    if path and _WORST:
        with open(path, "w") as f:
            json.dump(dict(sorted(_WORST.items())), f, indent=1)
