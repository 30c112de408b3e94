import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU run (minutes)")


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as o
    o.build()
    return o


# Measured errors of the parity tests, written to $LBM_PARITY_REPORT (JSON) at exit.
PARITY = {}


@pytest.fixture
def report(request):
    def rec(**kv):
        PARITY.setdefault(request.node.name, {}).update(
            {k: (float(v) if hasattr(v, "__float__") else v) for k, v in kv.items()})
    return rec


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("LBM_PARITY_REPORT")
    if path and PARITY:
        import json
        with open(path, "w") as f:
            json.dump(PARITY, f, indent=1, sort_keys=True)
