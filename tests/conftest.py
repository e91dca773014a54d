"""Shared pytest configuration: the ``gpu`` marker and common fixtures."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running test (minutes)")


@pytest.fixture
def parity_log(request):
    """record(quantity, measured, bound): the measured error of a result
    against the oracle and the bound the test asserts.  With ENS_PARITY_LOG
    set to a path, every record is appended there as one JSON line (test,
    quantity, measured, bound), so a run leaves the table of measured errors;
    without it the records go nowhere."""
    import json

    path = os.environ.get("ENS_PARITY_LOG")

    def record(quantity, measured, bound=None):
        if path:
            with open(path, "a") as f:
                f.write(json.dumps({"test": request.node.nodeid, "quantity": quantity,
                                    "measured": float(measured), "bound": bound}) + "\n")
        return measured

    return record
