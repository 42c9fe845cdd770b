import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


_RECORDS = []


@pytest.fixture(scope="session")
def parity_record():
    """record(test, case, quantity, achieved, bound, **extra): keeps the error a
    parity test achieved next to the bound it was held to.  When the
    environment variable DG_PARITY_RECORD names a file, the records of the
    session are written there as JSON at its end."""
    def record(test, case, quantity, achieved, bound, **extra):
        r = {"test": test, "case": case, "quantity": quantity, "achieved": float(achieved),
             "bound": None if bound is None else float(bound)}
        r.update({k: (float(v) if isinstance(v, float) else v) for k, v in extra.items()})
        _RECORDS.append(r)
    return record


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("DG_PARITY_RECORD")
    if path and _RECORDS:
        os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
        with open(path, "w") as f:
            json.dump(_RECORDS, f, indent=1)
