import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a GB300 GPU and the CUDA library (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long statistical test")


@pytest.fixture(scope="session", autouse=True)
def _build_cpu_helpers():
    import oracle
    import workloads
    oracle.build()
    workloads.build()


# Measured errors of the parity tests, written as JSON lines to the file
# named by SUSP_MEASURE_LOG (if set) when the session ends, so that each bar
# can be set to a stated multiple of the error it guards.
_MEASURED = []


@pytest.fixture
def record(request):
    def rec(name, value, bar=None):
        _MEASURED.append(dict(test=request.node.nodeid, name=name,
                              value=float(value),
                              bar=None if bar is None else float(bar)))
    return rec


def pytest_sessionfinish(session, exitstatus):
    path = os.environ.get("SUSP_MEASURE_LOG")
    if not path or not _MEASURED:
        return
    import json
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "a") as f:
        for m in _MEASURED:
            f.write(json.dumps(m) + "\n")
