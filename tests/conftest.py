import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(scope="session")
def orc():
    from oracle import Oracle
    # BP_ORACLE_LIB points at a deliberately mutated build of the oracle
    # (tests/test_oracle_mutations.py) to show that the pins catch it.
    return Oracle(os.environ.get("BP_ORACLE_LIB") or None)


def read_golden(name: str) -> dict:
    """key: value lines of tests/golden/<name>, '#' lines are citations."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split(":", 1)
            out[k.strip()] = v.split()
    return out
