import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long CPU test (oracle physics runs)")


def read_table(name):
    """Rows of a whitespace golden table; '-' becomes None."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            out = []
            for tok in line.split():
                if tok == "-":
                    out.append(None)
                else:
                    try:
                        out.append(float(tok))
                    except ValueError:
                        out.append(tok)
            rows.append(out)
    return rows


@pytest.fixture(scope="session")
def cases():
    import json
    with open(os.path.join(GOLDEN, "cases.json")) as fh:
        return json.load(fh)
