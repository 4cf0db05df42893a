import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


def read_golden(name):
    """Rows of a golden fixture: (header key=value dict, list of int rows)."""
    header, rows = {}, []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            if "=" in line:
                for tok in line.split():
                    k, v = tok.split("=", 1)
                    header[k] = v
            else:
                rows.append([int(x) for x in line.split()])
    return header, rows


@pytest.fixture(scope="session")
def oracle_mod():
    """The oracle; PHPRNG_ORACLE_SO selects another compiled copy of it (the
    mutation test points it at copies with planted mistakes)."""
    import oracle
    alt = os.environ.get("PHPRNG_ORACLE_SO")
    return oracle.Oracle(alt) if alt else oracle._default()


@pytest.fixture(scope="session")
def ph():
    """The product binding with libphprng.so built for sm_103a (nvcc cross-
    compiles here; host-only entry points run without a GPU)."""
    from paper_1411_2484_gb300 import build
    build.build()
    import paper_1411_2484_gb300
    paper_1411_2484_gb300._load()
    return paper_1411_2484_gb300
