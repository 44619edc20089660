import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_addoption(parser):
    parser.addoption("--fullsize", action="store_true", default=False,
                     help="also run the full-size workload tests (tens of minutes on one GB300)")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) GPU and the CUDA library")
    config.addinivalue_line("markers", "fullsize: full-size workloads (tens of minutes); run only with "
                                       "--fullsize or ANN_FULLSIZE=1")


def pytest_collection_modifyitems(config, items):
    """Full-size tests carry the gpu marker too, so a CPU run never selects
    them; a plain GPU run skips them unless asked for, which keeps it to a
    few minutes. Within a GPU run, the medium-size parity files come after
    the fast element-by-element files."""
    want = config.getoption("--fullsize") or os.environ.get("ANN_FULLSIZE") == "1"
    if not want:
        skip = pytest.mark.skip(reason="full-size workload: run with --fullsize or ANN_FULLSIZE=1")
        for it in items:
            if "fullsize" in it.keywords:
                it.add_marker(skip)


@pytest.fixture(scope="session")
def golden_dir():
    return GOLDEN
