import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libsvr.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(x) for x in line.split()])
    return rows


_CACHE = {}


def cached(key, fn):
    if key not in _CACHE:
        _CACHE[key] = fn()
    return _CACHE[key]


@pytest.fixture(autouse=True)
def _index_checks(request):
    """With the SVR_DEBUG build loaded (SVR_DEBUG=1), every GPU test ends with
    an empty device index-check report."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    from paper_2412_04459_gb300 import _native as N
    if not N.DEBUG or N._LIB is None:
        return
    count, site, index, bound = N.debug_report()
    assert count == 0, f"device index checks failed {count} times; first: site {site}, index {index}, bound {bound}"
