import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def golden_lines(name):
    """Non-comment, non-empty lines of a golden fixture."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.lstrip().startswith("#")]


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(autouse=True)
def _bounds_checks_clean(request):
    """With the debug library loaded (IMPIR_BOUNDS=1), every GPU test must end with no failed
    index check in the kernels it ran."""
    yield
    if os.environ.get("IMPIR_BOUNDS") == "1" and request.node.get_closest_marker("gpu"):
        import paper_2509_06514_gb300 as impir
        st = impir.impir_bounds_status()
        assert st["n_failed"] == 0, f"failed index checks: {st}"
