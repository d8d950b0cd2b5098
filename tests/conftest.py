import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the compiled library")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(autouse=True)
def _no_failed_range_check(request):
    """With FHD_CHECKED=1 (the checked build, every computed index range-checked): after each GPU test, no
    range check may have failed.  Tests that make a check fail on purpose take their own reading first."""
    yield
    if os.environ.get("FHD_CHECKED", "0") in ("", "0") or request.node.get_closest_marker("gpu") is None:
        return
    import torch
    if not torch.cuda.is_available():
        return
    import paper_2505_07158_gb300 as fhd
    rep = fhd.fhd_bounds_report()
    assert rep["count"] == 0, f"range checks failed: {rep}"
