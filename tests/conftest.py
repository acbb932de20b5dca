import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(autouse=True)
def _bounds_checked_build(request):
    """Under the bounds-checked build (GRIN_CHECKED=1) every GPU test ends
    with the device synchronised and no out-of-range index recorded."""
    yield
    if os.environ.get("GRIN_CHECKED") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import ctypes
    import torch
    from paper_2606_22655_b300 import _native as N
    if not torch.cuda.is_available():
        return
    lib = N.load()
    assert lib.grin_build_checked() == 1
    torch.cuda.synchronize()
    site = ctypes.c_int32(-1)
    st = lib.grin_checked_status(0, ctypes.byref(site))
    assert st == 0 and site.value == 0, f"out-of-range index at site {site.value}"
