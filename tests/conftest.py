import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


@pytest.fixture(scope="session", autouse=True)
def _oracle_built():
    from oracle.build import build_oracle
    build_oracle()


@pytest.fixture(autouse=True)
def _device_status_clean(request):
    """Under the bounds-checking library (LCL_DEBUG_BOUNDS=1), every GPU test must leave no
    out-of-range index behind: lcl_last_device_status is LCL_OK after the test."""
    yield
    if os.environ.get("LCL_DEBUG_BOUNDS") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    import torch

    from paper_2501_14807_gb300 import lcl
    assert lcl.lcl_build_flags() & lcl.LCL_BUILD_BOUNDS_CHECKS, "the bounds-checking library is not the one loaded"
    torch.cuda.synchronize()
    st = lcl.lcl_last_device_status()
    assert st == 0, f"device status after {request.node.nodeid}: {lcl.lcl_status_str(st)}: {lcl.lcl_last_error()}"
