import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long CPU oracle runs")


@pytest.fixture(autouse=True)
def _device_index_checks(request):
    """Under SAPMG_LIBRARY=debug (the MG_DEBUG build), every GPU test must end
    with no failed device-side index check, and with the debug build loaded."""
    yield
    if os.environ.get("SAPMG_LIBRARY") != "debug" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_1202_2462_gb300 import binding
    if binding._lib is None:
        return
    n = binding.mg_debug_failures()
    assert n == 0, (f"{n} failed device-side index check(s) (-1: not the MG_DEBUG build): "
                    + binding.lib().mg_last_error().decode(errors="replace"))
