import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


import pytest


@pytest.fixture(autouse=True)
def _workspace_guards(request):
    """After every GPU test: the guard words around every workspace region and
    basis vector of every live solver context are intact (no kernel wrote
    outside its region)."""
    yield
    if request.node.get_closest_marker("gpu") is None:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
        from paper_1810_00615_gb300 import AllAtOnce
    except Exception:  # noqa: BLE001 - no library, nothing to check
        return
    torch.cuda.synchronize()
    for a in AllAtOnce.live_instances():
        assert a.workspace_check() == 0, f"workspace guard damaged (n={a.n}, ell={a.ell})"
