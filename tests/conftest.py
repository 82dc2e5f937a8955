import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device in this process")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(autouse=True)
def _guard_bands(request):
    """After every GPU test: the sentinel bands around the segments the test
    helpers allocated must be intact (no kernel wrote past a segment)."""
    yield
    if "gpu" not in request.keywords:
        return
    gu = sys.modules.get("tests.gpu_util")
    if gu is None:
        return
    bad = gu.check_guards()
    assert not bad, "guard band overwritten: " + "; ".join(bad)
