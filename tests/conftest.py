import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device and the built library")


def pytest_collection_modifyitems(config, items):
    """A bound on every test's wall time when pytest-timeout is present: a
    host-side hang (a blocked queue, a lock) fails that test instead of the
    whole run.  Tests that set their own timeout keep it."""
    if not config.pluginmanager.hasplugin("timeout"):
        return
    for item in items:
        if item.get_closest_marker("timeout") is None:
            item.add_marker(pytest.mark.timeout(600 if item.get_closest_marker("gpu") else 300))


@pytest.fixture(scope="session")
def lib():
    """The built CUDA library through its Python binding (GPU tests only)."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2211_00645_gb300 as opm
    opm.load()
    return opm
