import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libvne.so")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def vctx():
    """A libvne context on cuda:0 (GPU tests only)."""
    from paper_2212_09642_gb300 import _build, vne
    _build.build_all()
    ctx = vne.vne_ctx_create(0)
    yield ctx
    vne.vne_ctx_destroy(ctx)
