import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


@pytest.fixture(scope="session")
def chamber():
    from paper_1911_09340_gb300 import synth
    return synth.make_chamber()


@pytest.fixture(scope="session")
def ctx():
    """A comet_ctx on cuda:0 (GPU tests only); builds the library first if needed."""
    from paper_1911_09340_gb300 import binding, build
    build.build()
    c = binding.Context(0)
    yield c
    c.close()
