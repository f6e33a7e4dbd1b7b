import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the CUDA build of liblk.so")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def native_built():
    """Build liblk.so / liblk_fake.so in-tree (nvcc cross-compiles without a GPU)."""
    from paper_2310_01212_gb300 import build

    build.build()
    return build
