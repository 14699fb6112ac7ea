import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and libvip.so")


@pytest.fixture(scope="session")
def vip():
    """The CUDA binding; builds libvip.so first (GPU tests only)."""
    import paper_1401_6513_gb300 as pkg
    pkg.build()
    return pkg.load()
