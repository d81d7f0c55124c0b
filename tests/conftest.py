import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
# keep torch's compile cache (created on import) inside the repository's ignored scratch
os.environ.setdefault("TORCHINDUCTOR_CACHE_DIR", os.path.join(ROOT, ".bench", "torchinductor"))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU-only test")


def pytest_collection_modifyitems(config, items):
    # run GPU tests in file order, the no-allocation entry point test last
    items.sort(key=lambda it: (os.path.basename(str(it.fspath)).startswith("test_zz"),))
