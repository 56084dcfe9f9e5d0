import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libd8")
    config.addinivalue_line("markers", "slow: large inputs (minutes of host time)")


@pytest.fixture(scope="session")
def d8():
    """The CUDA library binding; skips cleanly only when no GPU is present."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1605_05773_gb300 as lib

    lib.load()  # raises if the extension is missing: no fallback
    return lib
