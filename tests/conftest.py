import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libpcbp.so")


@pytest.fixture(scope="session")
def oracle():
    import oracle as O

    O.lib()
    return O


@pytest.fixture(scope="session")
def pcbp():
    """The library binding; builds libpcbp.so first when it is missing or stale."""
    from paper_1911_08868_gb300 import _build

    _build.build()
    from paper_1911_08868_gb300 import pcbp as P

    return P


@pytest.fixture(scope="session")
def golden_dir():
    return ROOT / "tests" / "golden"


def gpu_device():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("GPU test run without a CUDA device")
    return torch.device("cuda", int(os.environ.get("PCBP_TEST_DEVICE", "0")))
