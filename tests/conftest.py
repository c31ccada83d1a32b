import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long CPU oracle runs")
    config.addinivalue_line("markers", "gpu_long: full-size GPU checks of many minutes, run on request (-m gpu_long)")


@pytest.fixture(scope="session")
def cuda_stream():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch.cuda.current_stream().cuda_stream


@pytest.fixture(scope="session")
def csw(cuda_stream):
    from paper_2106_06280_gb300 import build
    build.build()
    from paper_2106_06280_gb300 import cswdg
    return cswdg
