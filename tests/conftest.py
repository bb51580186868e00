import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libpf")
    config.addinivalue_line("markers", "slow: long CPU runs of the checker")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def gpu():
    """CUDA device + built libpf; fails loudly if the library cannot be built or loaded."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2209_07969_gb300 import build, binding
    build.build()
    binding.lib()
    torch.cuda.init()
    return torch.device("cuda:0")
