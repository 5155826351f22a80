import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    # the C-ABI tests load the library; build it (nvcc cross-compiles) if it is missing
    lib = os.path.join(ROOT, "paper_1412_0595_gb300", "_build", "libsnn.so")
    if not os.path.exists(lib):
        import importlib.util
        spec = importlib.util.spec_from_file_location("_snn_build", os.path.join(ROOT, "paper_1412_0595_gb300", "build.py"))
        mod = importlib.util.module_from_spec(spec)
        spec.loader.exec_module(mod)
        mod.build()


@pytest.fixture(scope="session")
def gpu():
    """The CUDA library bound through its C-ABI; fails loudly when absent."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("test marked gpu but no CUDA device is visible")
    import paper_1412_0595_gb300 as snn
    return snn
