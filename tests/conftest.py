import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def _lib_is_stale():
    pkg = os.path.join(ROOT, "paper_2312_06567_gb300")
    lib = os.path.join(pkg, "libbgk.so")
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    srcs = [os.path.join(pkg, "csrc", f) for f in os.listdir(os.path.join(pkg, "csrc"))]
    srcs.append(os.path.join(ROOT, "include", "bgk.h"))
    return any(os.path.getmtime(s) > t for s in srcs)


@pytest.fixture(scope="session")
def libbgk():
    """The built C-ABI library (built in-tree first if missing or stale)."""
    if _lib_is_stale():
        from paper_2312_06567_gb300 import build
        build.build()
    from paper_2312_06567_gb300 import bgk
    return bgk.load()


@pytest.fixture(scope="session")
def cuda_device():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    torch.cuda.init()
    return torch.device("cuda:0")
