import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built kgpu library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def kgpu_lib():
    """The product library, built in-tree if needed (GPU tests only)."""
    import paper_1305_3345_gb300 as kg
    kg.ensure_built()
    return kg


@pytest.fixture(scope="session")
def ctx(kgpu_lib):
    """One library context on cuda:0 for the GPU tests."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = kgpu_lib.Context(0)
    yield c
    torch.cuda.synchronize()
    c.close()


def to_dev(a):
    """numpy uint8 -> CUDA uint8 tensor (copy)."""
    import torch
    return torch.from_numpy(a.copy()).cuda()


def to_np(t):
    return t.cpu().numpy()
