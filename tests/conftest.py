"""Shared pytest configuration: the `gpu` marker and repository import path."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running statistical check")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


@pytest.fixture(scope="session")
def gpu():
    """A CUDA device is required: GPU tests fail, never skip, without one."""
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    torch.cuda.init()
    from paper_2502_18624_gb300 import binding
    binding.load()
    return torch.device("cuda", 0)
