"""Shared fixtures.  `gpu` tests need a CUDA device and the built library;
everything else runs on the CPU (oracle pins, host logic, ABI exports)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and liblbm_gb300.so")
    config.addinivalue_line("markers", "slow: long CPU run (physics pins run to steady state)")


def cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def gpu_lib():
    if not cuda_available():
        pytest.skip("no CUDA device")
    from paper_1702_04910_gb300 import binding
    return binding.load()


@pytest.fixture(scope="session")
def lattice():
    from oracle import oracle
    return oracle.lattice()
