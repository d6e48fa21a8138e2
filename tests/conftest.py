"""Test configuration: the ``gpu`` marker and shared fixtures.

``-m "not gpu"`` runs the oracle pins, the host logic and the C-ABI symbol check on
the CPU; ``-m gpu`` runs the CUDA-path parity tests (they need a GPU and call the
library through its C ABI).
"""
import os
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU; compares the CUDA path to the oracle")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.lib()
    return oracle


def _cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@pytest.fixture(scope="session")
def native():
    """The CUDA library, loaded through its C ABI; GPU tests fail loudly without it."""
    if not _cuda_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    from paper_2308_10169_gb300 import _native
    return _native.lib()
