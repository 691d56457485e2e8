import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Planted-mistake runs (test_oracle_mistakes.py) point the oracle package at a mutated copy of
# its C source, compiled beforehand into a temporary directory.  Unset in every other run.
_MUTANT_SRC = os.environ.get("STENCIL_ORACLE_MUTANT_SRC")
if _MUTANT_SRC:
    import oracle as _oracle

    _oracle._SRC = _MUTANT_SRC
    _oracle._LIB = os.path.splitext(_MUTANT_SRC)[0] + ".so"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: minutes of CPU time (full-size oracle runs)")


@pytest.fixture(scope="session")
def cuda_lib():
    """The built CUDA library on a GPU machine; GPU tests fail loudly if it is missing."""
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but torch.cuda.is_available() is False")
    from paper_2406_08923_gb300 import _lib

    return _lib.load()
