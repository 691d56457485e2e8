import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Planted-mistake runs (test_oracle_mistakes.py) replace the oracle package by a copy in a
# temporary directory (its wrapper or its C source mutated, the library compiled beforehand).
# Unset in every other run.
_MUTANT_PKG = os.environ.get("STENCIL_ORACLE_MUTANT_PKG")
if _MUTANT_PKG:
    import importlib.util

    _spec = importlib.util.spec_from_file_location("oracle", os.path.join(_MUTANT_PKG, "__init__.py"),
                                                   submodule_search_locations=[_MUTANT_PKG])
    _mod = importlib.util.module_from_spec(_spec)
    sys.modules["oracle"] = _mod
    _spec.loader.exec_module(_mod)


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
