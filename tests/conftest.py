"""Test configuration: the `gpu` marker and the shared oracle fixture."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on the CPU")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


@pytest.fixture(scope="session", autouse=True)
def _checked_build_status_word():
    """Under the bounds-checked library (CI_PRNG_CHECKED=1, run by
    tests/test_gpu_checked.py), the device status word must still be clear
    when the session ends: a check that failed in any launch, including one
    whose entry point does not read the word itself, would have left it set."""
    yield
    if os.environ.get("CI_PRNG_CHECKED") != "1":
        return
    import ctypes

    import torch

    if not torch.cuda.is_available():
        return
    from paper_1112_5239_gb300 import _lib

    word = ctypes.c_uint64(0)
    rc = _lib.lib().ci_check_status(ctypes.byref(word), None)
    assert rc == _lib.CI_OK and word.value == 0, "bounds-check status word 0x%x" % word.value
