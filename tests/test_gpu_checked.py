"""The bounds-checked debugging build (ci_check_status / ci_check_probe in
include/ci_prng.h).

Built with -DCI_CHECKED into libci_prng_checked.so, the generation, batched
and split kernels check their warp groups, output columns, store alignment,
batch units and split segments before each warp's work; a failed check is
recorded in a device status word and the warp skips the guarded work, so
nothing traps and no out-of-range access happens.  compute-sanitizer is not
available here, so this build is the memory check:

- the small-shape GPU parity suites run unchanged against the checked
  library (CI_PRNG_CHECKED=1 in a child process).  Every generation, split
  and batch call there returns CI_E_INVAL if any check failed, and the
  session ends by reading the status word once more (tests/conftest.py), so
  a pass means no check failed anywhere;
- a probe whose check fails on purpose is reported as CI_E_INVAL naming the
  probe, and the word is clear afterwards;
- the ordinary library has the checks compiled out and says so.
"""
import ctypes
import os
import subprocess
import sys

import pytest

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL_SUITES = ["tests/test_gpu_parity.py", "tests/test_gpu_split.py", "tests/test_gpu_batched.py",
                "tests/test_gpu_bbs16.py", "tests/test_gpu_tuning.py"]


def _checked_lib():
    from paper_1112_5239_gb300 import build

    return build.build(checked=True)


def _child(args, timeout):
    env = dict(os.environ, CI_PRNG_CHECKED="1")
    r = subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=timeout)
    return r.returncode, (r.stdout + r.stderr)[-3000:]


def test_small_shape_parity_suites_pass_under_the_checked_build():
    cuda_or_skip()
    _checked_lib()
    rc, tail = _child([sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"]
                      + SMALL_SUITES, timeout=1800)
    assert rc == 0, tail
    assert " passed" in tail and "error" not in tail.lower(), tail


PROBE = r"""
import ctypes, sys
sys.path.insert(0, %r)
from paper_1112_5239_gb300 import _lib
assert _lib.CHECKED and _lib.LIB_PATH.endswith("libci_prng_checked.so")
L = _lib.lib()
rc = L.ci_check_probe(None)
msg = L.ci_last_error()
assert rc == _lib.CI_E_INVAL and b"probe" in msg, (rc, msg)
w = ctypes.c_uint64(5)
assert L.ci_check_status(ctypes.byref(w), None) == _lib.CI_OK and w.value == 0, w.value
print("probe reported and cleared")
""" % ROOT


def test_probe_failure_is_reported_and_cleared():
    cuda_or_skip()
    _checked_lib()
    rc, tail = _child([sys.executable, "-c", PROBE], timeout=300)
    assert rc == 0 and "probe reported and cleared" in tail, tail


def test_ordinary_build_has_the_checks_compiled_out():
    cuda_or_skip()
    from paper_1112_5239_gb300 import _lib

    if _lib.CHECKED:
        pytest.skip("this process runs the checked build")
    w = ctypes.c_uint64(7)
    assert _lib.lib().ci_check_status(ctypes.byref(w), None) == _lib.CI_E_STATE and w.value == 0
    assert _lib.lib().ci_check_probe(None) == _lib.CI_E_STATE
