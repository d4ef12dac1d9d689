"""The oracle built with the undefined-behaviour sanitizer (gcc
-fsanitize=undefined, every finding fatal: signed overflow, shifts past the
width, out-of-bounds indexing of fixed arrays, misaligned access) passes every
oracle pin.  The CUDA side has no sanitizer on this pool; the oracle, which
decides parity, is checked this way on the CPU."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["test_oracle_ci.py", "test_oracle_xorlike.py", "test_oracle_mixing.py", "test_oracle_bbs.py",
        "test_oracle_bbs16.py", "test_oracle_bg.py", "test_oracle_naive.py", "test_oracle_seeding_stats.py"]


def _cc():
    return os.environ.get("CC") or shutil.which("gcc")


@pytest.mark.skipif(_cc() is None, reason="no host C compiler")
def test_oracle_pins_under_ubsan(tmp_path):
    so = tmp_path / "liboracle_ubsan.so"
    r = subprocess.run([_cc(), "-O1", "-g", "-std=c11", "-fPIC", "-shared", "-fsanitize=undefined",
                        "-fno-sanitize-recover=all", "-o", str(so), os.path.join(ROOT, "oracle", "ci_oracle.c")],
                       capture_output=True, text=True)
    if r.returncode != 0:
        pytest.skip("no UBSan runtime for this compiler: " + r.stderr[-300:])
    env = dict(os.environ, CI_ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x"] + [os.path.join(ROOT, "tests", p) for p in PINS],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, (r.stdout[-3000:], r.stderr[-3000:])
    assert "runtime error" not in r.stderr
